// Implicit-GEMM convolution on the 5th-generation tensor cores (tcgen05,
// sm_100+): the same "fprop" GEMM as igemm_fprop_kernel in nn_kernels.cu
// (C[m][n] = sum_k A[m][k] B^T[n][k], A gathered from an NHWC bf16 tensor by
// taps, B^T the bf16 weights with k contiguous; conv 3x3 forward and input
// gradient, transposed-conv forward and input gradient), with the same
// epilogues and split-k partials.
//
// Per CTA: a 128 x BN output tile (BN = 32 ... 256), k in steps of 64.
// 128 threads gather the A and B tiles with 16-byte cp.async into a 4-stage
// shared-memory ring laid out as 8 x 16-byte core matrices (no swizzle,
// K-major: core matrices 128 B apart along k, 1024 B apart along m / n).
// After a barrier one thread issues four tcgen05.mma (M = 128, N = BN,
// K = 16, BF16 x BF16 -> FP32) that accumulate in tensor memory and commits
// them to the stage's mbarrier; a stage is refilled once that mbarrier says
// its MMAs are done.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes / tile rows 32w .. 32w + 31).
//
// Waits are bounded (~1 s): on a timeout the CTA sets *err, waits for its
// own copies, frees its tensor memory and leaves.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "nn_internal.h"

namespace dhfwi {
namespace nn {
namespace {

constexpr int UBM = 128, UBK = 64, USTAGES = 4;
constexpr unsigned A_STAGE_BYTES = UBM * UBK * 2;  // 16 KB

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(unsigned dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Shared-memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1 (bit 46),
// base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// The same for a K-major operand written by TMA with the 128-byte swizzle:
// rows of 128 B (64 bf16 of k) in 8-row atoms of 1024 B (stride-byte offset
// 1024; the leading-byte offset is unused), layout type 2 (SWIZZLE_128B) in
// bits 61-63.  A K = 16 slice starts 32 B further along the row.
__device__ __forceinline__ uint64_t smem_desc_sw128(unsigned saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// MN-major operand in the 128-byte swizzle: rows of 128 B hold 64 elements
// along M / N, 8-row groups along K are 1024 B apart (stride-byte offset),
// 64-element blocks along M / N `block` bytes apart (leading-byte offset),
// layout type 2.  A K = 16 step starts 2048 B further.
__device__ __forceinline__ uint64_t smem_desc_sw128_mn(unsigned saddr, unsigned block) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((block >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t da, uint64_t db, uint32_t idesc, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __noinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try(bar, parity)) return true;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        for (int i = 0; i < 32; i++)
            if (mbar_try(bar, parity)) return true;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

// Byte offset of 16-byte chunk ch (k = 8 ch .. 8 ch + 7) of tile row r in a
// K-major core-matrix tile with 8 chunks per row.
__device__ __forceinline__ unsigned core_off(int r, int ch) { return ((r >> 3) * 8 + ch) * 128 + (r & 7) * 16; }

template <int BN>
constexpr size_t umma_smem() {
    return (size_t)USTAGES * (A_STAGE_BYTES + BN * UBK * 2) + 2048;  // + 1 KB alignment slack, barriers, TMEM address
}

template <int BN, int EPI>
__global__ void __launch_bounds__(128) igemm_umma_kernel(FpropArgs P) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    constexpr unsigned B_STAGE_BYTES = BN * UBK * 2;
    constexpr unsigned STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
    constexpr unsigned TMEM_COLS = BN < 32 ? 32 : BN;
    const unsigned sbase = (smem_u32(smraw) + 1023u) & ~1023u;
    unsigned char *tail = smraw + (sbase - smem_u32(smraw)) + USTAGES * STAGE_BYTES;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(tail);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 8 * USTAGES);
    const unsigned bar0 = smem_u32(bars);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UBM, n0 = blockIdx.y * BN;
    const int K = P.ntaps * P.C;
    const int nk_all = (K + UBK - 1) / UBK;
    const int per = (nk_all + gridDim.z - 1) / gridDim.z;
    const int kt0 = blockIdx.z * per;
    const int nk = max(0, min(nk_all, kt0 + per) - kt0);
    const int HWo = P.Ho * P.Wo;

    if (tid == 0) {
        for (int s = 0; s < USTAGES; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    // This thread's A chunks: rows tid/8 + 16 i (i = 0..7), chunk tid % 8.
    const int ach = tid & 7;
    int a_img[8], a_ho[8], a_wo[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = m0 + (tid >> 3) + 16 * i;
        const int mm = m < P.M ? m : -1;
        a_img[i] = mm < 0 ? -1 : mm / HWo;
        const int r = mm < 0 ? 0 : mm - a_img[i] * HWo;
        a_ho[i] = r / P.Wo;
        a_wo[i] = r - a_ho[i] * P.Wo;
    }
    auto load_stage = [&](int st, int kt) {
        const unsigned sa = sbase + st * STAGE_BYTES, sb = sa + A_STAGE_BYTES;
        const int k = (kt0 + kt) * UBK + ach * 8;
        const bool kin = k < K;
        const int tap = kin ? k / P.C : 0;
        const int c = k - tap * P.C;
        const int dh = P.dh[tap], dw = P.dw[tap];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int row = (tid >> 3) + 16 * i;
            const int hs = P.scale * a_ho[i] + dh, ws = P.scale * a_wo[i] + dw;
            const bool ok = kin && a_img[i] >= 0 && hs >= 0 && hs < P.Hs && ws >= 0 && ws < P.Ws;
            const __nv_bfloat16 *src =
                ok ? P.src + (((long long)a_img[i] * P.Hs + hs) * P.Ws + ws) * P.src_stride + P.src_off + c : P.src;
            cp16(sa + core_off(row, ach), src, ok);
        }
#pragma unroll
        for (int i = 0; i < BN / 16; i++) {
            const int idx = tid + 128 * i;
            const int row = idx >> 3, ch = idx & 7;
            const int n = n0 + row, kb = (kt0 + kt) * UBK + ch * 8;
            const bool ok = n < P.N && kb < K;
            cp16(sb + core_off(row, ch), ok ? P.bt + (long long)n * K + kb : P.bt, ok);
        }
    };

    constexpr uint32_t IDESC = idesc_bf16(UBM, BN);
    bool good = true;
#pragma unroll
    for (int s = 0; s < USTAGES - 1; s++) {
        if (s < nk) load_stage(s, s);
        cp_commit();
    }
    for (int kt = 0; kt < nk; kt++) {
        const int st = kt % USTAGES;
        cp_wait<USTAGES - 2>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // cp.async data -> tensor-core reads
        if (!__syncthreads_and(good)) break;  // a timed-out wait ends the loop for the whole CTA
        if (tid == 0) {
            tc_fence_after();
            const unsigned sa = sbase + st * STAGE_BYTES, sb = sa + A_STAGE_BYTES;
#pragma unroll
            for (int kk = 0; kk < UBK / 16; kk++)
                mma_bf16(tmem, smem_desc(sa + kk * 256, 128, 1024), smem_desc(sb + kk * 256, 128, 1024), IDESC,
                         (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar0 + 8 * st);
        }
        const int nxt = kt + USTAGES - 1;
        if (nxt < nk) {
            // Stage nxt % USTAGES was last read by the MMAs of k-tile kt - 1.
            if (kt >= 1) good = mbar_wait(bar0 + 8 * ((kt - 1) % USTAGES), ((kt - 1) / USTAGES) & 1u);
            if (good) load_stage(nxt % USTAGES, nxt);
        }
        cp_commit();
    }
    if (good && nk > 0) good = mbar_wait(bar0 + 8 * ((nk - 1) % USTAGES), ((nk - 1) / USTAGES) & 1u);
    cp_wait<0>();
    good = __syncthreads_and(good);
    tc_fence_after();

    if (!good) {
        if (tid == 0 && P.err) atomicExch(P.err, 1u);
    } else {
        const int m = m0 + warp * 32 + lane;
        const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
        int img = 0, ho = 0, wo = 0;
        if (EPI == EPI_BF16_CONVT && m < P.M) {
            img = m / HWo;
            const int r = m - img * HWo;
            ho = r / P.Wo;
            wo = r - ho * P.Wo;
        }
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            if (n0 + c0 >= P.N) break;  // uniform across the warp
            float v[16];
            if (nk > 0) tmem_ld16(trow + c0, v);
            else
#pragma unroll
                for (int q = 0; q < 16; q++) v[q] = 0.f;
            if (m >= P.M) continue;
            const int nb = n0 + c0;
            const bool full16 = nb + 16 <= P.N;
            if (P.part) {  // split-k: raw partial sums
                float *out = P.part + (long long)blockIdx.z * P.M * P.N + (long long)m * P.N + nb;
                if (full16 && (P.N & 3) == 0) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(out + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                } else {
                    #pragma unroll
                    for (int q = 0; q < 16; q++)
                        if (nb + q < P.N) out[q] = v[q];
                }
                continue;
            }
            if (EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) {
                __nv_bfloat16 *o = P.dst_bf16 + (long long)m * P.dst_stride + P.dst_off + nb;
                __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    float x = v[q] + (nb + q < P.N ? P.bias[nb + q] : 0.f);
                    if (EPI == EPI_BF16_LEAKY) x = x > 0.f ? x : P.slope * x;
                    h[q] = __float2bfloat16_rn(x);
                }
                if (full16 && ((P.dst_stride | P.dst_off) & 7) == 0) {
                    reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(h)[0];
                    reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(h)[1];
                } else {
                    #pragma unroll
                    for (int q = 0; q < 16; q++)
                        if (nb + q < P.N) o[q] = h[q];
                }
            } else if (EPI == EPI_BF16_CONVT) {
                // Columns tap-major: n = (2a + b) * Co + co -> output pixel (2ho+a, 2wo+b), channel co.
                const int Co = P.N >> 2;
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int n = nb + q;
                    if (n >= P.N) continue;
                    const int tap = n / Co, co = n - tap * Co, a = tap >> 1, b = tap & 1;
                    const long long pix = ((long long)img * (2 * P.Ho) + 2 * ho + a) * (2 * P.Wo) + 2 * wo + b;
                    P.dst_bf16[pix * P.dst_stride + P.dst_off + co] = __float2bfloat16_rn(v[q] + P.bias[co]);
                }
            } else if (EPI == EPI_BF16_LEAKYBWD) {
                const __nv_bfloat16 *ap = P.act + (long long)m * P.act_stride + P.act_off + nb;
                __nv_bfloat16 *o = P.dst_bf16 + (long long)m * P.dst_stride + P.dst_off + nb;
#pragma unroll
                for (int q = 0; q < 16; q++)
                    if (nb + q < P.N) {
                        const float av = __bfloat162float(ap[q]);
                        o[q] = __float2bfloat16_rn(v[q] * (av > 0.f ? 1.0f : P.slope));
                    }
            } else {  // EPI_F32 / EPI_F32_ADD
                float *o = P.dst_f32 + (long long)m * P.dst_stride + P.dst_off + nb;
#pragma unroll
                for (int q = 0; q < 16; q++)
                    if (nb + q < P.N) o[q] = (EPI == EPI_F32_ADD ? o[q] : 0.f) + v[q];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

template <int BN, int EPI>
void umma_launch(const FpropArgs &a, cudaStream_t s) {
    const size_t sm = umma_smem<BN>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(igemm_umma_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    const int tiles = ((a.M + UBM - 1) / UBM) * ((a.N + BN - 1) / BN);
    const int nk = (a.ntaps * a.C + UBK - 1) / UBK;
    int splits = 1;
    if (a.part && a.part_floats > 0) {
        // Split k when the tiles fill less than one wave, keeping at least 4
        // k-tiles per split and the partials within their buffer.
        const int want = (152 + tiles - 1) / tiles;
        splits = std::min(want, nk / 4);
        const long long cap = a.part_floats / ((long long)a.M * a.N);
        if (splits > cap) splits = (int)cap;
        if (splits < 2) splits = 1;
    }
    FpropArgs b = a;
    if (splits == 1) b.part = nullptr;
    dim3 grid((a.M + UBM - 1) / UBM, (a.N + BN - 1) / BN, splits);
    igemm_umma_kernel<BN, EPI><<<grid, 128, sm, s>>>(b);
    if (splits > 1) launch_fprop_reduce(b, EPI, splits, s);
}

// ---------------------------------------------------------------------------
// TMA-fed, warp-specialised tcgen05 implicit GEMM for the 3x3 convolutions
// (stride 1, same grid in and out, C a multiple of 32, N >= 64): the forward
// and input-gradient GEMMs of the double-conv blocks below the top level.
//
// Output tile: 128 pixels (BI images x BH rows x BW columns: 1 x 8 x 16, or
// 2 x 8 x 8 and 1 x 16 x 8 on grids at most 8 wide) by BN output channels.
// K runs over (tap, block of BK channels); a k-tile is one tap's BK
// channels, so its A operand is the source shifted by that tap, loaded as
// 4-D TMA boxes (channels, BW, BH, BI) that the TMA fills with zero outside
// the grid (the convolution's padding).  With BK = 64 one box of 64
// channels lands as 128 rows of 128 B in the 128-byte swizzled K-major
// layout (8-row atoms of 1024 B), and the weights B^T [N][K] as BN such rows.
// With BK = 32 (32-channel sources) one box per 16-byte k-chunk lands as 128
// rows of 16 B, a column of 8-row core matrices: the no-swizzle K-major
// layout with core matrices 128 B apart along m and k-chunks 2048 B apart
// (leading-byte offset 2048, stride-byte offset 128); the weights the same
// way, BN rows per k-chunk (leading-byte offset 16 BN).
//
// Warps: 0 = producer (one lane issues a stage's TMA loads once the MMAs
// that read it have completed), 1 = TMEM owner and MMA issuer (one lane),
// 2-5 = epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31).  Hand-off on
// mbarriers: full[s] (the stage's bytes landed), empty[s] (tcgen05.commit of
// the MMAs that read it), accf (the accumulator is final).  Waits are
// bounded (~1 s): the thread that runs out sets *err, the producer still
// waits for its loads in flight, and TMEM is freed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init1(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int c0, int c1, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

struct ConvTile {
    int BW, BH, BI;  // tile = BI images x BH rows x BW columns (128 pixels)
    int tw, th;      // tiles along w and h (then images)
    int nk_all;      // k-tiles over all taps
    int nimg;
};

constexpr int TMA_THREADS = 192;

template <int BN, int BK, int ST>
constexpr size_t conv3_tma_smem() {
    return (size_t)ST * (128 * BK * 2 + BN * BK * 2) + 2048;  // + alignment slack, barriers, TMEM address
}

// Epilogue of one 128 x BN output tile of the TMA-fed conv kernels: warp q
// of the four epilogue warps reads TMEM lanes 32 q .. 32 q + 31 (tile rows)
// of the accumulator whose column base is `tmem` (nk == 0: an empty k-range,
// zeros), columns [cbeg, cend) of it, and writes the rows with the epilogue
// EPI, or raw partial sums to P.part[split] when k is split.
template <int BN, int EPI>
__device__ __forceinline__ void conv_tile_epilogue(const FpropArgs &P, const ConvTile &G, unsigned tmem, int q, int lane,
                                                   int i0, int h0, int w0, int n0, int nk, int split, int cbeg = 0,
                                                   int cend = BN) {
    const int r = q * 32 + lane;  // tile row = TMEM lane
    const int per_img = G.BW * G.BH;
    const int img = i0 + r / per_img, rem = r % per_img;
    const int ho = h0 + rem / G.BW, wo = w0 + rem % G.BW;
    const bool valid = img < G.nimg && ho < P.Ho && wo < P.Wo;
    const long long m = ((long long)img * P.Ho + ho) * P.Wo + wo;
    const unsigned trow = tmem + ((unsigned)(q * 32) << 16);
#pragma unroll 1
    for (int c0 = cbeg; c0 < cend; c0 += 16) {
        if (n0 + c0 >= P.N) break;  // uniform across the warp
        const int nb = n0 + c0;
        const bool full16 = nb + 16 <= P.N;
        // The chunk's bias (bf16 epilogues) is requested before the TMEM
        // load, 16 bytes at a time where aligned, so that the two overlap.
        float bias16[16];
        if ((EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) && !P.part && valid) {
            if (full16 && ((uintptr_t)(P.bias + nb) & 15) == 0) {
#pragma unroll
                for (int e = 0; e < 16; e += 4) {
                    const float4 b4 = *reinterpret_cast<const float4 *>(P.bias + nb + e);
                    bias16[e] = b4.x;
                    bias16[e + 1] = b4.y;
                    bias16[e + 2] = b4.z;
                    bias16[e + 3] = b4.w;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++) bias16[e] = nb + e < P.N ? P.bias[nb + e] : 0.f;
            }
        }
        // Likewise the activation the LeakyReLU backward reads (16-byte path).
        __align__(16) __nv_bfloat16 act16[16];
        const __nv_bfloat16 *ap = P.act + m * P.act_stride + P.act_off + nb;
        __nv_bfloat16 *ob = P.dst_bf16 + m * P.dst_stride + P.dst_off + nb;
        const bool act_vec = EPI == EPI_BF16_LEAKYBWD && !P.part && valid && full16 &&
                             (((uintptr_t)ap | (uintptr_t)ob) & 15) == 0;
        if (act_vec) {
            reinterpret_cast<uint4 *>(act16)[0] = reinterpret_cast<const uint4 *>(ap)[0];
            reinterpret_cast<uint4 *>(act16)[1] = reinterpret_cast<const uint4 *>(ap)[1];
        }
        float v[16];
        if (nk > 0) tmem_ld16(trow + c0, v);
        else
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] = 0.f;
        if (!valid) continue;
        if (P.part) {  // split-k: raw partial sums
            float *out = P.part + (long long)split * P.M * P.N + m * P.N + nb;
            if (full16 && (P.N & 3) == 0) {
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                    *reinterpret_cast<float4 *>(out + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++)
                    if (nb + e < P.N) out[e] = v[e];
            }
            continue;
        }
        if (EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) {
            __nv_bfloat16 *o = P.dst_bf16 + m * P.dst_stride + P.dst_off + nb;
            __align__(16) __nv_bfloat16 h[16];
#pragma unroll
            for (int e = 0; e < 16; e++) {
                float x = v[e] + bias16[e];
                if (EPI == EPI_BF16_LEAKY) x = x > 0.f ? x : P.slope * x;
                h[e] = __float2bfloat16_rn(x);
            }
            if (full16 && ((P.dst_stride | P.dst_off) & 7) == 0) {
                reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(h)[0];
                reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(h)[1];
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++)
                    if (nb + e < P.N) o[e] = h[e];
            }
        } else if (EPI == EPI_BF16_CONVT) {
            // Transposed conv, columns tap-major: column n = (2a + b) Co + co
            // of coarse pixel (img, ho, wo) is fine pixel (2 ho + a, 2 wo + b),
            // channel co; with Co a multiple of 16 the 16 columns are 16
            // channels of one fine pixel (one 32-byte store).
            const int Co = P.N >> 2;
            const int tap = nb / Co, co = nb - tap * Co;
            const long long pix =
                ((long long)img * (2 * P.Ho) + 2 * ho + (tap >> 1)) * (2 * P.Wo) + 2 * wo + (tap & 1);
            __nv_bfloat16 *o = P.dst_bf16 + pix * P.dst_stride + P.dst_off + co;
            if (full16 && (Co & 15) == 0 && ((uintptr_t)o & 15) == 0) {
                __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                for (int e = 0; e < 16; e++) h[e] = __float2bfloat16_rn(v[e] + P.bias[co + e]);
                reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(h)[0];
                reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(h)[1];
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    const int n = nb + e;
                    if (n >= P.N) continue;
                    const int t2 = n / Co, c2 = n - t2 * Co;
                    const long long px =
                        ((long long)img * (2 * P.Ho) + 2 * ho + (t2 >> 1)) * (2 * P.Wo) + 2 * wo + (t2 & 1);
                    P.dst_bf16[px * P.dst_stride + P.dst_off + c2] = __float2bfloat16_rn(v[e] + P.bias[c2]);
                }
            }
        } else if (EPI == EPI_BF16_LEAKYBWD) {
            __nv_bfloat16 *o = ob;
            if (act_vec) {  // 16-byte loads (issued above) and stores
                __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                for (int e = 0; e < 16; e++)
                    h[e] = __float2bfloat16_rn(v[e] * (__bfloat162float(act16[e]) > 0.f ? 1.0f : P.slope));
                reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(h)[0];
                reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(h)[1];
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++)
                    if (nb + e < P.N) {
                        const float av = __bfloat162float(ap[e]);
                        o[e] = __float2bfloat16_rn(v[e] * (av > 0.f ? 1.0f : P.slope));
                    }
            }
        } else {  // EPI_F32 / EPI_F32_ADD
            float *o = P.dst_f32 + m * P.dst_stride + P.dst_off + nb;
            if (full16 && ((uintptr_t)o & 15) == 0) {  // 16-byte loads and stores
#pragma unroll
                for (int e = 0; e < 16; e += 4) {
                    float4 x = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    if (EPI == EPI_F32_ADD) {
                        const float4 y = *reinterpret_cast<const float4 *>(o + e);
                        x.x += y.x;
                        x.y += y.y;
                        x.z += y.z;
                        x.w += y.w;
                    }
                    *reinterpret_cast<float4 *>(o + e) = x;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; e++)
                    if (nb + e < P.N) o[e] = (EPI == EPI_F32_ADD ? o[e] : 0.f) + v[e];
            }
        }
    }
}

template <int BN, int BK, int ST, int EPI>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    conv3_tma_umma_kernel(FpropArgs P, const __grid_constant__ CUtensorMap mapA,
                          const __grid_constant__ CUtensorMap mapB, ConvTile G) {
    // BK = 64: 128-byte rows, swizzled; BK = 32: 16-byte k-chunks, no swizzle.
    constexpr bool SW128 = BK == 64;
    constexpr unsigned A_CH = 128 * 16, B_CH = BN * 16;  // bytes of one 16-byte k-chunk (no swizzle)
    constexpr unsigned A_BYTES = A_CH * (BK / 8), B_BYTES = B_CH * (BK / 8), STAGE = A_BYTES + B_BYTES;
    constexpr unsigned TMEM_COLS = BN;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const unsigned sbase = (smem_u32(smraw) + 1023u) & ~1023u;
    unsigned char *tail = smraw + (sbase - smem_u32(smraw)) + ST * STAGE;
    const unsigned full0 = smem_u32(tail), empty0 = full0 + 8 * ST, accf = empty0 + 8 * ST;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 16 * ST + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int t = blockIdx.x;
    const int w0 = (t % G.tw) * G.BW;
    t /= G.tw;
    const int h0 = (t % G.th) * G.BH;
    const int i0 = (t / G.th) * G.BI;
    const int n0 = blockIdx.y * BN;
    const int per = (G.nk_all + gridDim.z - 1) / gridDim.z;
    const int kt0 = blockIdx.z * per;
    const int nk = max(0, min(G.nk_all, kt0 + per) - kt0);

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init1(full0 + 8 * s);
            mbar_init1(empty0 + 8 * s);
        }
        mbar_init1(accf);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % ST;
                if (kt >= ST && !mbar_wait(empty0 + 8 * s, ((kt / ST) - 1) & 1u)) {
                    if (P.err) atomicExch(P.err, 1u);
                    break;
                }
                const unsigned fb = full0 + 8 * s;
                mbar_expect_tx(fb, STAGE);
                const int k = (kt0 + kt) * BK;
                const int tap = k / P.C, c0 = k - tap * P.C;
                const int ws = w0 + P.dw[tap], hs = h0 + P.dh[tap];
                const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
                if constexpr (SW128) {  // one 128-byte-wide box per operand
                    tma_load_4d(sa, &mapA, c0, ws, hs, i0, fb);
                    tma_load_2d(sb, &mapB, k, n0, fb);
                } else {  // one box per 16-byte k-chunk
#pragma unroll
                    for (int ch = 0; ch < BK / 8; ch++)
                        tma_load_4d(sa + ch * A_CH, &mapA, c0 + 8 * ch, ws, hs, i0, fb);
#pragma unroll
                    for (int ch = 0; ch < BK / 8; ch++) tma_load_2d(sb + ch * B_CH, &mapB, k + 8 * ch, n0, fb);
                }
                issued = kt + 1;
            }
            // Loads in flight land before the CTA leaves (bounded as well).
            for (int kt = max(0, issued - ST); kt < issued; kt++) mbar_wait(full0 + 8 * (kt % ST), (kt / ST) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(UBM, BN);
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % ST;
                if (!mbar_wait(full0 + 8 * s, (kt / ST) & 1u)) {
                    if (P.err) atomicExch(P.err, 1u);
                    break;
                }
                tc_fence_after();
                const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; kk++) {
                    const uint64_t da = SW128 ? smem_desc_sw128(sa + 32 * kk) : smem_desc(sa + 2 * kk * A_CH, A_CH, 128);
                    const uint64_t db = SW128 ? smem_desc_sw128(sb + 32 * kk) : smem_desc(sb + 2 * kk * B_CH, B_CH, 128);
                    mma_bf16(tmem, da, db, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accf);  // arrives once every MMA issued above is complete
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        const bool good = mbar_wait(accf, 0);
        tc_fence_after();
        if (!good) {
            if (lane == 0 && P.err) atomicExch(P.err, 1u);
        } else {
            conv_tile_epilogue<BN, EPI>(P, G, tmem, q, lane, i0, h0, w0, n0, nk, blockIdx.z);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// Persistent form of conv3_tma_umma_kernel (large GEMMs): grid = the SMs
// (times the CTAs that fit), each CTA walks the work items (m-tile, n-tile,
// k-split) with a stride of gridDim.x.  The stage ring runs on across items
// (one k-tile counter), and the accumulator is double-buffered in TMEM
// (2 x BN columns) so that the epilogue warps write item i while the MMAs of
// item i+1 run.  Hand-off on mbarriers: full[s] / empty[s] for the stages as
// before, tfull[b] (tcgen05.commit: accumulator b is final) and tempty[b]
// (arrived by each of the four epilogue warps once it has read accumulator
// b).  Every wait is bounded (~1 s); a role that runs out sets *err and the
// CTA's abort word, and every role leaves its loop at the next item; the
// producer still waits (bounded) for its loads in flight, and TMEM is freed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive1(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init_n(unsigned bar, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(n) : "memory");
}

template <int BN, int BK, int ST, int EPI>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    conv3_tma_persistent_kernel(FpropArgs P, const __grid_constant__ CUtensorMap mapA,
                                const __grid_constant__ CUtensorMap mapB, ConvTile G, int mt, int ntn, int splits) {
    constexpr bool SW128 = BK == 64;
    constexpr unsigned A_CH = 128 * 16, B_CH = BN * 16;
    constexpr unsigned A_BYTES = A_CH * (BK / 8), B_BYTES = B_CH * (BK / 8), STAGE = A_BYTES + B_BYTES;
    constexpr unsigned TMEM_COLS = 2 * BN;  // two accumulators; a power of two >= 64
    extern __shared__ __align__(1024) unsigned char smraw[];
    const unsigned sbase = (smem_u32(smraw) + 1023u) & ~1023u;
    unsigned char *tail = smraw + (sbase - smem_u32(smraw)) + ST * STAGE;
    const unsigned full0 = smem_u32(tail), empty0 = full0 + 8 * ST, tfull0 = empty0 + 8 * ST, tempty0 = tfull0 + 16;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 16 * ST + 32);
    volatile unsigned *abort_word = reinterpret_cast<volatile unsigned *>(tail + 16 * ST + 36);
    const unsigned drain = full0 + 16 * ST + 40;  // the MMA lane's last commit

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int items = mt * ntn * splits;
    const int per = (G.nk_all + splits - 1) / splits;
    // Item -> (m-tile, n-tile, split): n-tiles of one m-tile are adjacent (the
    // source tile is reused from L2), splits outermost.
    auto decode = [&](int item, int &i0, int &h0, int &w0, int &n0, int &kt0, int &nk, int &z) {
        const int n = item % ntn;
        int t = item / ntn;
        const int m = t % mt;
        z = t / mt;
        t = m;
        w0 = (t % G.tw) * G.BW;
        t /= G.tw;
        h0 = (t % G.th) * G.BH;
        i0 = (t / G.th) * G.BI;
        n0 = n * BN;
        kt0 = z * per;
        nk = max(0, min(G.nk_all, kt0 + per) - kt0);
    };

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init1(full0 + 8 * s);
            mbar_init1(empty0 + 8 * s);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init1(tfull0 + 8 * b);
            mbar_init_n(tempty0 + 8 * b, 4);
        }
        mbar_init1(drain);
        *abort_word = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    auto fail = [&]() {
        *abort_word = 1u;
        if (P.err) atomicExch(P.err, 1u);
    };

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;  // k-tiles issued by this CTA
            for (int item = blockIdx.x; item < items && !*abort_word; item += gridDim.x) {
                int i0, h0, w0, n0, kt0, nk, z;
                decode(item, i0, h0, w0, n0, kt0, nk, z);
                bool ok = true;
                for (int kt = 0; kt < nk; kt++, g++) {
                    const int s = g % ST;
                    if (g >= ST && !mbar_wait(empty0 + 8 * s, ((g / ST) - 1) & 1u)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const unsigned fb = full0 + 8 * s;
                    mbar_expect_tx(fb, STAGE);
                    const int k = (kt0 + kt) * BK;
                    const int tap = k / P.C, c0 = k - tap * P.C;
                    const int ws = w0 + P.dw[tap], hs = h0 + P.dh[tap];
                    const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
                    if constexpr (SW128) {
                        tma_load_4d(sa, &mapA, c0, ws, hs, i0, fb);
                        tma_load_2d(sb, &mapB, k, n0, fb);
                    } else {
#pragma unroll
                        for (int ch = 0; ch < BK / 8; ch++)
                            tma_load_4d(sa + ch * A_CH, &mapA, c0 + 8 * ch, ws, hs, i0, fb);
#pragma unroll
                        for (int ch = 0; ch < BK / 8; ch++) tma_load_2d(sb + ch * B_CH, &mapB, k + 8 * ch, n0, fb);
                    }
                }
                if (!ok) break;
            }
            // Loads in flight land before the CTA leaves (bounded as well).
            for (int q = max(0, g - ST); q < g; q++) mbar_wait(full0 + 8 * (q % ST), (q / ST) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(UBM, BN);
            int g = 0, b = 0, use[2] = {0, 0};
            for (int item = blockIdx.x; item < items && !*abort_word; item += gridDim.x, b ^= 1) {
                int i0, h0, w0, n0, kt0, nk, z;
                decode(item, i0, h0, w0, n0, kt0, nk, z);
                // Accumulator b is free once the epilogue has read its last use.
                if (use[b] > 0 && !mbar_wait(tempty0 + 8 * b, (use[b] - 1) & 1u)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const unsigned acc = tmem + (unsigned)(b * BN);
                bool ok = true;
                for (int kt = 0; kt < nk; kt++, g++) {
                    const int s = g % ST;
                    if (!mbar_wait(full0 + 8 * s, (g / ST) & 1u)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; kk++) {
                        const uint64_t da =
                            SW128 ? smem_desc_sw128(sa + 32 * kk) : smem_desc(sa + 2 * kk * A_CH, A_CH, 128);
                        const uint64_t db =
                            SW128 ? smem_desc_sw128(sb + 32 * kk) : smem_desc(sb + 2 * kk * B_CH, B_CH, 128);
                        mma_bf16(acc, da, db, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(empty0 + 8 * s);
                }
                if (!ok) break;
                mma_commit(tfull0 + 8 * b);  // arrives once the item's MMAs are complete
                use[b]++;
            }
            // Every MMA issued is complete before TMEM is freed (after a
            // failure too; bounded).
            mma_commit(drain);
            mbar_wait(drain, 0);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        int b = 0, use[2] = {0, 0};
        for (int item = blockIdx.x; item < items; item += gridDim.x, b ^= 1) {
            int i0, h0, w0, n0, kt0, nk, z;
            decode(item, i0, h0, w0, n0, kt0, nk, z);
            const bool good = mbar_wait(tfull0 + 8 * b, use[b] & 1u);
            tc_fence_after();
            if (!__all_sync(0xffffffffu, good) || *abort_word) {
                if (lane == 0) fail();
                break;
            }
            conv_tile_epilogue<BN, EPI>(P, G, tmem + (unsigned)(b * BN), q, lane, i0, h0, w0, n0, nk, z);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(tempty0 + 8 * b);
            use[b]++;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// tcgen05 3x3 convolution with the input patch reused by all nine taps, for
// sources of 32 or 64 channels (the network's top levels, where a TMA box
// per tap re-reads the input nine times in 16-byte rows).  Output tile: 16
// rows x 8 columns of one image (128 pixels = the MMA's M), BN output
// channels.  The 18 x 10 input patch (the tile plus the 1-pixel ring) is
// staged once, channel-chunk-major: chunk c (8 channels, 16 B per pixel)
// holds the 180 pixels row after row.  For tap (dh, dw) the A operand is the
// patch window starting at pixel (1 + dh, 1 + dw): in the no-swizzle K-major
// layout its 8-row core matrices are the 8 pixels of one tile row, 16 B
// apart, the next tile row 10 pixels (160 B) further (stride-byte offset),
// the next 8 channels one chunk (2880 B) further (leading-byte offset); so
// one MMA per (tap, 16 channels) reads the shifted window in place.  The
// weights B^T [N][9 C] are staged as [k-chunk][n][8] (leading-byte offset
// 16 BN, stride-byte offset 128).  Loads: 16-byte cp.async by all threads
// with zero fill outside the grid (the padding); one thread issues the
// 9 C / 16 MMAs and commits them; the epilogue is conv_tile_epilogue's.
// The wait for the MMAs is bounded (~1 s) as in the other kernels.
// ---------------------------------------------------------------------------
constexpr int PT_H = 16, PT_W = 8, PP_H = PT_H + 2, PP_W = PT_W + 2, PP = PP_H * PP_W;  // 18 x 10 patch

template <int BN, int C>
constexpr size_t patch_smem() {
    return (size_t)(C / 8) * PP * 16 + (size_t)BN * 9 * C * 2 + 1024;  // + barrier, TMEM address, alignment
}

template <int BN, int C, int EPI>
__global__ void __launch_bounds__(128) conv3_patch_umma_kernel(FpropArgs P, ConvTile G) {
    constexpr int CH = C / 8;                           // 16-byte channel chunks
    constexpr unsigned CHUNK = PP * 16;                 // bytes of one chunk of the patch
    constexpr unsigned A_BYTES = CH * CHUNK, B_CH = BN * 16;
    constexpr int K = 9 * C;
    constexpr unsigned TMEM_COLS = BN < 32 ? 32 : BN;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const unsigned sa = (smem_u32(smraw) + 127u) & ~127u;
    const unsigned sb = sa + ((A_BYTES + 127u) & ~127u);
    unsigned char *tail = smraw + (sb - smem_u32(smraw)) + (size_t)(K / 8) * B_CH;
    const unsigned bar = smem_u32(tail);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int t = blockIdx.x;
    const int w0 = (t % G.tw) * PT_W;
    t /= G.tw;
    const int h0 = (t % G.th) * PT_H;
    const int i0 = t / G.th;
    const int n0 = blockIdx.y * BN;

    if (tid == 0) {
        mbar_init1(bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // The patch (zero outside the image) and the weights.
    for (int idx = tid; idx < CH * PP; idx += 128) {
        const int c = idx / PP, pix = idx - c * PP;
        const int hs = h0 - 1 + pix / PP_W, ws = w0 - 1 + pix % PP_W;
        const bool ok = hs >= 0 && hs < P.Hs && ws >= 0 && ws < P.Ws;
        const __nv_bfloat16 *src =
            ok ? P.src + (((long long)i0 * P.Hs + hs) * P.Ws + ws) * P.src_stride + P.src_off + 8 * c : P.src;
        cp16(sa + c * CHUNK + pix * 16, src, ok);
    }
    for (int idx = tid; idx < (K / 8) * BN; idx += 128) {
        const int kc = idx / BN, n = idx - kc * BN;
        const bool ok = n0 + n < P.N;
        cp16(sb + kc * B_CH + n * 16, ok ? P.bt + (long long)(n0 + n) * K + 8 * kc : P.bt, ok);
    }
    cp_commit();
    cp_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // cp.async data -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    if (tid == 0) {
        constexpr uint32_t IDESC = idesc_bf16(UBM, BN);
        int q = 0;
#pragma unroll 1
        for (int tap = 0; tap < 9; tap++) {
            const unsigned off = (unsigned)(((1 + P.dh[tap]) * PP_W + 1 + P.dw[tap]) * 16);
#pragma unroll
            for (int kk = 0; kk < C / 16; kk++, q++) {
                const uint64_t da = smem_desc(sa + 2 * kk * CHUNK + off, CHUNK, PP_W * 16);
                const uint64_t db = smem_desc(sb + (tap * (C / 8) + 2 * kk) * B_CH, B_CH, 128);
                mma_bf16(tmem, da, db, IDESC, q > 0 ? 1u : 0u);
            }
        }
        mma_commit(bar);
    }
    const bool good = mbar_wait(bar, 0);
    tc_fence_after();
    if (!__syncthreads_and(good)) {
        if (tid == 0 && P.err) atomicExch(P.err, 1u);
    } else {
        conv_tile_epilogue<BN, EPI>(P, G, tmem, warp, lane, i0, h0, w0, n0, 1, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

template <int BN, int C, int EPI>
void patch_launch(const FpropArgs &a, const ConvTile &G, cudaStream_t s) {
    const size_t sm = patch_smem<BN, C>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(conv3_patch_umma_kernel<BN, C, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    dim3 grid(G.tw * G.th * G.nimg, (a.N + BN - 1) / BN);
    conv3_patch_umma_kernel<BN, C, EPI><<<grid, 128, sm, s>>>(a, G);
}

template <int EPI>
bool patch_dispatch(const FpropArgs &a, const ConvTile &G, cudaStream_t s) {
    switch (a.C) {
    case 32: a.N <= 32 ? patch_launch<32, 32, EPI>(a, G, s) : patch_launch<64, 32, EPI>(a, G, s); return true;
    case 64: a.N <= 32 ? patch_launch<32, 64, EPI>(a, G, s) : patch_launch<64, 64, EPI>(a, G, s); return true;
    default: return false;
    }
}

bool launch_conv3_patch_persistent(const FpropArgs &a, const ConvTile &G, int epi, int mode, cudaStream_t s);

}  // namespace

// The patch kernel serves a 3x3 convolution (stride 1, shifts in {-1, 0, 1},
// same grid in and out) whose source has 32 or 64 channels (a 16-byte
// aligned slice) and whose output has 16..128 channels (N-tiles of 32 / 64):
// the persistent form from two waves of tiles on, else one tile per CTA.
// DHFWI_NN_PATCH=0 turns both off, =tile keeps the one-tile kernel,
// =persistent forces the persistent one on a small grid.  Returns false
// (nothing launched) when not applicable.
bool launch_conv3_patch(const FpropArgs &a, int epi, cudaStream_t s) {
    const char *e = getenv("DHFWI_NN_PATCH");
    if (e && strcmp(e, "0") == 0) return false;
    const int pmode = e && strcmp(e, "tile") == 0 ? 0 : e && strcmp(e, "persistent") == 0 ? 1 : 2;
    if (epi == EPI_BF16_CONVT || a.ntaps != 9 || a.scale != 1 || a.Ho != a.Hs || a.Wo != a.Ws) return false;
    if ((a.C != 32 && a.C != 64) || a.N < 16 || a.N > 128) return false;
    if (((a.src_stride | a.src_off) & 7) != 0) return false;
    if (((uintptr_t)(a.src + a.src_off) & 15) != 0 || ((uintptr_t)a.bt & 15) != 0) return false;
    for (int t = 0; t < 9; t++)
        if (a.dh[t] < -1 || a.dh[t] > 1 || a.dw[t] < -1 || a.dw[t] > 1) return false;
    const long long HW = (long long)a.Ho * a.Wo;
    if (HW <= 0 || a.M % HW != 0) return false;
    ConvTile G{};
    G.nimg = (int)(a.M / HW);
    G.BW = PT_W;
    G.BH = PT_H;
    G.BI = 1;
    G.tw = (a.Wo + PT_W - 1) / PT_W;
    G.th = (a.Ho + PT_H - 1) / PT_H;
    if ((long long)G.tw * G.th * G.nimg >= (1LL << 31)) return false;
    FpropArgs b = a;
    b.part = nullptr;  // the whole K in one tile: no split
    if (pmode != 0 && launch_conv3_patch_persistent(b, G, epi, pmode, s)) return true;
    switch (epi) {
    case EPI_BF16_LEAKY: return patch_dispatch<EPI_BF16_LEAKY>(b, G, s);
    case EPI_BF16: return patch_dispatch<EPI_BF16>(b, G, s);
    case EPI_F32: return patch_dispatch<EPI_F32>(b, G, s);
    case EPI_BF16_LEAKYBWD: return patch_dispatch<EPI_BF16_LEAKYBWD>(b, G, s);
    case EPI_F32_ADD: return patch_dispatch<EPI_F32_ADD>(b, G, s);
    default: return false;
    }
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tma_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

template <int BN, int BK, int EPI>
bool conv3_tma_launch(const FpropArgs &a, const ConvTile &G0, cudaStream_t s) {
    constexpr int ST = (BK == 32 ? 2 : 1) * (BN <= 128 ? 3 : 4);
    const size_t sm = conv3_tma_smem<BN, BK, ST>();
    EncodeTiledFn enc = tma_encoder();
    if (!enc) return false;
    ConvTile G = G0;
    G.nk_all = a.ntaps * a.C / BK;
    // A: the source [img][h][w][c] (channel stride src_stride, slice at
    // src_off), box (8, BW, BH, BI); B: the weights [N][K], box (8, BN).
    CUtensorMap ma, mb;
    {
        const cuuint64_t es = sizeof(__nv_bfloat16);
        cuuint64_t dims[4] = {(cuuint64_t)a.C, (cuuint64_t)a.Ws, (cuuint64_t)a.Hs, (cuuint64_t)G.nimg};
        cuuint64_t str[3] = {es * a.src_stride, es * a.src_stride * a.Ws, es * a.src_stride * a.Ws * a.Hs};
        const cuuint32_t inner = BK == 64 ? 64 : 8;
        const CUtensorMapSwizzle swz = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE;
        cuuint32_t box[4] = {inner, (cuuint32_t)G.BW, (cuuint32_t)G.BH, (cuuint32_t)G.BI}, estr[4] = {1, 1, 1, 1};
        if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a.src + a.src_off), dims, str, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        const cuuint64_t K = (cuuint64_t)a.ntaps * a.C;
        cuuint64_t dimsb[2] = {K, (cuuint64_t)a.N};
        cuuint64_t strb[1] = {es * K};
        cuuint32_t boxb[2] = {inner, (cuuint32_t)BN}, estrb[2] = {1, 1};
        if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.bt, dimsb, strb, boxb, estrb,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    static bool attr = false;
    static int wave = 152;  // CTAs resident at once
    if (!attr) {
        cudaFuncSetAttribute(conv3_tma_umma_kernel<BN, BK, ST, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv3_tma_umma_kernel<BN, BK, ST, EPI>, TMA_THREADS, sm);
        wave = std::max(1, nsm * occ);
        attr = true;
    }
    const int mt = G.tw * G.th * ((G.nimg + G.BI - 1) / G.BI);
    const int tiles = mt * ((a.N + BN - 1) / BN);
    int splits = 1;
    if (a.part && a.part_floats > 0) {
        // Split k when the tiles fill less than one wave (and no more than
        // one: a CTA that runs after the others doubles the time), keeping
        // at least 4 k-tiles per split and the partials within their buffer.
        const int want = std::max(1, wave / tiles);
        splits = std::min(want, G.nk_all / 4);
        const long long cap = a.part_floats / ((long long)a.M * a.N);
        if (splits > cap) splits = (int)cap;
        if (splits < 2) splits = 1;
    }
    FpropArgs b = a;
    if (splits == 1) b.part = nullptr;
    dim3 grid(mt, (a.N + BN - 1) / BN, splits);
    conv3_tma_umma_kernel<BN, BK, ST, EPI><<<grid, TMA_THREADS, sm, s>>>(b, ma, mb, G);
    if (splits > 1) launch_fprop_reduce(b, EPI, splits, s);
    return true;
}

// Stages of the persistent kernel: as many as fit in ~192 KB, at most 8.
template <int BN, int BK>
constexpr int persistent_stages() {
    constexpr int stage = 128 * BK * 2 + BN * BK * 2;
    return 196608 / stage > 8 ? 8 : 196608 / stage;
}

// Tensor maps of the conv3 GEMM's operands (see conv3_tma_launch).
template <int BK>
bool conv3_maps(const FpropArgs &a, const ConvTile &G, int BN, CUtensorMap *ma, CUtensorMap *mb) {
    EncodeTiledFn enc = tma_encoder();
    if (!enc) return false;
    const cuuint64_t es = sizeof(__nv_bfloat16);
    cuuint64_t dims[4] = {(cuuint64_t)a.C, (cuuint64_t)a.Ws, (cuuint64_t)a.Hs, (cuuint64_t)G.nimg};
    cuuint64_t str[3] = {es * a.src_stride, es * a.src_stride * a.Ws, es * a.src_stride * a.Ws * a.Hs};
    const cuuint32_t inner = BK == 64 ? 64 : 8;
    const CUtensorMapSwizzle swz = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE;
    cuuint32_t box[4] = {inner, (cuuint32_t)G.BW, (cuuint32_t)G.BH, (cuuint32_t)G.BI}, estr[4] = {1, 1, 1, 1};
    if (enc(ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a.src + a.src_off), dims, str, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t K = (cuuint64_t)a.ntaps * a.C;
    cuuint64_t dimsb[2] = {K, (cuuint64_t)a.N};
    cuuint64_t strb[1] = {es * K};
    cuuint32_t boxb[2] = {inner, (cuuint32_t)BN}, estrb[2] = {1, 1};
    return enc(mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.bt, dimsb, strb, boxb, estrb,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The persistent kernel's launch: same tiles and k-splits as
// conv3_tma_launch, one CTA per SM (its TMEM holds both accumulators).
template <int BN, int BK, int EPI>
bool conv3_persistent_launch(const FpropArgs &a, const ConvTile &G0, cudaStream_t s) {
    constexpr int ST = persistent_stages<BN, BK>();
    const size_t sm = conv3_tma_smem<BN, BK, ST>();
    ConvTile G = G0;
    G.nk_all = a.ntaps * a.C / BK;
    CUtensorMap ma, mb;
    if (!conv3_maps<BK>(a, G, BN, &ma, &mb)) return false;
    static bool attr = false;
    static int nsm = 0;
    if (!attr) {
        cudaFuncSetAttribute(conv3_tma_persistent_kernel<BN, BK, ST, EPI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        attr = true;
    }
    const int mt = G.tw * G.th * ((G.nimg + G.BI - 1) / G.BI);
    const int ntn = (a.N + BN - 1) / BN;
    const int tiles = mt * ntn;
    int splits = 1;
    if (a.part && a.part_floats > 0) {
        // Split k when the tiles fill less than one wave (no more than one
        // item per CTA: a CTA with two doubles the time), keeping at least 4
        // k-tiles per split and the partials within their buffer.
        const int want = std::max(1, nsm / tiles);
        splits = std::min(want, G.nk_all / 4);
        const long long cap = a.part_floats / ((long long)a.M * a.N);
        if (splits > cap) splits = (int)cap;
        if (splits < 2) splits = 1;
    }
    FpropArgs b = a;
    if (splits == 1) b.part = nullptr;
    const int items = tiles * splits;
    const int grid = std::min(items, nsm);
    conv3_tma_persistent_kernel<BN, BK, ST, EPI><<<grid, TMA_THREADS, sm, s>>>(b, ma, mb, G, mt, ntn, splits);
    if (splits > 1) launch_fprop_reduce(b, EPI, splits, s);
    return true;
}

// ---------------------------------------------------------------------------
// Persistent form of conv3_patch_umma_kernel (3x3 convolutions of 32- or
// 64-channel sources over many 16 x 8 output tiles, e.g. the top level of a
// batch of 128 x 128 patches): the weights of the CTA's BN output channels
// are staged once; the 18 x 10 input patches of its tiles (tile t =
// blockIdx.x, blockIdx.x + gridDim.x, ...) stream through a ring of ST
// stages, each patch as C / 8 TMA boxes (8 channels x 10 x 18 pixels, zero
// outside the image; one box = one 16-byte channel chunk of the patch,
// chunks 2944 B apart so that every box lands 128-byte aligned); and the
// accumulator is double-buffered in TMEM so that the epilogue of tile j
// overlaps the MMAs of tile j + 1 and the loads of the tiles after it.
// Roles and hand-off as in conv3_tma_persistent_kernel (warp 0 loads, warp
// 1 issues the 9 C / 16 MMAs of a tile), with eight epilogue warps (two per
// TMEM lane quarter, each writing half of the columns) for more stores in
// flight; every wait is bounded (~1 s).
// ---------------------------------------------------------------------------
constexpr unsigned PATCH_CHS = 2944;  // 180 pixels x 16 B rounded up to 128 B

template <int BN, int C>
constexpr int patchp_stages() {
    // Two CTAs per SM when at least three stages fit in ~110 KB, else one
    // CTA with up to five.
    constexpr int wbytes = 9 * C * BN * 2, stage = (C / 8) * (int)PATCH_CHS;
    return (110000 - wbytes) / stage >= 3 ? ((110000 - wbytes) / stage > 6 ? 6 : (110000 - wbytes) / stage)
                                          : ((195000 - wbytes) / stage > 5 ? 5 : (195000 - wbytes) / stage);
}

template <int BN, int C, int ST>
constexpr size_t patchp_smem() {
    return 128 + (size_t)ST * (C / 8) * PATCH_CHS + (size_t)9 * C * BN * 2 + (2 * ST + 6) * 8 + 64;
}

constexpr int PATCHP_THREADS = 320;  // loader, MMA issuer, 8 epilogue warps

template <int BN, int C, int ST, int EPI>
__global__ void __launch_bounds__(PATCHP_THREADS, 1)
    conv3_patch_persistent_kernel(FpropArgs P, const __grid_constant__ CUtensorMap mapX, ConvTile G, int T) {
    constexpr int CH = C / 8;
    constexpr unsigned STAGE = CH * PATCH_CHS, B_CH = BN * 16;
    constexpr int K = 9 * C;
    constexpr unsigned TMEM_COLS = 2 * BN;  // two accumulators (64 or 128 columns)
    extern __shared__ __align__(1024) unsigned char smraw[];
    const unsigned sa0 = (smem_u32(smraw) + 127u) & ~127u;
    const unsigned sb = sa0 + ST * STAGE;
    unsigned char *tail = smraw + (sb - smem_u32(smraw)) + (size_t)(K / 8) * B_CH;
    const unsigned full0 = smem_u32(tail), empty0 = full0 + 8 * ST, tfull0 = empty0 + 8 * ST, tempty0 = tfull0 + 16;
    const unsigned drain = tempty0 + 16;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 16 * ST + 40);
    volatile unsigned *abort_word = reinterpret_cast<volatile unsigned *>(tail + 16 * ST + 44);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * BN;
    auto decode = [&](int t, int &i0, int &h0, int &w0) {
        w0 = (t % G.tw) * PT_W;
        t /= G.tw;
        h0 = (t % G.th) * PT_H;
        i0 = t / G.th;
    };

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init1(full0 + 8 * s);
            mbar_init1(empty0 + 8 * s);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init1(tfull0 + 8 * b);
            mbar_init_n(tempty0 + 8 * b, 8);
        }
        mbar_init1(drain);
        *abort_word = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // The CTA's weights B^T [n0 .. n0 + BN)[9 C], as [k-chunk][n][8] (zero past N).
    for (int idx = tid; idx < (K / 8) * BN; idx += PATCHP_THREADS) {
        const int kc = idx / BN, n = idx - kc * BN;
        const bool ok = n0 + n < P.N;
        cp16(sb + kc * B_CH + n * 16, ok ? P.bt + (long long)(n0 + n) * K + 8 * kc : P.bt, ok);
    }
    cp_commit();
    cp_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // cp.async data -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    auto fail = [&]() {
        *abort_word = 1u;
        if (P.err) atomicExch(P.err, 1u);
    };

    if (warp == 0) {
        if (lane == 0) {
            int j = 0;  // patches issued by this CTA
            for (int t = blockIdx.x; t < T && !*abort_word; t += gridDim.x, j++) {
                const int s = j % ST;
                if (j >= ST && !mbar_wait(empty0 + 8 * s, ((j / ST) - 1) & 1u)) {
                    fail();
                    break;
                }
                int i0, h0, w0;
                decode(t, i0, h0, w0);
                const unsigned fb = full0 + 8 * s, sa = sa0 + s * STAGE;
                mbar_expect_tx(fb, CH * PP * 16);
#pragma unroll
                for (int c = 0; c < CH; c++) tma_load_4d(sa + c * PATCH_CHS, &mapX, 8 * c, w0 - 1, h0 - 1, i0, fb);
            }
            // Loads in flight land before the CTA leaves (bounded as well).
            for (int q = max(0, j - ST); q < j; q++) mbar_wait(full0 + 8 * (q % ST), (q / ST) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(UBM, BN);
            int j = 0, b = 0, use[2] = {0, 0};
            for (int t = blockIdx.x; t < T && !*abort_word; t += gridDim.x, j++, b ^= 1) {
                const int s = j % ST;
                // Accumulator b is free once the epilogue has read its last use.
                if (use[b] > 0 && !mbar_wait(tempty0 + 8 * b, (use[b] - 1) & 1u)) {
                    fail();
                    break;
                }
                if (!mbar_wait(full0 + 8 * s, (j / ST) & 1u)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const unsigned sa = sa0 + s * STAGE, acc = tmem + (unsigned)(b * BN);
                int q = 0;
#pragma unroll 1
                for (int tap = 0; tap < 9; tap++) {
                    const unsigned off = (unsigned)(((1 + P.dh[tap]) * PP_W + 1 + P.dw[tap]) * 16);
#pragma unroll
                    for (int kk = 0; kk < C / 16; kk++, q++) {
                        const uint64_t da = smem_desc(sa + 2 * kk * PATCH_CHS + off, PATCH_CHS, PP_W * 16);
                        const uint64_t db = smem_desc(sb + (tap * (C / 8) + 2 * kk) * B_CH, B_CH, 128);
                        mma_bf16(acc, da, db, IDESC, q > 0 ? 1u : 0u);
                    }
                }
                mma_commit(empty0 + 8 * s);  // the patch stage is free once these MMAs are done
                mma_commit(tfull0 + 8 * b);  // and the accumulator final
                use[b]++;
            }
            // Every MMA issued is complete before TMEM is freed (bounded).
            mma_commit(drain);
            mbar_wait(drain, 0);
        }
        __syncwarp();
    } else {
        // Warps 2-9: TMEM lane quarter warp % 4, column half (warp - 2) / 4.
        const int q = warp & 3, cb = ((warp - 2) >> 2) * (BN / 2);
        int b = 0, use[2] = {0, 0};
        for (int t = blockIdx.x; t < T; t += gridDim.x, b ^= 1) {
            int i0, h0, w0;
            decode(t, i0, h0, w0);
            const bool good = mbar_wait(tfull0 + 8 * b, use[b] & 1u);
            tc_fence_after();
            if (!__all_sync(0xffffffffu, good) || *abort_word) {
                if (lane == 0) fail();
                break;
            }
            conv_tile_epilogue<BN, EPI>(P, G, tmem + (unsigned)(b * BN), q, lane, i0, h0, w0, n0, 1, 0, cb,
                                        cb + BN / 2);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(tempty0 + 8 * b);
            use[b]++;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Launch of the persistent patch kernel: grid = (the CTAs that fit on the
// SMs, shared out over the N-tiles) x N-tiles; `small` (the forced mode
// DHFWI_NN_PATCH=persistent) caps it at 2 CTAs per N-tile so that every CTA
// walks many tiles (ring wrap-around and accumulator reuse).
template <int BN, int C, int EPI>
bool patchp_launch(const FpropArgs &a, const ConvTile &G, bool small, cudaStream_t s) {
    constexpr int ST = patchp_stages<BN, C>();
    const size_t sm = patchp_smem<BN, C, ST>();
    EncodeTiledFn enc = tma_encoder();
    if (!enc) return false;
    CUtensorMap mx;
    {
        const cuuint64_t es = sizeof(__nv_bfloat16);
        cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)a.Ws, (cuuint64_t)a.Hs, (cuuint64_t)G.nimg};
        cuuint64_t str[3] = {es * a.src_stride, es * a.src_stride * a.Ws, es * a.src_stride * a.Ws * a.Hs};
        cuuint32_t box[4] = {8, (cuuint32_t)PP_W, (cuuint32_t)PP_H, 1}, estr[4] = {1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a.src + a.src_off), dims, str, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    static bool attr = false;
    static int cap = 0;
    if (!attr) {
        cudaFuncSetAttribute(conv3_patch_persistent_kernel<BN, C, ST, EPI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        // All of the SM's unified memory as shared memory, so that two CTAs
        // of the smaller instances fit.
        cudaFuncSetAttribute(conv3_patch_persistent_kernel<BN, C, ST, EPI>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv3_patch_persistent_kernel<BN, C, ST, EPI>,
                                                      PATCHP_THREADS, sm);
        // The runtime's answer has come back as 1 where the launch's own
        // limits (registers, shared memory) allow 2: take the larger of it
        // and those limits, at most 2.
        cudaFuncAttributes fa{};
        int per_sm_smem = 0;
        cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (cudaFuncGetAttributes(&fa, conv3_patch_persistent_kernel<BN, C, ST, EPI>) == cudaSuccess &&
            fa.numRegs > 0 && per_sm_smem > 0) {
            const int by_regs = 65536 / (((fa.numRegs * 32 + 255) / 256 * 256) * (PATCHP_THREADS / 32));
            const int by_smem = per_sm_smem / (int)(sm + 1024);
            occ = std::max(occ, std::min(2, std::min(by_regs, by_smem)));
        }
        cudaGetLastError();
        cap = nsm * std::max(occ, 1);
        attr = true;
    }
    const int T = G.tw * G.th * G.nimg, ntn = (a.N + BN - 1) / BN;
    const int per_n = small ? 2 : std::max(1, cap / ntn);
    dim3 grid(std::min(T, per_n), ntn);
    conv3_patch_persistent_kernel<BN, C, ST, EPI><<<grid, PATCHP_THREADS, sm, s>>>(a, mx, G, T);
    return true;
}

// Waves of CTAs the one-tile patch kernel would need (tiles over resident
// CTAs); the persistent one is used from two waves on.
template <int EPI>
bool patchp_dispatch(const FpropArgs &a, const ConvTile &G, int mode, cudaStream_t s) {
    const bool small = mode == 1;
    if (mode == 2) {  // automatic: many tiles per SM
        const long long tiles = (long long)G.tw * G.th * G.nimg * ((a.N + 63) / 64);
        if (tiles < 2LL * 2 * 152) return false;
    }
    switch (a.C) {
    case 32: return a.N <= 32 ? patchp_launch<32, 32, EPI>(a, G, small, s) : patchp_launch<64, 32, EPI>(a, G, small, s);
    case 64: return a.N <= 32 ? patchp_launch<32, 64, EPI>(a, G, small, s) : patchp_launch<64, 64, EPI>(a, G, small, s);
    default: return false;
    }
}

// The persistent patch kernel for a GEMM launch_conv3_patch accepted (mode
// 1 forced, 2 automatic); false: not launched (the one-tile kernel runs).
bool launch_conv3_patch_persistent(const FpropArgs &a, const ConvTile &G, int epi, int mode, cudaStream_t s) {
    switch (epi) {
    case EPI_BF16_LEAKY: return patchp_dispatch<EPI_BF16_LEAKY>(a, G, mode, s);
    case EPI_BF16: return patchp_dispatch<EPI_BF16>(a, G, mode, s);
    case EPI_F32: return patchp_dispatch<EPI_F32>(a, G, mode, s);
    case EPI_BF16_LEAKYBWD: return patchp_dispatch<EPI_BF16_LEAKYBWD>(a, G, mode, s);
    case EPI_F32_ADD: return patchp_dispatch<EPI_F32_ADD>(a, G, mode, s);
    default: return false;
    }
}

// Kernel choice for a conv3 GEMM: DHFWI_NN_CONV=tile (one tile per CTA),
// =persistent, or unset: the persistent kernel when the GEMM has at least
// four waves of 128 x 128 output tiles (large layers, where the overlap of
// one tile's epilogue with the next tile's MMAs pays), else one tile per CTA
// (measured at least as fast on the small layers of the 128 x 128 patches).
int conv3_mode() {
    const char *e = getenv("DHFWI_NN_CONV");
    if (e && strcmp(e, "tile") == 0) return 0;
    if (e && strcmp(e, "persistent") == 0) return 1;
    return 2;
}
bool conv3_persistent(const FpropArgs &a) {
    const int m = conv3_mode();
    if (m != 2) return m == 1;
    const long long tiles = ((long long)a.M + 127) / 128 * ((a.N + 127) / 128);
    return tiles >= 4 * 152;
}

template <int EPI>
bool conv3_tma_dispatch(const FpropArgs &a, const ConvTile &G, cudaStream_t s) {
    if (conv3_persistent(a)) {
        if (a.C % 64 == 0) {
            if (a.N <= 32) return conv3_persistent_launch<32, 64, EPI>(a, G, s);
            if (a.N <= 64) return conv3_persistent_launch<64, 64, EPI>(a, G, s);
            if (a.N <= 128) return conv3_persistent_launch<128, 64, EPI>(a, G, s);
            return conv3_persistent_launch<256, 64, EPI>(a, G, s);
        }
        if (a.N <= 32) return conv3_persistent_launch<32, 32, EPI>(a, G, s);
        if (a.N <= 64) return conv3_persistent_launch<64, 32, EPI>(a, G, s);
        if (a.N <= 128) return conv3_persistent_launch<128, 32, EPI>(a, G, s);
        return conv3_persistent_launch<256, 32, EPI>(a, G, s);
    }
    // DHFWI_NN_CONV_BN=64|128 caps the N tile of the one-tile-per-CTA form.
    const char *bn = getenv("DHFWI_NN_CONV_BN");
    const int cap = bn ? atoi(bn) : 256;
    if (a.C % 64 == 0) {
        if (a.N <= 64 || cap <= 64) return conv3_tma_launch<64, 64, EPI>(a, G, s);
        if (a.N <= 128 || cap <= 128) return conv3_tma_launch<128, 64, EPI>(a, G, s);
        return conv3_tma_launch<256, 64, EPI>(a, G, s);
    }
    if (a.N <= 64 || cap <= 64) return conv3_tma_launch<64, 32, EPI>(a, G, s);
    if (a.N <= 128 || cap <= 128) return conv3_tma_launch<128, 32, EPI>(a, G, s);
    return conv3_tma_launch<256, 32, EPI>(a, G, s);
}

template <int EPI>
void umma_dispatch(const FpropArgs &a, cudaStream_t s) {
    if (a.N <= 32) umma_launch<32, EPI>(a, s);
    else if (a.N <= 64) umma_launch<64, EPI>(a, s);
    else if (a.N <= 128) umma_launch<128, EPI>(a, s);
    else umma_launch<256, EPI>(a, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3 convolution on tcgen05 (input channels ci and
// output channels co multiples of 32; a 32-channel tensor is read as 64
// channels, the TMA filling the missing half with zeros):
//   part[z][co][tap * ci + c] = sum over the pixels of split z of
//                               G[p][co] X[p + shift(tap)][c].
// The MMA's M = 128 rows are two (tap, 64-channel block) pairs of the input
// X, N = NB output channels of the output gradient G, K = pixels in blocks
// of 128 (the conv kernel's tile geometry).  Both operands arrive as 4-D TMA
// boxes (64 channels, BW, BH, BI) of the NHWC tensors (X shifted by the
// pair's tap, zero outside the grid), i.e. MN-major in the 128-byte
// swizzle: 64-channel blocks 16 KB apart (leading-byte offset 16384),
// 8-pixel groups 1024 B apart (stride-byte offset 1024), a K = 16 step
// 2048 B further.  Same warp roles, mbarrier hand-off and bounded waits as
// conv3_tma_umma_kernel.  The epilogue writes lane r's row (one input
// channel of one tap) for 16 output channels at a time, so a warp stores 32
// consecutive columns of part.  The CTAs of the first M tile also write the
// bias column (column nw: the sum of G's column over the split's pixels).
// ---------------------------------------------------------------------------
struct WgradTile {
    int BW, BH, BI, tw, th;
    int npb;        // pixel blocks in total
    int per;        // pixel blocks per split
    int pairs;      // (tap, 64-channel block) pairs: taps * ci / 64
    int nimg;
    int taps;       // 9 (3x3 conv, taps shifted by -1..1) or 1 (no shift: a transposed conv's
                    // gradient in space-to-depth layout)
};

template <int NB, int ST>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    wgrad_tma_umma_kernel(WgradArgs P, const __grid_constant__ CUtensorMap mapX,
                          const __grid_constant__ CUtensorMap mapG, WgradTile G) {
    constexpr unsigned BOX = 16384;  // 64 channels x 128 pixels of bf16
    constexpr unsigned A_BYTES = 2 * BOX, B_BYTES = (NB / 64) * BOX, STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const unsigned sbase = (smem_u32(smraw) + 1023u) & ~1023u;
    unsigned char *tail = smraw + (sbase - smem_u32(smraw)) + ST * STAGE;
    const unsigned full0 = smem_u32(tail), empty0 = full0 + 8 * ST, accf = empty0 + 8 * ST;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 16 * ST + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = 2 * blockIdx.x;  // first (tap, channel block) pair of this M tile
    const bool two = q0 + 1 < G.pairs;
    const int cbn = (P.ci + 63) / 64;  // 64-channel blocks of X (the last one zero-filled past ci)
    const int co0 = blockIdx.y * NB;
    const int pb0 = blockIdx.z * G.per;
    const int nk = max(0, min(G.npb, pb0 + G.per) - pb0);
    const unsigned stage_tx = (two ? 2 : 1) * BOX + B_BYTES;

    // The first M tile's CTAs also sum the output gradient's columns (the
    // bias gradient) from the staged G boxes: its four epilogue warps read
    // every stage too, so a stage is free after the MMAs' commit and their
    // four arrivals.
    const bool bias = blockIdx.x == 0;

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init1(full0 + 8 * s);
            mbar_init_n(empty0 + 8 * s, bias ? 5u : 1u);
        }
        mbar_init1(accf);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((unsigned)NB));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int tapv[2], cbv[2];
            for (int h = 0; h < 2; h++) {
                const int q = q0 + h < G.pairs ? q0 + h : q0;
                tapv[h] = q / cbn;
                cbv[h] = q - tapv[h] * cbn;
            }
            int issued = 0;
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % ST;
                if (kt >= ST && !mbar_wait(empty0 + 8 * s, ((kt / ST) - 1) & 1u)) {
                    if (P.err) atomicExch(P.err, 1u);
                    break;
                }
                const unsigned fb = full0 + 8 * s;
                mbar_expect_tx(fb, stage_tx);
                int b = pb0 + kt;
                const int w0 = (b % G.tw) * G.BW;
                b /= G.tw;
                const int h0 = (b % G.th) * G.BH;
                const int i0 = (b / G.th) * G.BI;
                const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
                for (int h = 0; h < (two ? 2 : 1); h++) {
                    const int t = tapv[h];
                    const int sw = G.taps == 9 ? t % 3 - 1 : 0, sh = G.taps == 9 ? t / 3 - 1 : 0;
                    tma_load_4d(sa + h * BOX, &mapX, cbv[h] * 64, w0 + sw, h0 + sh, i0, fb);
                }
#pragma unroll
                for (int j = 0; j < NB / 64; j++) tma_load_4d(sb + j * BOX, &mapG, co0 + 64 * j, w0, h0, i0, fb);
                issued = kt + 1;
            }
            for (int kt = max(0, issued - ST); kt < issued; kt++) mbar_wait(full0 + 8 * (kt % ST), (kt / ST) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // M = 128, N = NB, both operands MN-major (bits 15, 16).
            constexpr uint32_t IDESC = idesc_bf16(UBM, NB) | (1u << 15) | (1u << 16);
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % ST;
                if (!mbar_wait(full0 + 8 * s, (kt / ST) & 1u)) {
                    if (P.err) atomicExch(P.err, 1u);
                    break;
                }
                tc_fence_after();
                const unsigned sa = sbase + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < 8; kk++)
                    mma_bf16(tmem, smem_desc_sw128_mn(sa + 2048 * kk, BOX), smem_desc_sw128_mn(sb + 2048 * kk, BOX),
                             IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accf);
        }
        __syncwarp();
    } else {
        const int qw = warp & 3;
        if (bias) {
            // Thread t: channel pair cp (channels co0 + 2 cp, + 1) over the
            // pixel rows grp, grp + ngrp, ... of each 128-pixel block; the
            // G box rows are 128 B (64 channels) with 16-byte chunks
            // swizzled by the row's low three bits.
            constexpr int NP = NB / 2, NGRP = 128 / NP;
            const int t = qw * 32 + lane, cp = t % NP, grp = t / NP;
            const int c = 2 * cp, bx = c >> 6, cc = c & 63;
            float s0 = 0.f, s1 = 0.f;
            bool ok = true;
            for (int kt = 0; kt < nk; kt++) {
                const int s = kt % ST;
                if (!mbar_wait(full0 + 8 * s, (kt / ST) & 1u)) {
                    ok = false;
                    break;
                }
                const unsigned gb = sbase + s * STAGE + A_BYTES + bx * BOX;
#pragma unroll 4
                for (int p = grp; p < 128; p += NGRP) {
                    unsigned v;
                    asm volatile("ld.shared.b32 %0, [%1];"
                                 : "=r"(v)
                                 : "r"(gb + p * 128 + (((cc >> 3) ^ (p & 7)) << 4) + ((cc & 7) << 1)));
                    __nv_bfloat162 h;
                    memcpy(&h, &v, 4);
                    const float2 f = __bfloat1622float2(h);
                    s0 += f.x;
                    s1 += f.y;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive1(empty0 + 8 * s);
            }
            if (!ok && lane == 0 && P.err) atomicExch(P.err, 1u);
            // Groups summed in order; the bias column nw of this split's partial.
            float *red = reinterpret_cast<float *>(tail + 16 * ST + 64);
            red[2 * t] = s0;
            red[2 * t + 1] = s1;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (grp == 0) {
                float a0 = 0.f, a1 = 0.f;
                for (int g = 0; g < NGRP; g++) {
                    a0 += red[2 * (g * NP + cp)];
                    a1 += red[2 * (g * NP + cp) + 1];
                }
                float *out = P.part + (long long)blockIdx.z * P.M * P.N + P.nw;
                if (co0 + c < P.M) out[(long long)(co0 + c) * P.N] = a0;
                if (co0 + c + 1 < P.M) out[(long long)(co0 + c + 1) * P.N] = a1;
            }
        }
        const bool good = mbar_wait(accf, 0);
        tc_fence_after();
        if (!good) {
            if (lane == 0 && P.err) atomicExch(P.err, 1u);
        } else {
            const int r = qw * 32 + lane;
            const int q = q0 + (r >> 6);
            const int tap = q / cbn, cb = q - tap * cbn;
            // Rows past ci (a 32-channel X read as a 64-channel box) are zero.
            const bool valid = q < G.pairs && (r < 64 || two) && cb * 64 + (r & 63) < P.ci;
            const int n = tap * P.ci + cb * 64 + (r & 63);
            float *out = P.part + (long long)blockIdx.z * P.M * P.N + n;
            const unsigned trow = tmem + ((unsigned)(qw * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < NB; c0 += 16) {
                float v[16];
                if (nk > 0) tmem_ld16(trow + c0, v);
                else
#pragma unroll
                    for (int e = 0; e < 16; e++) v[e] = 0.f;
                if (!valid) continue;
#pragma unroll
                for (int e = 0; e < 16; e++)  // columns past M: a 32-channel G read as 64
                    if (co0 + c0 + e < P.M) out[(long long)(co0 + c0 + e) * P.N] = v[e];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)NB));
    }
}

template <int NB>
int wgrad_tma_launch(const WgradArgs &a, int max_splits, cudaStream_t s) {
    constexpr int ST = NB == 64 ? 4 : NB == 128 ? 3 : 2;
    const size_t sm = (size_t)ST * (2 * 16384 + (NB / 64) * 16384) + 2048 + 1024;  // + bias-sum scratch
    EncodeTiledFn enc = tma_encoder();
    if (!enc) return 0;
    WgradTile G{};
    G.nimg = a.nimg;
    G.BW = a.W > 8 ? 16 : 8;
    G.BI = (G.BW == 8 && a.H <= 8) ? 2 : 1;
    G.BH = 128 / (G.BW * G.BI);
    G.tw = (a.W + G.BW - 1) / G.BW;
    G.th = (a.H + G.BH - 1) / G.BH;
    G.npb = G.tw * G.th * ((a.nimg + G.BI - 1) / G.BI);
    G.taps = a.mode == WG_CONV ? 9 : 1;
    G.pairs = G.taps * ((a.ci + 63) / 64);
    const int mt = (G.pairs + 1) / 2, ntl = (a.M + NB - 1) / NB;
    const int tiles = mt * ntl;
    // One CTA per SM (~192 KB of stages): at most one wave, so that no CTA
    // runs after the others.
    int splits = std::max(1, 152 / tiles);
    splits = std::min(splits, std::max(1, G.npb / 4));
    splits = std::max(1, std::min(splits, max_splits));
    G.per = (G.npb + splits - 1) / splits;
    splits = (G.npb + G.per - 1) / G.per;
    CUtensorMap mx, mg;
    const cuuint64_t es = sizeof(__nv_bfloat16);
    cuuint32_t box[4] = {64, (cuuint32_t)G.BW, (cuuint32_t)G.BH, (cuuint32_t)G.BI}, estr[4] = {1, 1, 1, 1};
    {
        cuuint64_t dims[4] = {(cuuint64_t)a.ci, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.nimg};
        cuuint64_t str[3] = {es * a.x_stride, es * a.x_stride * a.W, es * a.x_stride * a.W * a.H};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a.x + a.x_off), dims, str, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return 0;
    }
    {
        cuuint64_t dims[4] = {(cuuint64_t)a.M, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.nimg};
        cuuint64_t str[3] = {es * a.g_stride, es * a.g_stride * a.W, es * a.g_stride * a.W * a.H};
        if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)a.g, dims, str, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return 0;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(wgrad_tma_umma_kernel<NB, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    // The 7 columns after the bias column are not written by the kernel.
    cudaMemsetAsync(a.part, 0, sizeof(float) * (size_t)splits * a.M * a.N, s);
    wgrad_tma_umma_kernel<NB, ST><<<dim3(mt, ntl, splits), TMA_THREADS, sm, s>>>(a, mx, mg, G);
    return splits;
}

// The TMA-fed kernel serves a GEMM when it is a 3x3 convolution (taps with
// shifts in {-1, 0, 1}, stride 1, same grid in and out) with C a multiple of
// 32, at least 64 output channels, 16-byte aligned operands and a row
// stride that is a multiple of 8 channels.  Returns false (nothing launched)
// otherwise.
bool launch_conv3_tma(const FpropArgs &a, int epi, cudaStream_t s) {
    // 32-channel outputs go to tcgen05 only when the persistent kernel is
    // forced (BN = 32); by default the shared-memory halo kernel takes them
    // (it reuses the input patch for all nine taps, measured 2x faster).
    const int min_n = conv3_mode() == 1 ? 32 : 64;
    // Also the transposed conv's forward GEMM: one tap without shift on the
    // coarse grid, scattered to the fine grid by the epilogue.
    const bool one_tap = a.ntaps == 1 && a.dh[0] == 0 && a.dw[0] == 0;
    if (getenv("DHFWI_NN_CONVT") && strcmp(getenv("DHFWI_NN_CONVT"), "mma") == 0 && epi == EPI_BF16_CONVT)
        return false;
    if ((epi == EPI_BF16_CONVT && !one_tap) || a.N < min_n || (a.ntaps != 9 && !one_tap) || a.scale != 1 ||
        a.Ho != a.Hs || a.Wo != a.Ws || a.C % 32 != 0 || a.C <= 0)
        return false;
    if (((a.src_stride | a.src_off) & 7) != 0) return false;
    if (((uintptr_t)(a.src + a.src_off) & 15) != 0 || ((uintptr_t)a.bt & 15) != 0) return false;
    for (int t = 0; t < 9; t++)
        if (a.dh[t] < -1 || a.dh[t] > 1 || a.dw[t] < -1 || a.dw[t] > 1) return false;
    const long long HW = (long long)a.Ho * a.Wo;
    if (HW <= 0 || a.M % HW != 0) return false;
    ConvTile G{};
    G.nimg = (int)(a.M / HW);
    G.BW = a.Wo > 8 ? 16 : 8;
    G.BI = (G.BW == 8 && a.Ho <= 8) ? 2 : 1;
    G.BH = 128 / (G.BW * G.BI);
    G.tw = (a.Wo + G.BW - 1) / G.BW;
    G.th = (a.Ho + G.BH - 1) / G.BH;
    switch (epi) {
    case EPI_BF16_LEAKY: return conv3_tma_dispatch<EPI_BF16_LEAKY>(a, G, s);
    case EPI_BF16: return conv3_tma_dispatch<EPI_BF16>(a, G, s);
    case EPI_F32: return conv3_tma_dispatch<EPI_F32>(a, G, s);
    case EPI_BF16_LEAKYBWD: return conv3_tma_dispatch<EPI_BF16_LEAKYBWD>(a, G, s);
    case EPI_F32_ADD: return conv3_tma_dispatch<EPI_F32_ADD>(a, G, s);
    case EPI_BF16_CONVT: return conv3_tma_dispatch<EPI_BF16_CONVT>(a, G, s);
    default: return false;
    }
}

// The tcgen05 weight gradient (the default; DHFWI_NN_WGRAD=mma or
// DHFWI_NN_GEMM=mma keep the mma.sync one) for WG_CONV, and WG_CONVT with a
// space-to-depth output gradient, with ci and co multiples of 32 and aligned
// operands.  Partials as igemm_wgrad_kernel's,
// bias column the sum of G's column.  Returns the number of splits written (0: not
// applicable, nothing launched).
int launch_wgrad_tma(const WgradArgs &a, int max_splits, cudaStream_t s) {
    const char *e = getenv("DHFWI_NN_WGRAD"), *g = getenv("DHFWI_NN_GEMM");
    if ((e && strcmp(e, "mma") == 0) || (g && strcmp(g, "mma") == 0)) return 0;
    // ci and co multiples of 32: a 32-channel operand is read as a 64-channel
    // TMA box whose upper half the copy fills with zeros (rows and columns the
    // epilogue does not write).
    // A transposed conv's weight gradient with its output gradient in
    // space-to-depth layout is the one-tap (unshifted) form of the same GEMM,
    // with the output's columns m = ab*Co + co as the reduction expects.
    const bool s2d = a.mode == WG_CONVT && a.g_s2d;
    if ((a.mode != WG_CONV && !s2d) || a.ci % 32 != 0 || a.M % 32 != 0 || a.ci <= 0 || a.M <= 0) return 0;
    if (a.nw != (s2d ? 1 : 9) * a.ci || a.N != a.nw + 8) return 0;
    if (((a.x_stride | a.x_off | a.g_stride) & 7) != 0) return 0;
    if ((((uintptr_t)(a.x + a.x_off)) | (uintptr_t)a.g) & 15) return 0;
    if ((long long)a.nimg * a.H * a.W >= (1LL << 31)) return 0;
    // N tile: 64 output channels for the short reductions of the narrower
    // layers (fewer than 64 blocks of 128 pixels and at most 512 output
    // channels, or fewer than 512 blocks and at most 256 channels: more
    // stages and CTAs in flight; the 128 x 128 patches' network
    // trained at 247 against 232 TFLOP/s with 64 everywhere), else at most
    // 128 (the full-image paper-size network: 683 against 659 TFLOP/s with
    // 256 and 630-637 with 64 on its wide layers, which then re-read their
    // input too often); DHFWI_NN_WGRAD_NB=64|128|256 caps it instead.
    const char *nb = getenv("DHFWI_NN_WGRAD_NB");
    const long long npb = ((long long)a.nimg * a.H * a.W + 127) / 128;
    const int nb_cap = nb ? atoi(nb) : ((a.M <= 512 && npb < 64) || (a.M <= 256 && npb < 512)) ? 64 : 128;
    if (a.M % 256 == 0 && nb_cap >= 256) return wgrad_tma_launch<256>(a, max_splits, s);
    if (a.M % 128 == 0 && nb_cap >= 128) return wgrad_tma_launch<128>(a, max_splits, s);
    return wgrad_tma_launch<64>(a, max_splits, s);
}

void launch_fprop_umma(const FpropArgs &a, int epi, cudaStream_t s) {
    switch (epi) {
    case EPI_BF16_LEAKY: umma_dispatch<EPI_BF16_LEAKY>(a, s); break;
    case EPI_BF16: umma_dispatch<EPI_BF16>(a, s); break;
    case EPI_BF16_CONVT: umma_dispatch<EPI_BF16_CONVT>(a, s); break;
    case EPI_F32: umma_dispatch<EPI_F32>(a, s); break;
    case EPI_BF16_LEAKYBWD: umma_dispatch<EPI_BF16_LEAKYBWD>(a, s); break;
    default: umma_dispatch<EPI_F32_ADD>(a, s); break;
    }
}

}  // namespace nn
}  // namespace dhfwi
