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
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int n = nb + q;
                    if (n >= P.N) continue;
                    // n = co*4 + a*2 + b -> output pixel (2ho+a, 2wo+b), channel co.
                    const int co = n >> 2, a = (n >> 1) & 1, b = n & 1;
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

template <int EPI>
void umma_dispatch(const FpropArgs &a, cudaStream_t s) {
    if (a.N <= 32) umma_launch<32, EPI>(a, s);
    else if (a.N <= 64) umma_launch<64, EPI>(a, s);
    else if (a.N <= 128) umma_launch<128, EPI>(a, s);
    else umma_launch<256, EPI>(a, s);
}

}  // namespace

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
