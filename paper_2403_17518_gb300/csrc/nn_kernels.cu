// Kernels of the deblurring network (Section 2.4 / Appendix A of arXiv
// 2403.17518): BF16 implicit-GEMM convolutions on the tensor cores with FP32
// accumulation (forward, input gradient, weight gradient; 3x3 and 2x2-stride-2
// transposed), average pooling, LeakyReLU backward, MSE, Adam with cosine
// annealing, and the image <-> patch plumbing.  Activations are NHWC bf16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "nn_internal.h"

namespace dhfwi {
namespace nn {

// ---------------------------------------------------------------------------
// PTX helpers: asynchronous copies, ldmatrix, mma.sync m16n8k16 bf16
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp16(void *smem, const void *gmem, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Implicit GEMM "fprop" form: C[m][n] = sum_k A[m][k] B[k][n].
//   m: output pixel (img, ho, wo) of an Ho x Wo grid;
//   k = tap * C + c: source pixel (img, scale*ho + dh[tap], scale*wo + dw[tap]),
//     channel c of a NHWC bf16 tensor (zero outside the source grid);
//   B^T[n][k] dense bf16 row-major (k contiguous).
// Covers: conv 3x3 forward (taps dh,dw in -1..1), conv 3x3 input gradient
// (taps 1-dh), transposed-conv forward (1 tap, n = (co,a,b)) and transposed-
// conv input gradient (scale 2, taps (a,b)).
// Tile 128 x BN x 32, 4 warps along m, 3-stage cp.async pipeline.
// ---------------------------------------------------------------------------
constexpr int BM = 128, BK = 32, STAGES = 3, SK = BK + 8;  // +8 halves: conflict-free ldmatrix

template <int BN>
struct FpropSmem {
    __nv_bfloat16 a[STAGES][BM][SK];
    __nv_bfloat16 b[STAGES][BN][SK];
};

template <int BN, int EPI>
__global__ void __launch_bounds__(128) igemm_fprop_kernel(FpropArgs P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FpropSmem<BN> &S = *reinterpret_cast<FpropSmem<BN> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int K = P.ntaps * P.C;
    const int nk_all = (K + BK - 1) / BK;
    // Split-k: this CTA takes k-tiles [kt0, kt0 + nk).
    const int per = (nk_all + gridDim.z - 1) / gridDim.z;
    const int kt0 = blockIdx.z * per;
    const int nk = max(0, min(nk_all, kt0 + per) - kt0);
    const int HWo = P.Ho * P.Wo;

    // Each thread loads fixed 16-byte chunks of the A and B tiles.
    // A: 128 rows x 4 chunks = 512 chunks -> 4 per thread; B: BN x 4.
    int a_img[4], a_ho[4], a_wo[4];
    bool a_ok[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int row = (tid + i * 128) >> 2;
        const int m = m0 + row;
        a_ok[i] = m < P.M;
        const int mm = a_ok[i] ? m : 0;
        a_img[i] = mm / HWo;
        const int r = mm - a_img[i] * HWo;
        a_ho[i] = r / P.Wo;
        a_wo[i] = r - a_ho[i] * P.Wo;
    }
    auto load_stage = [&](int st, int kt) {
        kt += kt0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int idx = tid + i * 128;
            const int row = idx >> 2, ch = idx & 3;
            const int k = kt * BK + ch * 8;
            bool ok = a_ok[i] && k < K;
            const __nv_bfloat16 *src = P.src;
            if (ok) {
                const int tap = k / P.C, c = k - tap * P.C;
                const int hs = P.scale * a_ho[i] + P.dh[tap], ws = P.scale * a_wo[i] + P.dw[tap];
                ok = hs >= 0 && hs < P.Hs && ws >= 0 && ws < P.Ws;
                if (ok) src = P.src + (((long long)a_img[i] * P.Hs + hs) * P.Ws + ws) * P.src_stride + P.src_off + c;
            }
            cp16(&S.a[st][row][ch * 8], src, ok);
        }
#pragma unroll
        for (int i = 0; i < (BN * 4 + 127) / 128; i++) {
            const int idx = tid + i * 128;
            if (idx < BN * 4) {
                const int row = idx >> 2, ch = idx & 3;
                const int n = n0 + row, k = kt * BK + ch * 8;
                const bool ok = n < P.N && k < K;
                cp16(&S.b[st][row][ch * 8], ok ? P.bt + (long long)n * K + k : P.bt, ok);
            }
        }
    };

    float acc[2][BN / 8][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < BN / 8; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;

#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if (s < nk) load_stage(s, s);
        cp_commit();
    }
    for (int kt = 0; kt < nk; kt++) {
        cp_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nxt = kt + STAGES - 1;
            if (nxt < nk) load_stage(nxt % STAGES, nxt);
            cp_commit();
        }
        const int st = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = warp * 32 + i * 16 + (lane & 15);
                ldsm_x4(af[i], &S.a[st][r][kk + (lane >> 4) * 8]);
            }
#pragma unroll
            for (int j = 0; j < BN / 8; j += 2) {
                unsigned bf[4];
                const int r = j * 8 + (lane & 7) + ((lane >> 4) << 3);
                ldsm_x4(bf, &S.b[st][r][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    mma16816(acc[i][j], af[i], bf[0], bf[1]);
                    mma16816(acc[i][j + 1], af[i], bf[2], bf[3]);
                }
            }
        }
    }
    cp_wait<0>();

    // Epilogue.
    const int g = lane >> 2, t = lane & 3;
    if (P.part) {  // split-k: raw partial sums, the epilogue runs in fprop_reduce_kernel
        float *out = P.part + (long long)blockIdx.z * P.M * P.N;
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int m = m0 + warp * 32 + i * 16 + g + half * 8;
                if (m >= P.M) continue;
#pragma unroll
                for (int j = 0; j < BN / 8; j++)
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int n = n0 + j * 8 + 2 * t + e;
                        if (n < P.N) out[(long long)m * P.N + n] = acc[i][j][half * 2 + e];
                    }
            }
        return;
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int m = m0 + warp * 32 + i * 16 + g + half * 8;
            if (m >= P.M) continue;
            const int img = m / HWo;
            const int r = m - img * HWo;
            const int ho = r / P.Wo, wo = r - ho * P.Wo;
#pragma unroll
            for (int j = 0; j < BN / 8; j++) {
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int n = n0 + j * 8 + 2 * t + e;
                    if (n >= P.N) continue;
                    float v = acc[i][j][half * 2 + e];
                    if (EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) {
                        v += P.bias[n];
                        if (EPI == EPI_BF16_LEAKY) v = v > 0.f ? v : P.slope * v;
                        const long long o = (long long)m * P.dst_stride + P.dst_off + n;
                        P.dst_bf16[o] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_BF16_CONVT) {
                        // Columns tap-major: n = (2a + b) * Co + co -> output pixel
                        // (2ho+a, 2wo+b), channel co.
                        const int Co = P.N >> 2, tap = n / Co, co = n - tap * Co, a = tap >> 1, b = tap & 1;
                        v += P.bias[co];
                        const long long pix = ((long long)img * (2 * P.Ho) + 2 * ho + a) * (2 * P.Wo) + 2 * wo + b;
                        P.dst_bf16[pix * P.dst_stride + P.dst_off + co] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_BF16_LEAKYBWD) {
                        const float av = __bfloat162float(P.act[(long long)m * P.act_stride + P.act_off + n]);
                        P.dst_bf16[(long long)m * P.dst_stride + P.dst_off + n] =
                            __float2bfloat16_rn(v * (av > 0.f ? 1.0f : P.slope));
                    } else {  // EPI_F32 / EPI_F32_ADD
                        const long long o = (long long)m * P.dst_stride + P.dst_off + n;
                        if (EPI == EPI_F32_ADD) v += P.dst_f32[o];
                        P.dst_f32[o] = v;
                    }
                }
            }
        }
    }
}

// Split-k reduction of the fprop partials (fixed split order) with the
// epilogue of igemm_fprop_kernel.
// Sum over the splits z = 0 .. splits-1 of p[z * stride], in split order;
// loads are issued eight at a time so that their latencies overlap (the
// additions keep the order, so the result is that of the plain loop).
__device__ __forceinline__ float split_sum(const float *__restrict__ p, int splits, long long stride) {
    float s = 0.f;
    int z = 0;
    for (; z + 8 <= splits; z += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = p[(long long)(z + k) * stride];
#pragma unroll
        for (int k = 0; k < 8; k++) s += v[k];
    }
    for (; z < splits; z++) s += p[(long long)z * stride];
    return s;
}

// One thread per output (grid-stride), the splits summed in order.
template <int EPI>
__global__ void fprop_reduce_kernel(FpropArgs P, int splits) {
    const long long MN = (long long)P.M * P.N;
    const int HWo = P.Ho * P.Wo;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < MN;
         idx += (long long)gridDim.x * blockDim.x) {
        float v = split_sum(P.part + idx, splits, MN);
        const int m = (int)(idx / P.N), n = (int)(idx - (long long)m * P.N);
        if (EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) {
            v += P.bias[n];
            if (EPI == EPI_BF16_LEAKY) v = v > 0.f ? v : P.slope * v;
            P.dst_bf16[(long long)m * P.dst_stride + P.dst_off + n] = __float2bfloat16_rn(v);
        } else if (EPI == EPI_BF16_CONVT) {
            const int img = m / HWo;
            const int r = m - img * HWo;
            const int ho = r / P.Wo, wo = r - ho * P.Wo;
            const int Co = P.N >> 2, tap = n / Co, co = n - tap * Co, a = tap >> 1, b = tap & 1;  // tap-major columns
            v += P.bias[co];
            const long long pix = ((long long)img * (2 * P.Ho) + 2 * ho + a) * (2 * P.Wo) + 2 * wo + b;
            P.dst_bf16[pix * P.dst_stride + P.dst_off + co] = __float2bfloat16_rn(v);
        } else if (EPI == EPI_BF16_LEAKYBWD) {
            const float av = __bfloat162float(P.act[(long long)m * P.act_stride + P.act_off + n]);
            P.dst_bf16[(long long)m * P.dst_stride + P.dst_off + n] = __float2bfloat16_rn(v * (av > 0.f ? 1.0f : P.slope));
        } else {
            const long long o = (long long)m * P.dst_stride + P.dst_off + n;
            if (EPI == EPI_F32_ADD) v += P.dst_f32[o];
            P.dst_f32[o] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Implicit GEMM "wgrad" form (split over k): C[m][n] = sum_k A[m][k] B[k][n]
//   k: pixel (img, h, w) of an H x W grid (range [k_begin, k_end) per CTA);
//   A[m][k] = G[pixel'(k, m)][m-channel], B[k][n] = X[pixel''(k, n)][n-channel].
// Conv 3x3 weight gradient: m = co (G = output gradient at pixel k),
//   n = tap*Ci + ci (X = input at pixel k shifted by tap).
// Transposed conv weight gradient: m = (a*2+b)*Co + co (G at the fine pixel
//   (2h+a, 2w+b)), n = ci (X at the coarse pixel k).
// Tiles are stored k-major in shared memory and read with ldmatrix.trans.
// Each CTA writes its partial C tile to part[blockIdx.z][M][N].
// ---------------------------------------------------------------------------
constexpr int WBK = 32;

// Tile shape: WMW x WNW warps of 32 x 32 (BM = 32 WMW, BN = 32 WNW, 4 warps):
// 64 x 64 in general, 32 x 128 when M <= 32 (no half-empty m tiles).
template <int WMW, int WNW>
struct WgradTile {
    static constexpr int BM = 32 * WMW, BN = 32 * WNW, SM = BM + 8, SN = BN + 8;
    static constexpr int ACH = BM / 8, BCH = BN / 8;  // 16-byte chunks per k-row
    static constexpr int AI = WBK * ACH / 128, BI = WBK * BCH / 128;  // chunks per thread
    __nv_bfloat16 a[STAGES][WBK][SM];
    __nv_bfloat16 b[STAGES][WBK][SN];
};

template <int WMW, int WNW>
__global__ void __launch_bounds__(128) igemm_wgrad_kernel(WgradArgs P) {
    using TL = WgradTile<WMW, WNW>;
    constexpr int BM = TL::BM, BN = TL::BN;
    extern __shared__ __align__(16) unsigned char smraw[];
    TL &S = *reinterpret_cast<TL *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    // Pixel indices fit in 32 bits (the host checks nimg * H * W < 2^31).
    const int HW = P.H * P.W;
    const int KP = P.nimg * HW;
    const int per = (KP + gridDim.z - 1) / gridDim.z;
    const int kb = blockIdx.z * per;
    const int ke = kb + per < KP ? kb + per : KP;
    const int nk = ke > kb ? (ke - kb + WBK - 1) / WBK : 0;

    // B chunks: fixed column chunk per slot, so the tap split of n is done
    // once; the pixel (img, h, w) of each slot's k-row advances by WBK per
    // stage.
    int b_row[TL::BI], b_off[TL::BI], b_dh[TL::BI], b_dw[TL::BI], b_img[TL::BI], b_h[TL::BI], b_w[TL::BI];
    unsigned b_kind = 0;  // bit i: slot i is the ones column; bit 16+i: slot i is empty
#pragma unroll
    for (int i = 0; i < TL::BI; i++) {
        const int idx = tid + i * 128;
        b_row[i] = idx / TL::BCH;
        const int n = n0 + (idx % TL::BCH) * 8;
        b_off[i] = n;
        b_dh[i] = b_dw[i] = 0;
        if (n >= P.N || n > P.nw) b_kind |= 1u << (16 + i);
        else if (n == P.nw) b_kind |= 1u << i;
        else if (P.mode == WG_CONV) {
            const int tap = n / P.ci;
            b_off[i] = n - tap * P.ci;
            b_dh[i] = tap / 3 - 1;
            b_dw[i] = tap % 3 - 1;
        }
        const int k = kb + b_row[i];
        b_img[i] = k / HW;
        const int r = k - b_img[i] * HW;
        b_h[i] = r / P.W;
        b_w[i] = r - b_h[i] * P.W;
    }
    auto load_stage = [&](int st, int kt) {
#pragma unroll
        for (int i = 0; i < TL::AI; i++) {
            const int idx = tid + i * 128;
            const int kr = idx / TL::ACH, ch = idx % TL::ACH;
            const int k = kb + kt * WBK + kr;
            const int m = m0 + ch * 8;
            const bool ok = k < ke && m < P.M;
            const __nv_bfloat16 *src = P.g;
            if (ok) {
                if (P.mode == WG_CONV || P.g_s2d) {  // (space-to-depth: column m of coarse pixel k)
                    src = P.g + (long long)k * P.g_stride + m;
                } else {  // WG_CONVT: m = ab*Co + co at the fine pixel (2h + a, 2w + b)
                    const int img = k / HW;
                    const int r = k - img * HW;
                    const int h = r / P.W, w = r - h * P.W;
                    const int ab = m / P.co, co = m - ab * P.co;
                    const long long pix =
                        ((long long)img * (2 * P.H) + 2 * h + (ab >> 1)) * (2 * P.W) + 2 * w + (ab & 1);
                    src = P.g + pix * P.g_stride + co;
                }
            }
            cp16(&S.a[st][kr][ch * 8], src, ok);
        }
#pragma unroll
        for (int i = 0; i < TL::BI; i++) {
            const int idx = tid + i * 128;
            const int ch = idx % TL::BCH;
            const int k = kb + kt * WBK + b_row[i];
            bool ok = k < ke && !((b_kind >> (16 + i)) & 1u);
            const __nv_bfloat16 *src = P.x;
            if (ok && ((b_kind >> i) & 1u)) {
                src = P.ones;
            } else if (ok) {
                if (P.mode == WG_CONV) {
                    const int hs = b_h[i] + b_dh[i], ws = b_w[i] + b_dw[i];
                    ok = hs >= 0 && hs < P.H && ws >= 0 && ws < P.W;
                    if (ok) src = P.x + (((long long)b_img[i] * P.H + hs) * P.W + ws) * P.x_stride + P.x_off + b_off[i];
                } else {
                    src = P.x + (long long)k * P.x_stride + P.x_off + b_off[i];
                }
            }
            cp16(&S.b[st][b_row[i]][ch * 8], src, ok);
            // Next stage of this slot: pixel k + WBK.
            b_w[i] += WBK;
            while (b_w[i] >= P.W) {
                b_w[i] -= P.W;
                if (++b_h[i] == P.H) {
                    b_h[i] = 0;
                    b_img[i]++;
                }
            }
        }
    };

    // Warps: WMW x WNW over the tile, each 32 x 32.
    const int wm = (warp % WMW) * 32, wn = (warp / WMW) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;

    // Stages are loaded in order kt = 0, 1, 2, ...: the per-slot pixel
    // counters above advance once per load.
#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if (s < nk) load_stage(s, s);
        cp_commit();
    }
    for (int kt = 0; kt < nk; kt++) {
        cp_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nxt = kt + STAGES - 1;
            if (nxt < nk) load_stage(nxt % STAGES, nxt);
            cp_commit();
        }
        const int st = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < WBK; kk += 16) {
            unsigned af[2][4];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                // matrices (m0-7,k0-7) (m8-15,k0-7) (m0-7,k8-15) (m8-15,k8-15), stored k-major
                const int mat = lane >> 3;
                const int krow = kk + (lane & 7) + ((mat >> 1) << 3);
                const int mcol = wm + i * 16 + ((mat & 1) << 3);
                ldsm_x4_t(af[i], &S.a[st][krow][mcol]);
            }
#pragma unroll
            for (int j = 0; j < 4; j += 2) {
                unsigned bf[4];
                // matrices (k0-7,n0-7) (k8-15,n0-7) (k0-7,n8-15) (k8-15,n8-15), stored k-major
                const int mat = lane >> 3;
                const int krow = kk + (lane & 7) + ((mat & 1) << 3);
                const int ncol = wn + j * 8 + ((mat >> 1) << 3);
                ldsm_x4_t(bf, &S.b[st][krow][ncol]);
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    mma16816(acc[i][j], af[i], bf[0], bf[1]);
                    mma16816(acc[i][j + 1], af[i], bf[2], bf[3]);
                }
            }
        }
    }
    cp_wait<0>();
    float *out = P.part + (long long)blockIdx.z * P.M * P.N;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int m = m0 + wm + i * 16 + g + half * 8;
            if (m >= P.M) continue;
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int n = n0 + wn + j * 8 + 2 * t + e;
                    if (n < P.N) out[(long long)m * P.N + n] = acc[i][j][half * 2 + e];
                }
        }
}

// Sum of the weight-gradient split partials in split order (one thread per
// output); writes the weight gradient in the parameter layout (conv:
// [co][tap][ci] = C[co][n]; transposed conv: [co][a][b][ci] =
// C[(a*2+b)*Co + co][ci]) and the bias gradient from the bias column
// (transposed conv: summed over the four (a, b) rows).
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int splits, int M, int N, int nw, int mode,
                                    int co_n, float *__restrict__ dw, float *__restrict__ db) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)M * N) return;
    const int m = (int)(idx / N), n = (int)(idx - (long long)m * N);
    if (n > nw) return;
    if (n == nw) {
        if (mode == WG_CONV) {
            db[m] = split_sum(part + idx, splits, (long long)M * N);
        } else if (m < co_n) {  // one thread per co sums the rows (ab*co_n + m)
            float s = 0.f;
            for (int ab = 0; ab < 4; ab++)
                for (int z = 0; z < splits; z++) s += part[(long long)z * M * N + (long long)(ab * co_n + m) * N + n];
            db[m] = s;
        }
        return;
    }
    const float s = split_sum(part + idx, splits, (long long)M * N);
    long long o;
    if (mode == WG_CONV) {
        o = (long long)m * nw + n;
    } else {
        const int ab = m / co_n, co = m - ab * co_n;
        o = ((long long)co * 4 + ab) * nw + n;
    }
    dw[o] = s;
}

// One warp per channel: lane l sums the partials l, l+32, ..., then a
// shuffle tree (fixed order, so deterministic).
__global__ void bias_grad_final_kernel(const float *__restrict__ part, int nblk, int C, float *__restrict__ db) {
    const int c = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (c >= C) return;
    float s = 0.f;
    for (int b = lane; b < nblk; b += 32) s += part[(long long)b * C + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) db[c] = s;
}

// ---------------------------------------------------------------------------
// Elementwise and small kernels
// ---------------------------------------------------------------------------
// Average pool 3x3, stride 2, zero padding 1 counted (divide by 9); output bf16.
__global__ void avgpool_fwd_kernel(const __nv_bfloat16 *__restrict__ x, int xs, int xo, int nimg, int H, int W, int C,
                                   __nv_bfloat16 *__restrict__ y) {
    const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
    const long long n = (long long)nimg * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long r = i / C;
        const int wo = (int)(r % Wo);
        r /= Wo;
        const int ho = (int)(r % Ho);
        const int img = (int)(r / Ho);
        float s = 0.f;
        for (int a = 0; a < 3; a++) {
            const int h = 2 * ho + a - 1;
            if (h < 0 || h >= H) continue;
            for (int b = 0; b < 3; b++) {
                const int w = 2 * wo + b - 1;
                if (w < 0 || w >= W) continue;
                s += __bfloat162float(x[(((long long)img * H + h) * W + w) * xs + xo + c]);
            }
        }
        y[i] = __float2bfloat16_rn(s * (1.0f / 9.0f));
    }
}

// dx[h][w] (+)= sum of dy/9 over the pooling windows containing (h, w).
// Four channels per thread (C a multiple of 4, 16-byte aligned rows): the
// same sums in the same order as avgpool_bwd_kernel.
__global__ void avgpool_bwd4_kernel(const float *__restrict__ dy, int nimg, int H, int W, int C4,
                                    float *__restrict__ dx, int accumulate) {
    const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
    const long long n = (long long)nimg * H * W * C4;
    const float4 *dy4 = reinterpret_cast<const float4 *>(dy);
    float4 *dx4 = reinterpret_cast<float4 *>(dx);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C4);
        const long long r0 = i / C4;
        const int w = (int)(r0 % W);
        const long long r1 = r0 / W;
        const int h = (int)(r1 % H);
        const long long img = r1 / H;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int ho = (h > 0 ? h / 2 : 0); ho <= (h + 1) / 2 && ho < Ho; ho++) {
            if (2 * ho - 1 > h || 2 * ho + 1 < h) continue;
            for (int wo = (w > 0 ? w / 2 : 0); wo <= (w + 1) / 2 && wo < Wo; wo++) {
                if (2 * wo - 1 > w || 2 * wo + 1 < w) continue;
                const float4 v = dy4[((img * Ho + ho) * Wo + wo) * C4 + c];
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
        }
        const float k = 1.0f / 9.0f;
        s.x *= k;
        s.y *= k;
        s.z *= k;
        s.w *= k;
        if (accumulate) {
            const float4 o = dx4[i];
            s.x = o.x + s.x;
            s.y = o.y + s.y;
            s.z = o.z + s.z;
            s.w = o.w + s.w;
        }
        dx4[i] = s;
    }
}

__global__ void avgpool_bwd_kernel(const float *__restrict__ dy, int nimg, int H, int W, int C, float *__restrict__ dx,
                                   int accumulate) {
    const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
    const long long n = (long long)nimg * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long r = i / C;
        const int w = (int)(r % W);
        r /= W;
        const int h = (int)(r % H);
        const int img = (int)(r / H);
        float s = 0.f;
        // Windows (ho, wo) with 2ho-1 <= h <= 2ho+1.
        for (int ho = (h > 0 ? (h) / 2 : 0); ho <= (h + 1) / 2 && ho < Ho; ho++) {
            if (2 * ho - 1 > h || 2 * ho + 1 < h) continue;
            for (int wo = (w > 0 ? (w) / 2 : 0); wo <= (w + 1) / 2 && wo < Wo; wo++) {
                if (2 * wo - 1 > w || 2 * wo + 1 < w) continue;
                s += dy[(((long long)img * Ho + ho) * Wo + wo) * C + c];
            }
        }
        s *= (1.0f / 9.0f);
        dx[i] = accumulate ? dx[i] + s : s;
    }
}

// g = bf16(dA * (a > 0 ? 1 : slope)) for a LeakyReLU output a (bf16, with
// channel stride/offset), dA float32 dense [P][C].
__global__ void leaky_bwd_kernel(const float *__restrict__ dA, const __nv_bfloat16 *__restrict__ a, int as, int ao,
                                 long long P, int C, float slope, __nv_bfloat16 *__restrict__ g) {
    const long long n = P * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        const float av = __bfloat162float(a[p * as + ao + c]);
        g[i] = __float2bfloat16_rn(dA[i] * (av > 0.f ? 1.0f : slope));
    }
}

// Four channels per thread (C, strides and offsets multiples of 4, aligned
// pointers): the same per-element arithmetic as the kernels above and below.
struct alignas(8) Bf16x4 {
    __nv_bfloat162 lo, hi;
};
__device__ __forceinline__ float4 bf4_to_f4(Bf16x4 v) {
    const float2 a = __bfloat1622float2(v.lo), b = __bfloat1622float2(v.hi);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ Bf16x4 f4_to_bf4(float4 v) {
    Bf16x4 r;
    r.lo = __halves2bfloat162(__float2bfloat16_rn(v.x), __float2bfloat16_rn(v.y));
    r.hi = __halves2bfloat162(__float2bfloat16_rn(v.z), __float2bfloat16_rn(v.w));
    return r;
}

__global__ void leaky_bwd4_kernel(const float4 *__restrict__ dA, const __nv_bfloat16 *__restrict__ a, int as, int ao,
                                  long long P, int C4, float slope, Bf16x4 *__restrict__ g) {
    const long long n = P * C4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C4;
        const int c = (int)(i - p * C4) * 4;
        const float4 av = bf4_to_f4(*reinterpret_cast<const Bf16x4 *>(a + p * as + ao + c));
        const float4 d = dA[i];
        g[i] = f4_to_bf4(make_float4(d.x * (av.x > 0.f ? 1.0f : slope), d.y * (av.y > 0.f ? 1.0f : slope),
                                     d.z * (av.z > 0.f ? 1.0f : slope), d.w * (av.w > 0.f ? 1.0f : slope)));
    }
}

__global__ void f32_to_bf16_slice4_kernel(const float *__restrict__ x, int xs, int xo, long long P, int C4,
                                          Bf16x4 *__restrict__ y) {
    const long long n = P * C4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C4;
        const int c = (int)(i - p * C4) * 4;
        y[i] = f4_to_bf4(*reinterpret_cast<const float4 *>(x + p * xs + xo + c));
    }
}

__global__ void add_slice4_kernel(const float *__restrict__ src, int ss, int so, long long P, int C4,
                                  float4 *__restrict__ dst) {
    const long long n = P * C4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C4;
        const int c = (int)(i - p * C4) * 4;
        const float4 v = *reinterpret_cast<const float4 *>(src + p * ss + so + c);
        float4 d = dst[i];
        d.x += v.x;
        d.y += v.y;
        d.z += v.z;
        d.w += v.w;
        dst[i] = d;
    }
}

// d(cat) [P][2C] of a decoder level (H x W grid) split into its halves: the
// skip half copied (f32, [P][C]) for the encoder's backward, the upsampled
// half rounded to bf16 in space-to-depth layout [img][H/2][W/2][2a+b][C]
// (fine pixel (2h+a, 2w+b)) as the transposed conv's output gradient.
__global__ void split_cat4_kernel(const float *__restrict__ src, int nimg, int H, int W, int C4,
                                  float4 *__restrict__ skip, Bf16x4 *__restrict__ up) {
    const int rows = nimg * H;
    for (int rw = blockIdx.y; rw < rows; rw += gridDim.y) {
        const int img = rw / H, h = rw - img * H;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < W * C4; t += gridDim.x * blockDim.x) {
            const int w = t / C4, c = t - w * C4;
            const long long p = (long long)rw * W + w, i = p * C4 + c;
            const float *row = src + p * 8 * C4;
            skip[i] = *reinterpret_cast<const float4 *>(row + 4 * c);
            const long long q = (((long long)img * (H / 2) + h / 2) * (W / 2) + w / 2) * 4 + (h & 1) * 2 + (w & 1);
            up[q * C4 + c] = f4_to_bf4(*reinterpret_cast<const float4 *>(row + 4 * C4 + 4 * c));
        }
    }
}

// f32 [img][2H][2W][C] -> bf16 space-to-depth [img][H][W][2a+b][C].
__global__ void to_bf16_s2d_kernel(const float *__restrict__ x, int nimg, int H, int W, int C,
                                   __nv_bfloat16 *__restrict__ y) {
    const long long n = (long long)nimg * 4 * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;  // fine pixel
        const int w = (int)(p % (2 * W));
        const long long r = p / (2 * W);
        const int h = (int)(r % (2 * H));
        const long long img = r / (2 * H);
        const long long q = ((img * H + h / 2) * W + w / 2) * 4 + (h & 1) * 2 + (w & 1);
        y[q * C + c] = __float2bfloat16_rn(x[i]);
    }
}

// Backward of the 3x3 / stride-2 average pool (as avgpool_bwd4_kernel),
// plus the skip gradient of the same activation, times the LeakyReLU
// derivative of that activation (bf16 act, stride as, offset ao): the next
// block's output gradient g in bf16, as avgpool_bwd, add_slice and
// leaky_bwd in turn would give it.
__global__ void avgpool_bwd_leaky4_kernel(const float *__restrict__ dy, int nimg, int H, int W, int C4,
                                          const float4 *__restrict__ skip, const __nv_bfloat16 *__restrict__ act,
                                          int as, int ao, float slope, Bf16x4 *__restrict__ g) {
    const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1, rows = nimg * H;
    const float4 *dy4 = reinterpret_cast<const float4 *>(dy);
    for (int rw = blockIdx.y; rw < rows; rw += gridDim.y)
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < W * C4; t += gridDim.x * blockDim.x) {
        const long long img = rw / H;
        const int h = rw - (int)img * H, w = t / C4, c = t - w * C4;
        const long long r0 = (long long)rw * W + w, i = r0 * C4 + c;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int ho = (h > 0 ? h / 2 : 0); ho <= (h + 1) / 2 && ho < Ho; ho++) {
            if (2 * ho - 1 > h || 2 * ho + 1 < h) continue;
            for (int wo = (w > 0 ? w / 2 : 0); wo <= (w + 1) / 2 && wo < Wo; wo++) {
                if (2 * wo - 1 > w || 2 * wo + 1 < w) continue;
                const float4 v = dy4[((img * Ho + ho) * Wo + wo) * C4 + c];
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
        }
        const float k = 1.0f / 9.0f;
        const float4 o = skip[i];
        // Rounded product then sum (no contraction), as the separate passes.
        const float4 d = make_float4(__fadd_rn(__fmul_rn(s.x, k), o.x), __fadd_rn(__fmul_rn(s.y, k), o.y),
                                     __fadd_rn(__fmul_rn(s.z, k), o.z), __fadd_rn(__fmul_rn(s.w, k), o.w));
        const float4 av = bf4_to_f4(*reinterpret_cast<const Bf16x4 *>(act + r0 * as + ao + 4 * c));
        g[i] = f4_to_bf4(make_float4(d.x * (av.x > 0.f ? 1.0f : slope), d.y * (av.y > 0.f ? 1.0f : slope),
                                     d.z * (av.z > 0.f ? 1.0f : slope), d.w * (av.w > 0.f ? 1.0f : slope)));
    }
}

__global__ void avgpool_fwd4_kernel(const __nv_bfloat16 *__restrict__ x, int xs, int xo, int nimg, int H, int W,
                                    int C4, Bf16x4 *__restrict__ y) {
    // Rows (img, ho) on blockIdx.y, (wo, channel quad) on x: no 64-bit index division.
    const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1, rows = nimg * Ho;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int img = row / Ho, ho = row - img * Ho;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Wo * C4; t += gridDim.x * blockDim.x) {
            const int wo = t / C4, c = (t - wo * C4) * 4;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int a = 0; a < 3; a++) {
                const int h = 2 * ho + a - 1;
                if (h < 0 || h >= H) continue;
                for (int b = 0; b < 3; b++) {
                    const int w = 2 * wo + b - 1;
                    if (w < 0 || w >= W) continue;
                    const float4 v = bf4_to_f4(
                        *reinterpret_cast<const Bf16x4 *>(x + (((long long)img * H + h) * W + w) * xs + xo + c));
                    s.x += v.x;
                    s.y += v.y;
                    s.z += v.z;
                    s.w += v.w;
                }
            }
            const float k = 1.0f / 9.0f;
            y[(long long)row * Wo * C4 + t] = f4_to_bf4(make_float4(s.x * k, s.y * k, s.z * k, s.w * k));
        }
    }
}

// Copy channels [off, off+C) of a float32 [P][Ct] tensor into bf16 [P][C].
__global__ void f32_to_bf16_slice_kernel(const float *__restrict__ x, int xs, int xo, long long P, int C,
                                         __nv_bfloat16 *__restrict__ y) {
    const long long n = P * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        y[i] = __float2bfloat16_rn(x[p * xs + xo + c]);
    }
}

// dst[P][C] += src[P][Cs] channels [off, off+C)  (float32)
__global__ void add_slice_kernel(const float *__restrict__ src, int ss, int so, long long P, int C,
                                 float *__restrict__ dst) {
    const long long n = P * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C;
        const int c = (int)(i - p * C);
        dst[i] += src[p * ss + so + c];
    }
}

// Output layer 1x1 conv (Cin -> 1), fp32 out: out[p] = b + sum_c bf16(W[c]) a[p][c].
__global__ void conv1x1_fwd_kernel(const __nv_bfloat16 *__restrict__ a, int C, long long P,
                                   const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b,
                                   float *__restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        if ((C & 7) == 0) {  // 16-byte loads of 8 channels (rows are 16-byte aligned when C is a multiple of 8)
            const uint4 *row = reinterpret_cast<const uint4 *>(a + p * C);
            for (int c8 = 0; c8 < C / 8; c8++) {
                const uint4 q = row[c8];
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
                for (int e = 0; e < 8; e++) s = fmaf(__bfloat162float(w[8 * c8 + e]), __bfloat162float(h[e]), s);
            }
        } else {
            for (int c = 0; c < C; c++) s = fmaf(__bfloat162float(w[c]), __bfloat162float(a[p * C + c]), s);
        }
        out[p] = s + b[0];
    }
}

// MSE over P outputs: loss partials (double) and g = bf16(2 (out - y) / P).
__global__ void mse_kernel(const float *__restrict__ out, const float *__restrict__ y, long long P,
                           __nv_bfloat16 *__restrict__ g, double *__restrict__ partial) {
    double acc = 0.0;
    const float sc = 2.0f / (float)P;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        const float r = out[i] - y[i];
        acc += (double)r * r;
        g[i] = __float2bfloat16_rn(sc * r);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

// Output layer (1x1 conv, C -> 1) backward fused with the activation
// backward of its input: per pixel p, g = g_out[p] (bf16); the next block's
// output gradient gn[p][c] = bf16(bf16(W[c]) g * leaky'(a[p][c])), and
// per-block partial sums part[blk][c] = sum g a[p][c], part[blk][C] = sum g.
// Threads (c, j): channel c (blockDim.x = C + 1 rounded up to 32) over the
// pixels p0 + j, p0 + j + S, ... (S = blockDim.y streams), the streams then
// summed in order j = 0, 1, ... (deterministic).
__global__ void __launch_bounds__(512) conv1x1_bwd_leaky_kernel(const __nv_bfloat16 *__restrict__ g, const __nv_bfloat16 *__restrict__ a,
                                         long long P, int C, const __nv_bfloat16 *__restrict__ w, float slope,
                                         __nv_bfloat16 *__restrict__ gn, int rows, float *__restrict__ part) {
    extern __shared__ float red[];  // [S][blockDim.x]
    const int c = threadIdx.x, j = threadIdx.y, S = blockDim.y;
    const long long p0 = (long long)blockIdx.x * rows;
    const long long p1 = p0 + rows < P ? p0 + rows : P;
    const float wc = c < C ? __bfloat162float(w[c]) : 0.f;
    float s = 0.f;
    if (c <= C) {
        long long p = p0 + j;
        for (; p + 7 * S < p1; p += 8 * S) {  // eight pixels' loads issued before their sums
            float gv[8], av[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                gv[k] = __bfloat162float(g[p + k * S]);
                av[k] = c < C ? __bfloat162float(a[(p + k * S) * C + c]) : 1.f;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                s += gv[k] * av[k];
                if (c < C) gn[(p + k * S) * C + c] = __float2bfloat16_rn(wc * gv[k] * (av[k] > 0.f ? 1.0f : slope));
            }
        }
        for (; p < p1; p += S) {
            const float gv = __bfloat162float(g[p]);
            const float av = c < C ? __bfloat162float(a[p * C + c]) : 1.f;
            s += gv * av;
            if (c < C) gn[p * C + c] = __float2bfloat16_rn(wc * gv * (av > 0.f ? 1.0f : slope));
        }
    }
    red[j * blockDim.x + c] = s;
    __syncthreads();
    if (j == 0 && c <= C) {
        float t = red[c];
        for (int q = 1; q < S; q++) t += red[q * blockDim.x + c];
        part[(long long)blockIdx.x * (C + 1) + c] = t;
    }
}

// Adam with bias correction (Adam's step t is 1-based), master weights fp32,
// and the bf16 shadow copy refreshed.
__global__ void adam_kernel(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2, __nv_bfloat16 *__restrict__ shadow) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        const float th = theta[i] - lr * mh / (sqrtf(vh) + eps);
        theta[i] = th;
        shadow[i] = __float2bfloat16_rn(th);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, long long n, __nv_bfloat16 *__restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void bf16_to_f32_kernel(const __nv_bfloat16 *__restrict__ x, long long n, float *__restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __bfloat162float(x[i]);
}

// Transposed weights for the input-gradient GEMM:
// wt[ci][tap][co] = w[co][tap][ci] (bf16), taps = 9 (conv) or 4 (transposed conv).
__global__ void transpose_w_kernel(const __nv_bfloat16 *__restrict__ w, int co, int taps, int ci,
                                   __nv_bfloat16 *__restrict__ wt) {
    const long long n = (long long)co * taps * ci;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ci);
        long long r = i / ci;
        const int t = (int)(r % taps);
        const int o = (int)(r / taps);
        wt[((long long)c * taps + t) * co + o] = w[i];
    }
}

// The transposes of several layers in one launch: job j = blockIdx.y, and
// blockIdx.x one 32 x 32 tile (output channels o x input channels c) of one
// tap t, staged in shared memory so that both the reads along c and the
// writes along o are contiguous.
__global__ void transpose_w_batch_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt,
                                         TransposeJobs J) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int j = blockIdx.y;
    const long long off = J.off[j];
    const int co = J.co[j], taps = J.taps[j], ci = J.ci[j];
    const int to = (co + 31) / 32, tc = (ci + 31) / 32;
    int b = blockIdx.x;
    if (b >= to * tc * taps) return;
    const int t = b % taps;
    b /= taps;
    const int c0 = (b % tc) * 32, o0 = (b / tc) * 32;
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;  // 32 x 8 threads
    for (int r = y; r < 32; r += 8) {  // read rows o0 + r along c
        const int o = o0 + r, c = c0 + x;
        if (o < co && c < ci) tile[r][x] = w[off + ((long long)o * taps + t) * ci + c];
    }
    __syncthreads();
    for (int r = y; r < 32; r += 8) {  // write rows c0 + r along o
        const int c = c0 + r, o = o0 + x;
        if (o < co && c < ci) wt[off + ((long long)c * taps + t) * co + o] = tile[x][r];
    }
}

// The transposed convolutions' forward GEMM takes its weight rows
// tap-major: [co][4][ci] -> [4][co][ci] (job j = blockIdx.y), so that an
// output tile's 16 consecutive columns are 16 channels of one output
// sub-pixel (contiguous stores).
__global__ void convt_tapmajor_batch_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wp,
                                            TransposeJobs J) {
    const int j = blockIdx.y;
    const long long off = J.off[j];
    const int co = J.co[j], ci = J.ci[j];
    const long long n = 4LL * co * ci;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ci);
        const long long r = i / ci;
        const int t = (int)(r & 3), o = (int)(r >> 2);
        wp[off + ((long long)t * co + o) * ci + c] = w[off + i];
    }
}

// Input image (float32 [img][H][W]) into a bf16 NHWC tensor of Cp channels
// (channel 0 = the image, others 0).
__global__ void input_pack_kernel(const float *__restrict__ x, long long P, int Cp, __nv_bfloat16 *__restrict__ y) {
    const long long n = P * Cp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % Cp);
        y[i] = __float2bfloat16_rn(c == 0 ? x[i / Cp] : 0.f);
    }
}

// Patches: dst[b][i][j] = img[oz + i][ox + j] * scale for patch b = sel[b]
// (0 in the first `mute` image rows).
__global__ void gather_patches_kernel(const float *__restrict__ img, int nx, const int *__restrict__ oz,
                                      const int *__restrict__ ox, const int *__restrict__ sel, int nb, int p,
                                      const float *__restrict__ scale, int mute, float *__restrict__ dst) {
    const long long n = (long long)nb * p * p;
    const float sc = *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i % p);
        long long r = i / p;
        const int ii = (int)(r % p);
        const int b = (int)(r / p);
        const int pi = sel[b];
        const int row = oz[pi] + ii;
        dst[i] = row < mute ? 0.f : img[(long long)row * nx + ox[pi] + j] * sc;
    }
}

// Full-image input: zero padded to Hp x Wp, scaled, first `mute` rows 0.
__global__ void pad_image_kernel(const float *__restrict__ img, int nz, int nx, int Hp, int Wp,
                                 const float *__restrict__ scale, int mute, float *__restrict__ dst) {
    const long long n = (long long)Hp * Wp;
    const float sc = *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(i % Wp), h = (int)(i / Wp);
        dst[i] = (h >= mute && h < nz && w < nx) ? img[(long long)h * nx + w] * sc : 0.f;
    }
}

__global__ void crop_image_kernel(const float *__restrict__ src, int Hp, int Wp, int nz, int nx,
                                  const float *__restrict__ scale, float *__restrict__ dst) {
    const long long n = (long long)nz * nx;
    const float sc = *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(i % nx), h = (int)(i / nx);
        dst[i] = src[(long long)h * Wp + w] * sc;
    }
}

// max |x| over n values -> *out as float bits via atomicMax (values >= 0).
__global__ void absmax_kernel(const float *__restrict__ x, long long n, unsigned *out) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// scale_out[0] = 1 / max (or 1 if max == 0); scale_out[1] = max.
__global__ void absmax_finish_kernel(const unsigned *mx, float *scale_out) {
    const float m = __uint_as_float(*mx);
    scale_out[0] = m > 0.f ? 1.0f / m : 1.0f;
    scale_out[1] = m > 0.f ? m : 1.0f;
}

// First layer (one input channel) padded to cpad channels: wp[co][tap][c] =
// w[co][tap] for c == 0, else 0; and the gradient taken back from channel 0.
// Weight and bias gradients of the first 3x3 convolution, whose input has
// one real channel (channel 0 of xin, the others zero):
//   dW[co][t] = sum_p G[p][co] x[p + shift(t)],   db[co] = sum_p G[p][co],
// a reduction over the pixels on CUDA cores (the tensor-core GEMM would
// spend 72 of its 80 columns on the zero channels).  Lane = output channel
// (32 per pass); a warp takes row segments of 32 pixels (row = img * H + h)
// and walks each in chunks of 8 pixels whose output-gradient values and
// 3 x 10 input window are all loaded before the chunk's sums (one memory
// latency per chunk); per-block sums [b][co][10] in a fixed order, then
// first_wgrad_final_kernel sums the blocks.
__global__ void __launch_bounds__(256) first_wgrad_kernel(const __nv_bfloat16 *__restrict__ g, int co_n,
                                                          const __nv_bfloat16 *__restrict__ xin, int cpad, int nimg,
                                                          int H, int W, float *__restrict__ part) {
    __shared__ float red[8][32][10];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (W + 31) / 32, tasks = nimg * H * segs, nwarps = gridDim.x * 8;
    for (int cb = 0; cb < co_n; cb += 32) {
        const int co = cb + lane;
        const bool valid = co < co_n;
        float acc[10];
#pragma unroll
        for (int k = 0; k < 10; k++) acc[k] = 0.f;
        for (int task = blockIdx.x * 8 + warp; task < tasks; task += nwarps) {
            const int row = task / segs, ws = (task - row * segs) * 32;
            const int h = row % H, we = min(W, ws + 32);
            const long long rbase = (long long)(row - h) * W;  // first pixel of the row's image
            for (int w0 = ws; w0 < we; w0 += 8) {
                float gv[8], xc[3][10];
#pragma unroll
                for (int e = 0; e < 8; e++)
                    gv[e] = valid && w0 + e < we ? __bfloat162float(g[((long long)row * W + w0 + e) * co_n + co]) : 0.f;
                {  // lane l < 30 loads window element (l / 10, l % 10); shuffled to all lanes
                    const int la = lane / 10, le = lane - 10 * la;
                    const int hh = h + la - 1, ww = w0 - 1 + le;
                    const float mine = lane < 30 && hh >= 0 && hh < H && ww >= 0 && ww < W
                                           ? __bfloat162float(xin[(rbase + (long long)hh * W + ww) * cpad])
                                           : 0.f;
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int e = 0; e < 10; e++) xc[a][e] = __shfl_sync(0xffffffffu, mine, a * 10 + e);
                }
#pragma unroll
                for (int e = 0; e < 8; e++) {
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int b = 0; b < 3; b++) acc[a * 3 + b] += gv[e] * xc[a][e + b];
                    acc[9] += gv[e];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 10; k++) red[warp][lane][k] = acc[k];
        __syncthreads();
        if (warp == 0 && valid) {
#pragma unroll
            for (int k = 0; k < 10; k++) {
                float t = 0.f;
                for (int q = 0; q < 8; q++) t += red[q][lane][k];
                part[((long long)blockIdx.x * co_n + co) * 10 + k] = t;
            }
        }
        __syncthreads();
    }
}

// dw[co][9] and db[co] from the per-block sums: block i = output (co, k);
// thread t sums blocks t, t + 256, ... in order, then a fixed shared-memory
// tree.
__global__ void first_wgrad_final_kernel(const float *__restrict__ part, int nblk, int co_n, float *__restrict__ dw,
                                         float *__restrict__ db) {
    __shared__ float red[256];
    const int i = blockIdx.x, co = i / 10, k = i - co * 10;
    float s = 0.f;
    for (int b = threadIdx.x; b < nblk; b += 256) s += part[((long long)b * co_n + co) * 10 + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (k < 9) dw[co * 9 + k] = red[0];
        else db[co] = red[0];
    }
}

// The first 3x3 convolution (one real input channel: channel 0 of xin) with
// bias and LeakyReLU, on CUDA cores: y[p][co] = leaky(sum_t W[co][t]
// x[p + shift(t)] + b[co]) in bf16.  Thread: one pixel, 8 output channels
// (fp32 sums over the taps in order; 16-byte store); the weights (bf16
// [co][9]) and the bias are staged in shared memory as floats.
__global__ void __launch_bounds__(256) first_conv_kernel(const __nv_bfloat16 *__restrict__ xin, int cpad, int nimg,
                                                         int H, int W, const __nv_bfloat16 *__restrict__ w,
                                                         const float *__restrict__ bias, int co_n, float slope,
                                                         __nv_bfloat16 *__restrict__ y, int ys) {
    extern __shared__ float sw[];  // [co_n][9] weights, then [co_n] bias
    for (int i = threadIdx.x; i < co_n * 10; i += blockDim.x)
        sw[i] = i < co_n * 9 ? __bfloat162float(w[i]) : bias[i - co_n * 9];
    __syncthreads();
    // blockIdx.y: image row (img * H + h); x: (pixel of the row, channel group).
    const int groups = co_n / 8, row = blockIdx.y, h0 = row % H;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w0 = t / groups, c0 = 8 * (t - w0 * groups);
    if (w0 >= W) return;
    const long long p = (long long)row * W + w0;
    float xv[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int dh = k / 3 - 1, dw = k % 3 - 1;
        const bool in = h0 + dh >= 0 && h0 + dh < H && w0 + dw >= 0 && w0 + dw < W;
        xv[k] = in ? __bfloat162float(xin[(p + (long long)dh * W + dw) * cpad]) : 0.f;
    }
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const float *wr = sw + (c0 + e) * 9;
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < 9; k++) a = fmaf(wr[k], xv[k], a);
        a += sw[co_n * 9 + c0 + e];
        o[e] = __float2bfloat16_rn(a > 0.f ? a : slope * a);
    }
    *reinterpret_cast<uint4 *>(y + p * ys + c0) = *reinterpret_cast<const uint4 *>(o);
}

__global__ void pad_first_w_kernel(const __nv_bfloat16 *__restrict__ w, int co, int cpad,
                                   __nv_bfloat16 *__restrict__ wp) {
    const int n = co * 9 * cpad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i % cpad;
        wp[i] = c == 0 ? w[i / cpad] : __float2bfloat16_rn(0.f);
    }
}

__global__ void unpad_first_grad_kernel(const float *__restrict__ gp, int co, int cpad, float *__restrict__ g) {
    const int n = co * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) g[i] = gp[i * cpad];
}

// acc[0] += weight * sum(partial) (single thread, fixed order).
__global__ void loss_accum_kernel(const double *__restrict__ partial, int nblocks, double weight, double *acc) {
    double s = 0.0;
    for (int i = 0; i < nblocks; i++) s += partial[i];
    acc[0] += weight * s;
}

// ---------------------------------------------------------------------------
// 3x3 convolutions (forward and input gradient: nine taps, shifts in
// {-1, 0, 1}, stride 1) with a shared-memory halo tile: a CTA computes a
// block of 8 x 16 output pixels for BN output channels.  For each slice of
// 32 input channels the block's input patch (10 x 18 pixels) is staged once
// and the nine taps read their A fragments from it with ldmatrix at shifted
// row addresses, instead of gathering every tap from global memory.  The
// k-steps (channel slice, tap) run through a 3-stage pipeline of weight
// tiles; patches are double-buffered and loaded with the first tap of their
// slice.  Same GEMM (k = tap * C + c), accumulation and epilogues as
// igemm_fprop_kernel, no split-k.
// ---------------------------------------------------------------------------
constexpr int HBH = 8, HBW = 16;                          // output block
constexpr int HPH = HBH + 2, HPW = HBW + 2, HPOS = HPH * HPW;  // 10 x 18 patch
constexpr int HCB = 32, HSK = HCB + 8;                     // channels per slice, padded row

template <int BN>
struct HaloSmem {
    __nv_bfloat16 patch[2][HPOS][HSK];
    __nv_bfloat16 b[STAGES][BN][HSK];
};

template <int BN, int EPI>
__global__ void __launch_bounds__(128) conv3_halo_kernel(FpropArgs P, int bh_n, int bw_n) {
    extern __shared__ __align__(16) unsigned char smraw[];
    HaloSmem<BN> &S = *reinterpret_cast<HaloSmem<BN> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int blk = blockIdx.x;
    const int bw = blk % bw_n;
    blk /= bw_n;
    const int bh = blk % bh_n;
    const int img = blk / bh_n;
    const int h0 = bh * HBH, w0 = bw * HBW;
    const int n0 = blockIdx.y * BN;
    const int H = P.Hs, W = P.Ws;
    const int nslices = P.C / HCB;
    const int nk = nslices * 9;  // k-steps (slice, tap)
    const int K = 9 * P.C;

    auto load_step = [&](int st, int ks) {
        const int sl = ks / 9, tap = ks - sl * 9;
        if (tap == 0) {  // the slice's patch, into buffer sl & 1
            for (int idx = tid; idx < HPOS * (HCB / 8); idx += 128) {
                const int pos = idx >> 2, ch = idx & 3;
                const int hs = h0 - 1 + pos / HPW, ws = w0 - 1 + pos % HPW;
                const bool ok = hs >= 0 && hs < H && ws >= 0 && ws < W;
                const __nv_bfloat16 *src =
                    ok ? P.src + (((long long)img * H + hs) * W + ws) * P.src_stride + P.src_off + sl * HCB + ch * 8
                       : P.src;
                cp16(&S.patch[sl & 1][pos][ch * 8], src, ok);
            }
        }
        for (int idx = tid; idx < BN * (HCB / 8); idx += 128) {
            const int row = idx >> 2, ch = idx & 3;
            const int n = n0 + row;
            const bool ok = n < P.N;
            cp16(&S.b[st][row][ch * 8], ok ? P.bt + (long long)n * K + tap * P.C + sl * HCB + ch * 8 : P.bt, ok);
        }
    };

    float acc[2][BN / 8][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < BN / 8; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;

#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if (s < nk) load_step(s, s);
        cp_commit();
    }
    for (int ks = 0; ks < nk; ks++) {
        cp_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nxt = ks + STAGES - 1;
            if (nxt < nk) load_step(nxt % STAGES, nxt);
            cp_commit();
        }
        const int st = ks % STAGES;
        const int sl = ks / 9, tap = ks - sl * 9;
        const int dh = P.dh[tap], dw = P.dw[tap];
        const __nv_bfloat16(*patch)[HSK] = S.patch[sl & 1];
#pragma unroll
        for (int kk = 0; kk < HCB; kk += 16) {
            unsigned af[2][4];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int p = warp * 32 + i * 16 + (lane & 15);  // pixel of the block
                const int pos = (p / HBW + 1 + dh) * HPW + p % HBW + 1 + dw;
                ldsm_x4(af[i], &patch[pos][kk + (lane >> 4) * 8]);
            }
#pragma unroll
            for (int j = 0; j < BN / 8; j += 2) {
                unsigned bf[4];
                const int r = j * 8 + (lane & 7) + ((lane >> 4) << 3);
                ldsm_x4(bf, &S.b[st][r][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    mma16816(acc[i][j], af[i], bf[0], bf[1]);
                    mma16816(acc[i][j + 1], af[i], bf[2], bf[3]);
                }
            }
        }
    }
    cp_wait<0>();

    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; i++) {
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int p = warp * 32 + i * 16 + g + half * 8;
            const int h = h0 + p / HBW, w = w0 + p % HBW;
            if (h >= H || w >= W) continue;
            const long long m = ((long long)img * H + h) * W + w;
#pragma unroll
            for (int j = 0; j < BN / 8; j++) {
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int n = n0 + j * 8 + 2 * t + e;
                    if (n >= P.N) continue;
                    float v = acc[i][j][half * 2 + e];
                    if (EPI == EPI_BF16_LEAKY || EPI == EPI_BF16) {
                        v += P.bias[n];
                        if (EPI == EPI_BF16_LEAKY) v = v > 0.f ? v : P.slope * v;
                        P.dst_bf16[m * P.dst_stride + P.dst_off + n] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_BF16_LEAKYBWD) {
                        const float av = __bfloat162float(P.act[m * P.act_stride + P.act_off + n]);
                        P.dst_bf16[m * P.dst_stride + P.dst_off + n] = __float2bfloat16_rn(v * (av > 0.f ? 1.0f : P.slope));
                    } else {  // EPI_F32 / EPI_F32_ADD
                        const long long o = m * P.dst_stride + P.dst_off + n;
                        if (EPI == EPI_F32_ADD) v += P.dst_f32[o];
                        P.dst_f32[o] = v;
                    }
                }
            }
        }
    }
}

// ===========================================================================
// Host launchers
// ===========================================================================
// Grid of the row kernels: x over one row's elements (256 per block), y over
// the rows (at most 65535; the kernels stride over the rest).
static dim3 row_grid(int per_row, int rows) {
    return dim3((unsigned)std::max(1, (per_row + 255) / 256), (unsigned)std::max(1, std::min(rows, 65535)));
}
static int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

template <int BN, int EPI>
static void fprop_launch(const FpropArgs &a, cudaStream_t s) {
    const size_t sm = sizeof(FpropSmem<BN>);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(igemm_fprop_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    const int tiles = ((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
    const int nk = (a.ntaps * a.C + BK - 1) / BK;
    int splits = 1;
    if (a.part && a.part_floats > 0) {
        // Split k when the tiles fill less than ~2 waves (4 CTAs per SM), keeping
        // at least 8 k-tiles per split and the partials within their buffer.
        const int want = (2 * 152 * 4 + tiles - 1) / tiles;
        splits = std::min(want, nk / 8);
        const long long cap = a.part_floats / ((long long)a.M * a.N);
        if (splits > cap) splits = (int)cap;
        if (splits < 2) splits = 1;
    }
    FpropArgs b = a;
    if (splits == 1) b.part = nullptr;
    dim3 grid((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, splits);
    igemm_fprop_kernel<BN, EPI><<<grid, 128, sm, s>>>(b);
    if (splits > 1) {
        const long long mn = (long long)a.M * a.N;
        fprop_reduce_kernel<EPI><<<grid_for(mn), 256, 0, s>>>(b, splits);
    }
}

void launch_fprop_reduce(const FpropArgs &a, int epi, int splits, cudaStream_t s) {
    const int g = grid_for((long long)a.M * a.N);
    const int b = 256;
    switch (epi) {
    case EPI_BF16_LEAKY: fprop_reduce_kernel<EPI_BF16_LEAKY><<<g, b, 0, s>>>(a, splits); break;
    case EPI_BF16: fprop_reduce_kernel<EPI_BF16><<<g, b, 0, s>>>(a, splits); break;
    case EPI_BF16_CONVT: fprop_reduce_kernel<EPI_BF16_CONVT><<<g, b, 0, s>>>(a, splits); break;
    case EPI_F32: fprop_reduce_kernel<EPI_F32><<<g, b, 0, s>>>(a, splits); break;
    case EPI_BF16_LEAKYBWD: fprop_reduce_kernel<EPI_BF16_LEAKYBWD><<<g, b, 0, s>>>(a, splits); break;
    default: fprop_reduce_kernel<EPI_F32_ADD><<<g, b, 0, s>>>(a, splits); break;
    }
}

// Forward-form GEMM kernels.  By default the 3x3 convolutions with at least
// 64 output channels run on the TMA-fed tcgen05 kernel (nn_umma.cu) and the
// rest on mma.sync (halo tiles for the 3x3 convolutions).  DHFWI_NN_GEMM=mma
// keeps every GEMM on mma.sync; DHFWI_NN_GEMM=tc puts every one on the
// cp.async-fed tcgen05 kernel.  Read per launch so a process can switch.
enum { GEMM_DEFAULT = 0, GEMM_UMMA_ALL = 1, GEMM_MMA_ONLY = 2 };
static int gemm_mode() {
    const char *e = getenv("DHFWI_NN_GEMM");
    if (e && strcmp(e, "tc") == 0) return GEMM_UMMA_ALL;
    if (e && strcmp(e, "mma") == 0) return GEMM_MMA_ONLY;
    return GEMM_DEFAULT;
}

template <int BN, int EPI>
static void halo_launch(const FpropArgs &a, int bh_n, int bw_n, int nimg, cudaStream_t s) {
    const size_t sm = sizeof(HaloSmem<BN>);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(conv3_halo_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    dim3 grid(nimg * bh_n * bw_n, (a.N + BN - 1) / BN);
    conv3_halo_kernel<BN, EPI><<<grid, 128, sm, s>>>(a, bh_n, bw_n);
}

template <int EPI>
static void halo_dispatch(const FpropArgs &a, int bh_n, int bw_n, int nimg, cudaStream_t s) {
    if (a.N <= 32) halo_launch<32, EPI>(a, bh_n, bw_n, nimg, s);
    else halo_launch<64, EPI>(a, bh_n, bw_n, nimg, s);
}

// The halo-tile kernel serves every 3x3 convolution (nine taps with shifts
// in {-1, 0, 1}, stride 1, same grid in and out) with input channels in
// slices of 32: measured faster than the gathering kernel with split-k also
// on the small grids of the deep levels.  DHFWI_NN_HALO=0 turns it off.
static bool halo_eligible(const FpropArgs &a, int epi, int *bh_n, int *bw_n, int *nimg) {
    const char *e = getenv("DHFWI_NN_HALO");
    if (e && strcmp(e, "0") == 0) return false;
    if (a.ntaps != 9 || a.scale != 1 || a.Ho != a.Hs || a.Wo != a.Ws || a.C % HCB != 0) return false;
    if (epi == EPI_BF16_CONVT) return false;
    if ((a.src_stride | a.src_off) & 7) return false;
    for (int t = 0; t < 9; t++)
        if (a.dh[t] < -1 || a.dh[t] > 1 || a.dw[t] < -1 || a.dw[t] > 1) return false;
    const long long HW = (long long)a.Hs * a.Ws;
    if (HW <= 0 || a.M % HW != 0) return false;
    *nimg = (int)(a.M / HW);
    *bh_n = (a.Hs + HBH - 1) / HBH;
    *bw_n = (a.Ws + HBW - 1) / HBW;
    return true;
}

void launch_fprop(const FpropArgs &a, int epi, cudaStream_t s) {
    const int mode = gemm_mode();
    if (mode == GEMM_UMMA_ALL) {
        launch_fprop_umma(a, epi, s);
        return;
    }
    if (mode == GEMM_DEFAULT && (launch_conv3_patch(a, epi, s) || launch_conv3_tma(a, epi, s))) return;
    int bh_n, bw_n, nimg;
    if (halo_eligible(a, epi, &bh_n, &bw_n, &nimg)) {
        switch (epi) {
        case EPI_BF16_LEAKY: halo_dispatch<EPI_BF16_LEAKY>(a, bh_n, bw_n, nimg, s); break;
        case EPI_BF16: halo_dispatch<EPI_BF16>(a, bh_n, bw_n, nimg, s); break;
        case EPI_F32: halo_dispatch<EPI_F32>(a, bh_n, bw_n, nimg, s); break;
        case EPI_BF16_LEAKYBWD: halo_dispatch<EPI_BF16_LEAKYBWD>(a, bh_n, bw_n, nimg, s); break;
        default: halo_dispatch<EPI_F32_ADD>(a, bh_n, bw_n, nimg, s); break;
        }
        return;
    }
    const bool small = a.N <= 32;
    switch (epi) {
    case EPI_BF16_LEAKY: small ? fprop_launch<32, EPI_BF16_LEAKY>(a, s) : fprop_launch<64, EPI_BF16_LEAKY>(a, s); break;
    case EPI_BF16: small ? fprop_launch<32, EPI_BF16>(a, s) : fprop_launch<64, EPI_BF16>(a, s); break;
    case EPI_BF16_CONVT: small ? fprop_launch<32, EPI_BF16_CONVT>(a, s) : fprop_launch<64, EPI_BF16_CONVT>(a, s); break;
    case EPI_F32: small ? fprop_launch<32, EPI_F32>(a, s) : fprop_launch<64, EPI_F32>(a, s); break;
    case EPI_BF16_LEAKYBWD:
        small ? fprop_launch<32, EPI_BF16_LEAKYBWD>(a, s) : fprop_launch<64, EPI_BF16_LEAKYBWD>(a, s);
        break;
    default: small ? fprop_launch<32, EPI_F32_ADD>(a, s) : fprop_launch<64, EPI_F32_ADD>(a, s); break;
    }
}

// Tile shape of the weight-gradient GEMM for an M-row problem.
static bool wgrad_narrow(int M) { return M <= 32; }

int wgrad_splits(long long kpix, int M, int N) {
    const int BM = wgrad_narrow(M) ? 32 : 64, BN = wgrad_narrow(M) ? 128 : 64;
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    long long want = (152LL * 4 + tiles - 1) / tiles;
    long long maxs = (kpix + 255) / 256;  // at least 256 pixels per split
    if (want > maxs) want = maxs;
    if (want < 1) want = 1;
    if (want > 512) want = 512;
    return (int)want;
}

template <int WMW, int WNW>
static void wgrad_launch(const WgradArgs &a, int splits, cudaStream_t s) {
    using TL = WgradTile<WMW, WNW>;
    const size_t sm = sizeof(TL);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(igemm_wgrad_kernel<WMW, WNW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    dim3 grid((a.M + TL::BM - 1) / TL::BM, (a.N + TL::BN - 1) / TL::BN, splits);
    igemm_wgrad_kernel<WMW, WNW><<<grid, 128, sm, s>>>(a);
}

int launch_wgrad(const WgradArgs &a, int splits, float *dw, float *db, cudaStream_t s) {
    const long long mn = (long long)a.M * a.N;
    const int tsp = launch_wgrad_tma(a, splits, s);
    if (tsp > 0) {  // partials with the bias column: weight and bias gradients in one reduction
        wgrad_reduce_kernel<<<(int)((mn + 255) / 256), 256, 0, s>>>(a.part, tsp, a.M, a.N, a.nw, a.mode, a.co, dw,
                                                                     db);
        return 2;
    }
    if (wgrad_narrow(a.M)) wgrad_launch<1, 4>(a, splits, s);
    else wgrad_launch<2, 2>(a, splits, s);
    wgrad_reduce_kernel<<<(int)((mn + 255) / 256), 256, 0, s>>>(a.part, splits, a.M, a.N, a.nw, a.mode, a.co, dw,
                                                                 db);
    return 2;
}

void launch_avgpool_fwd(const __nv_bfloat16 *x, int xs, int xo, int nimg, int H, int W, int C, __nv_bfloat16 *y,
                        cudaStream_t s) {
    const long long n = (long long)nimg * ((H - 1) / 2 + 1) * ((W - 1) / 2 + 1) * C;
    if (C % 4 == 0 && ((xs | xo) & 3) == 0 && (((uintptr_t)x | (uintptr_t)y) & 7) == 0)
        avgpool_fwd4_kernel<<<row_grid(((W - 1) / 2 + 1) * (C / 4), nimg * ((H - 1) / 2 + 1)), 256, 0, s>>>(
            x, xs, xo, nimg, H, W, C / 4,
                                                            reinterpret_cast<Bf16x4 *>(y));
    else
        avgpool_fwd_kernel<<<grid_for(n), 256, 0, s>>>(x, xs, xo, nimg, H, W, C, y);
}
void launch_avgpool_bwd(const float *dy, int nimg, int H, int W, int C, float *dx, int accumulate, cudaStream_t s) {
    const long long n = (long long)nimg * H * W * C;
    if (C % 4 == 0 && (((uintptr_t)dy | (uintptr_t)dx) & 15) == 0)
        avgpool_bwd4_kernel<<<grid_for(n / 4), 256, 0, s>>>(dy, nimg, H, W, C / 4, dx, accumulate);
    else
        avgpool_bwd_kernel<<<grid_for(n), 256, 0, s>>>(dy, nimg, H, W, C, dx, accumulate);
}
bool launch_split_cat(const float *src, int nimg, int H, int W, int C, float *skip, __nv_bfloat16 *up,
                      cudaStream_t s) {
    if (C % 4 != 0 || (H | W) & 1 || (((uintptr_t)src | (uintptr_t)skip) & 15) != 0 || ((uintptr_t)up & 7) != 0)
        return false;
    const long long P = (long long)nimg * H * W;
    split_cat4_kernel<<<row_grid(W * (C / 4), nimg * H), 256, 0, s>>>(src, nimg, H, W, C / 4,
                                                                      reinterpret_cast<float4 *>(skip),
                                                          reinterpret_cast<Bf16x4 *>(up));
    return true;
}
void launch_to_bf16_s2d(const float *x, int nimg, int H, int W, int C, __nv_bfloat16 *y, cudaStream_t s) {
    to_bf16_s2d_kernel<<<grid_for((long long)nimg * 4 * H * W * C), 256, 0, s>>>(x, nimg, H, W, C, y);
}
bool launch_avgpool_bwd_leaky(const float *dy, int nimg, int H, int W, int C, const float *skip,
                              const __nv_bfloat16 *act, int as, int ao, float slope, __nv_bfloat16 *g,
                              cudaStream_t s) {
    if (C % 4 != 0 || ((as | ao) & 3) != 0 || (((uintptr_t)dy | (uintptr_t)skip) & 15) != 0 ||
        (((uintptr_t)act | (uintptr_t)g) & 7) != 0)
        return false;
    const long long n = (long long)nimg * H * W * C;
    avgpool_bwd_leaky4_kernel<<<row_grid(W * (C / 4), nimg * H), 256, 0, s>>>(dy, nimg, H, W, C / 4,
                                                              reinterpret_cast<const float4 *>(skip), act, as, ao,
                                                              slope, reinterpret_cast<Bf16x4 *>(g));
    return true;
}
void launch_leaky_bwd(const float *dA, const __nv_bfloat16 *a, int as, int ao, long long P, int C, float slope,
                      __nv_bfloat16 *g, cudaStream_t s) {
    if (C % 4 == 0 && ((as | ao) & 3) == 0 && (((uintptr_t)a | (uintptr_t)g) & 7) == 0 && ((uintptr_t)dA & 15) == 0)
        leaky_bwd4_kernel<<<grid_for(P * C / 4), 256, 0, s>>>(reinterpret_cast<const float4 *>(dA), a, as, ao, P,
                                                              C / 4, slope, reinterpret_cast<Bf16x4 *>(g));
    else
        leaky_bwd_kernel<<<grid_for(P * C), 256, 0, s>>>(dA, a, as, ao, P, C, slope, g);
}
void launch_f32_to_bf16_slice(const float *x, int xs, int xo, long long P, int C, __nv_bfloat16 *y, cudaStream_t s) {
    if (C % 4 == 0 && ((xs | xo) & 3) == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 7) == 0)
        f32_to_bf16_slice4_kernel<<<grid_for(P * C / 4), 256, 0, s>>>(x, xs, xo, P, C / 4,
                                                                      reinterpret_cast<Bf16x4 *>(y));
    else
        f32_to_bf16_slice_kernel<<<grid_for(P * C), 256, 0, s>>>(x, xs, xo, P, C, y);
}
void launch_add_slice(const float *src, int ss, int so, long long P, int C, float *dst, cudaStream_t s) {
    if (C % 4 == 0 && ((ss | so) & 3) == 0 && (((uintptr_t)src | (uintptr_t)dst) & 15) == 0)
        add_slice4_kernel<<<grid_for(P * C / 4), 256, 0, s>>>(src, ss, so, P, C / 4, reinterpret_cast<float4 *>(dst));
    else
        add_slice_kernel<<<grid_for(P * C), 256, 0, s>>>(src, ss, so, P, C, dst);
}
void launch_conv1x1_fwd(const __nv_bfloat16 *a, int C, long long P, const __nv_bfloat16 *w, const float *b, float *out,
                        cudaStream_t s) {
    conv1x1_fwd_kernel<<<grid_for(P), 256, 0, s>>>(a, C, P, w, b, out);
}
void launch_mse(const float *out, const float *y, long long P, __nv_bfloat16 *g, double *partial, int nblocks,
                cudaStream_t s) {
    mse_kernel<<<nblocks, 256, 0, s>>>(out, y, P, g, partial);
}
void launch_conv1x1_bwd_leaky(const __nv_bfloat16 *g, const __nv_bfloat16 *a, long long P, int C,
                              const __nv_bfloat16 *w, float slope, __nv_bfloat16 *gn, float *part, int max_blocks,
                              float *dw_db, cudaStream_t s) {
    int rows = (int)((P + max_blocks - 1) / max_blocks);
    if (rows < 64) rows = 64;
    const int nblk = (int)((P + rows - 1) / rows);
    const int cx = ((C + 1 + 31) / 32) * 32;
    const int streams = std::max(1, std::min(8, 512 / cx));  // at most 512 threads (the kernel's bound)
    conv1x1_bwd_leaky_kernel<<<nblk, dim3(cx, streams), sizeof(float) * cx * streams, s>>>(g, a, P, C, w, slope, gn,
                                                                                             rows, part);
    bias_grad_final_kernel<<<((C + 1) * 32 + 255) / 256, 256, 0, s>>>(part, nblk, C + 1, dw_db);
}
void launch_adam(float *theta, const float *grad, float *m, float *v, long long n, float lr, float b1, float b2,
                 float eps, int t, __nv_bfloat16 *shadow, cudaStream_t s) {
    const float bc1 = 1.0f - powf(b1, (float)t), bc2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n), 256, 0, s>>>(theta, grad, m, v, n, lr, b1, b2, eps, bc1, bc2, shadow);
}
void launch_to_bf16(const float *x, long long n, __nv_bfloat16 *y, cudaStream_t s) {
    to_bf16_kernel<<<grid_for(n), 256, 0, s>>>(x, n, y);
}
void launch_bf16_to_f32(const __nv_bfloat16 *x, long long n, float *y, cudaStream_t s) {
    bf16_to_f32_kernel<<<grid_for(n), 256, 0, s>>>(x, n, y);
}
void launch_transpose_w(const __nv_bfloat16 *w, int co, int taps, int ci, __nv_bfloat16 *wt, cudaStream_t s) {
    transpose_w_kernel<<<grid_for((long long)co * taps * ci), 256, 0, s>>>(w, co, taps, ci, wt);
}
void launch_transpose_w_batch(const __nv_bfloat16 *w, __nv_bfloat16 *wt, const TransposeJobs &jobs, cudaStream_t s) {
    if (jobs.n <= 0) return;
    int most = 0;
    for (int j = 0; j < jobs.n; j++)
        most = std::max(most, ((jobs.co[j] + 31) / 32) * ((jobs.ci[j] + 31) / 32) * jobs.taps[j]);
    transpose_w_batch_kernel<<<dim3(most, jobs.n), 256, 0, s>>>(w, wt, jobs);
}

void launch_convt_tapmajor_batch(const __nv_bfloat16 *w, __nv_bfloat16 *wp, const TransposeJobs &jobs,
                                 cudaStream_t s) {
    if (jobs.n <= 0) return;
    long long most = 0;
    for (int j = 0; j < jobs.n; j++) most = std::max(most, 4LL * jobs.co[j] * jobs.ci[j]);
    convt_tapmajor_batch_kernel<<<dim3(grid_for(most), jobs.n), 256, 0, s>>>(w, wp, jobs);
}

void launch_input_pack(const float *x, long long P, int Cp, __nv_bfloat16 *y, cudaStream_t s) {
    input_pack_kernel<<<grid_for(P * Cp), 256, 0, s>>>(x, P, Cp, y);
}
void launch_gather_patches(const float *img, int nx, const int *oz, const int *ox, const int *sel, int nb, int p,
                           const float *scale, int mute, float *dst, cudaStream_t s) {
    gather_patches_kernel<<<grid_for((long long)nb * p * p), 256, 0, s>>>(img, nx, oz, ox, sel, nb, p, scale, mute,
                                                                          dst);
}
void launch_pad_image(const float *img, int nz, int nx, int Hp, int Wp, const float *scale, int mute, float *dst,
                      cudaStream_t s) {
    pad_image_kernel<<<grid_for((long long)Hp * Wp), 256, 0, s>>>(img, nz, nx, Hp, Wp, scale, mute, dst);
}
void launch_crop_image(const float *src, int Hp, int Wp, int nz, int nx, const float *scale, float *dst,
                       cudaStream_t s) {
    crop_image_kernel<<<grid_for((long long)nz * nx), 256, 0, s>>>(src, Hp, Wp, nz, nx, scale, dst);
}
int launch_first_wgrad(const __nv_bfloat16 *g, int co, const __nv_bfloat16 *xin, int cpad, int nimg, int H, int W,
                       float *part, long long part_floats, float *dw, float *db, cudaStream_t s) {
    const long long tasks = (long long)nimg * H * ((W + 31) / 32);
    int nblk = (int)std::min<long long>(152 * 8, (tasks + 7) / 8);
    if ((long long)nblk * co * 10 > part_floats) nblk = (int)(part_floats / (10LL * co));
    if (nblk < 1) return 0;
    first_wgrad_kernel<<<nblk, 256, 0, s>>>(g, co, xin, cpad, nimg, H, W, part);
    first_wgrad_final_kernel<<<co * 10, 256, 0, s>>>(part, nblk, co, dw, db);
    return 2;
}
bool launch_first_conv(const __nv_bfloat16 *xin, int cpad, int nimg, int H, int W, const __nv_bfloat16 *w,
                       const float *bias, int co, float slope, __nv_bfloat16 *y, int ys, cudaStream_t s) {
    if (co % 8 != 0 || ys % 8 != 0 || ((uintptr_t)y & 15) != 0) return false;
    if ((long long)nimg * H > 65535) return false;
    const dim3 grid((unsigned)(((long long)W * (co / 8) + 255) / 256), (unsigned)(nimg * H));
    first_conv_kernel<<<grid, 256, sizeof(float) * co * 10, s>>>(xin, cpad, nimg, H, W, w, bias, co, slope, y, ys);
    return true;
}
void launch_pad_first_w(const __nv_bfloat16 *w, int co, int cpad, __nv_bfloat16 *wp, cudaStream_t s) {
    pad_first_w_kernel<<<grid_for((long long)co * 9 * cpad), 256, 0, s>>>(w, co, cpad, wp);
}
void launch_unpad_first_grad(const float *gp, int co, int cpad, float *g, cudaStream_t s) {
    unpad_first_grad_kernel<<<grid_for((long long)co * 9), 256, 0, s>>>(gp, co, cpad, g);
}
void launch_loss_accum(const double *partial, int nblocks, double weight, double *acc, cudaStream_t s) {
    loss_accum_kernel<<<1, 1, 0, s>>>(partial, nblocks, weight, acc);
}
void launch_absmax(const float *x, long long n, unsigned *mx, float *scale_out, cudaStream_t s) {
    cudaMemsetAsync(mx, 0, sizeof(unsigned), s);
    absmax_kernel<<<grid_for(n), 256, 0, s>>>(x, n, mx);
    absmax_finish_kernel<<<1, 1, 0, s>>>(mx, scale_out);
}

}  // namespace nn
}  // namespace dhfwi
