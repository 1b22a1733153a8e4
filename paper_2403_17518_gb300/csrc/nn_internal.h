// Internal declarations of the deblurring-network kernels (nn_kernels.cu)
// used by the network host code (nn_net.cu).  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dhfwi {
namespace nn {

// Epilogues of the forward-form GEMM: bf16 with bias and LeakyReLU, bf16
// with bias, transposed-conv scatter, f32 store, f32 accumulate, and bf16 of
// the result times the LeakyReLU derivative of a stored activation (act),
// i.e. an input gradient fused with the next layer's activation backward.
enum { EPI_BF16_LEAKY = 0, EPI_BF16 = 1, EPI_BF16_CONVT = 2, EPI_F32 = 3, EPI_F32_ADD = 4, EPI_BF16_LEAKYBWD = 5 };
enum { WG_CONV = 0, WG_CONVT = 1 };

// Implicit GEMM C[m][n] = sum_k A[m][k] B^T[n][k]; see igemm_fprop_kernel.
struct FpropArgs {
    const __nv_bfloat16 *src;   // NHWC source, channel stride src_stride, offset src_off
    int src_stride, src_off;
    int Hs, Ws;                 // source grid
    int C;                      // channels per tap (multiple of 8)
    int ntaps, scale;
    int dh[9], dw[9];
    int Ho, Wo;                 // output grid (m = img*Ho*Wo + ho*Wo + wo)
    int M, N;
    const __nv_bfloat16 *bt;    // [N][ntaps*C]
    const float *bias;          // [N] (or [N/4] for the transposed conv)
    float slope;
    __nv_bfloat16 *dst_bf16;
    float *dst_f32;
    int dst_stride, dst_off;
    float *part;                // optional split-k scratch ([splits][M][N] float32)
    long long part_floats;      // its capacity
    unsigned *err;              // nullable: set to 1 by a tensor-core GEMM whose bounded wait ran out
    const __nv_bfloat16 *act;   // EPI_BF16_LEAKYBWD: activation [M][act_stride] at act_off
    int act_stride, act_off;
};

// Split-k weight-gradient GEMM; see igemm_wgrad_kernel.
struct WgradArgs {
    int mode;
    const __nv_bfloat16 *g;     // output gradient (NHWC, stride g_stride)
    int g_stride;
    const __nv_bfloat16 *x;     // layer input (NHWC, stride x_stride, offset x_off)
    int x_stride, x_off;
    int nimg, H, W;             // grid of the summed pixels (coarse grid for WG_CONVT)
    int co, ci;                 // channels (co used by WG_CONVT, ci by WG_CONV)
    int M, N;                   // N = nw + 8: weight columns, then a ones column (bias) and 7 zero columns
    int nw;                     // weight columns (9*ci for WG_CONV, ci for WG_CONVT)
    const __nv_bfloat16 *ones;  // 8 bf16 values {1, 0, ..., 0}
    float *part;                // [splits][M][N]
    unsigned *err;              // nullable: set to 1 by a tensor-core GEMM whose bounded wait ran out
    // WG_CONVT only: g is the output gradient in space-to-depth layout
    // [coarse pixel][ab][co] (row stride g_stride = 4 co), i.e. column m =
    // ab*Co + co of coarse pixel k, so the weight gradient is a one-tap GEMM.
    bool g_s2d = false;
};

// mma.sync GEMM (igemm_fprop_kernel), or the tcgen05 one (nn_umma.cu) when
// DHFWI_NN_GEMM=tc.
void launch_fprop(const FpropArgs &a, int epi, cudaStream_t s);
void launch_fprop_umma(const FpropArgs &a, int epi, cudaStream_t s);
// TMA-fed tcgen05 kernel for the 3x3 convolutions with >= 64 output channels
// (nn_umma.cu); false when the GEMM is not of that form (nothing launched).
bool launch_conv3_tma(const FpropArgs &a, int epi, cudaStream_t s);
// tcgen05 3x3 convolution with the input patch staged once for all nine
// taps (nn_umma.cu), for sources of 32 or 64 channels and at most 128
// outputs; false when not applicable (nothing launched).
bool launch_conv3_patch(const FpropArgs &a, int epi, cudaStream_t s);
// tcgen05 weight gradient of a 3x3 convolution (nn_umma.cu; off with
// DHFWI_NN_WGRAD=mma or DHFWI_NN_GEMM=mma): the splits it wrote (partials
// with the bias column), 0 when not applicable.
int launch_wgrad_tma(const WgradArgs &a, int max_splits, cudaStream_t s);
// Sum of split-k partials a.part[splits][M][N] with the epilogue epi.
void launch_fprop_reduce(const FpropArgs &a, int epi, int splits, cudaStream_t s);
int wgrad_splits(long long kpix, int M, int N);
// Weight gradient into dw (parameter layout) and bias gradient into db.
// Returns the number of kernels launched.
int launch_wgrad(const WgradArgs &a, int splits, float *dw, float *db, cudaStream_t s);
void launch_avgpool_fwd(const __nv_bfloat16 *x, int xs, int xo, int nimg, int H, int W, int C, __nv_bfloat16 *y,
                        cudaStream_t s);
void launch_avgpool_bwd(const float *dy, int nimg, int H, int W, int C, float *dx, int accumulate, cudaStream_t s);
void launch_leaky_bwd(const float *dA, const __nv_bfloat16 *a, int as, int ao, long long P, int C, float slope,
                      __nv_bfloat16 *g, cudaStream_t s);
void launch_f32_to_bf16_slice(const float *x, int xs, int xo, long long P, int C, __nv_bfloat16 *y, cudaStream_t s);
// Fused forms (false: not launched, shapes or alignment not met): d(cat)
// [P][2C] on an H x W grid into its skip half (f32, [P][C]) and upsampled
// half (bf16, space-to-depth onto the H/2 x W/2 grid, see WgradArgs::g_s2d); the average
// pool's backward plus a skip gradient times the LeakyReLU derivative of
// act, in bf16 (avgpool_bwd, add_slice and leaky_bwd in one pass).
bool launch_split_cat(const float *src, int nimg, int H, int W, int C, float *skip, __nv_bfloat16 *up,
                      cudaStream_t s);
// f32 output gradient of a transposed conv on the fine grid (nimg x 2H x 2W x
// C) into bf16 space-to-depth layout [nimg][H][W][2a+b][C].
void launch_to_bf16_s2d(const float *x, int nimg, int H, int W, int C, __nv_bfloat16 *y, cudaStream_t s);
bool launch_avgpool_bwd_leaky(const float *dy, int nimg, int H, int W, int C, const float *skip,
                              const __nv_bfloat16 *act, int as, int ao, float slope, __nv_bfloat16 *g,
                              cudaStream_t s);
void launch_add_slice(const float *src, int ss, int so, long long P, int C, float *dst, cudaStream_t s);
void launch_conv1x1_fwd(const __nv_bfloat16 *a, int C, long long P, const __nv_bfloat16 *w, const float *b, float *out,
                        cudaStream_t s);
void launch_mse(const float *out, const float *y, long long P, __nv_bfloat16 *g, double *partial, int nblocks,
                cudaStream_t s);
// Output layer backward fused with the LeakyReLU backward of its input a
// (bf16 [P][C]): the next block's output gradient gn (bf16 [P][C]) and the
// layer's weight and bias gradients (dw_db[0..C), dw_db[C]).
void launch_conv1x1_bwd_leaky(const __nv_bfloat16 *g, const __nv_bfloat16 *a, long long P, int C,
                              const __nv_bfloat16 *w, float slope, __nv_bfloat16 *gn, float *part, int max_blocks,
                              float *dw_db, cudaStream_t s);
void launch_adam(float *theta, const float *grad, float *m, float *v, long long n, float lr, float b1, float b2,
                 float eps, int t, __nv_bfloat16 *shadow, cudaStream_t s);
void launch_to_bf16(const float *x, long long n, __nv_bfloat16 *y, cudaStream_t s);
void launch_bf16_to_f32(const __nv_bfloat16 *x, long long n, float *y, cudaStream_t s);
void launch_transpose_w(const __nv_bfloat16 *w, int co, int taps, int ci, __nv_bfloat16 *wt, cudaStream_t s);
// Several layers' transposes [co][taps][ci] -> [ci][taps][co] in one launch,
// each at its parameter offset in w and wt.
struct TransposeJobs {
    static constexpr int MAX = 32;
    int n;
    long long off[MAX];
    int co[MAX], taps[MAX], ci[MAX];
};
void launch_transpose_w_batch(const __nv_bfloat16 *w, __nv_bfloat16 *wt, const TransposeJobs &jobs, cudaStream_t s);
// Transposed-conv weights [co][4][ci] -> [4][co][ci] (jobs' taps ignored):
// the B^T of the transposed convolutions' forward GEMM, whose columns are
// tap-major (n = tap * co + channel) in every EPI_BF16_CONVT epilogue.
void launch_convt_tapmajor_batch(const __nv_bfloat16 *w, __nv_bfloat16 *wp, const TransposeJobs &jobs,
                                 cudaStream_t s);
void launch_input_pack(const float *x, long long P, int Cp, __nv_bfloat16 *y, cudaStream_t s);
void launch_gather_patches(const float *img, int nx, const int *oz, const int *ox, const int *sel, int nb, int p,
                           const float *scale, int mute, float *dst, cudaStream_t s);
void launch_pad_image(const float *img, int nz, int nx, int Hp, int Wp, const float *scale, int mute, float *dst,
                      cudaStream_t s);
void launch_crop_image(const float *src, int Hp, int Wp, int nz, int nx, const float *scale, float *dst,
                       cudaStream_t s);
void launch_absmax(const float *x, long long n, unsigned *mx, float *scale_out, cudaStream_t s);
void launch_pad_first_w(const __nv_bfloat16 *w, int co, int cpad, __nv_bfloat16 *wp, cudaStream_t s);
void launch_unpad_first_grad(const float *gp, int co, int cpad, float *g, cudaStream_t s);
// The first convolution (one real input channel, channel 0 of xin; weights
// bf16 [co][9]) with bias and LeakyReLU into y (bf16, row stride ys), on
// CUDA cores; false when co or the output alignment does not allow it.
bool launch_first_conv(const __nv_bfloat16 *xin, int cpad, int nimg, int H, int W, const __nv_bfloat16 *w,
                       const float *bias, int co, float slope, __nv_bfloat16 *y, int ys, cudaStream_t s);
// Weight ([co][9]) and bias gradients of the first convolution from its
// output gradient g ([P][co] bf16) and its one-channel input (channel 0 of
// xin, cpad channels per pixel); part: scratch of part_floats floats.
// Returns the kernels launched (0: scratch too small, nothing launched).
int launch_first_wgrad(const __nv_bfloat16 *g, int co, const __nv_bfloat16 *xin, int cpad, int nimg, int H, int W,
                       float *part, long long part_floats, float *dw, float *db, cudaStream_t s);
void launch_loss_accum(const double *partial, int nblocks, double weight, double *acc, cudaStream_t s);

}  // namespace nn
}  // namespace dhfwi
