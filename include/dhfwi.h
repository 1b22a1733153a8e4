/*
 * dhfwi.h - C ABI of the GB300 (sm_103a) implementation of the wave-equation
 * hot path of "Robust Full Waveform Inversion with deep Hessian deblurring"
 * (Alfarhan, Ravasi, Chen, Alkhalifah; arXiv 2403.17518).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Model arrays (velocity v, perturbation dv, gradient, image) are float32,
 *   row-major [nz][nx] with x fastest, in device memory owned by the caller.
 *   Velocity is in m/s (the paper's m(x) is the medium velocity, Section 2.1,
 *   Eq. 1).
 * - Data arrays are float32 device memory owned by the caller, packed shot
 *   after shot in shot order; shot s occupies nt[s] * nrec_s values laid out
 *   [nt_s][nrec_s] (time slow, receiver fast), nrec_s = rec_off[s+1]-rec_off[s].
 *   Sample n of a shot is the wavefield produced by time step n, i.e. at time
 *   (n+1)*dt.
 * - Geometry arrays (dhfwi_geom) are HOST memory owned by the caller; they are
 *   read during the call and cached on the device by content.
 * - `stream` is a cudaStream_t (0 = the legacy default stream).  Work is
 *   enqueued on it.  Every call first validates the model on the device and
 *   waits for that check (one stream synchronisation); calls that return host
 *   scalars (misfit_out, loss_hist) synchronise the stream again before
 *   returning.  Calls on one context must not run concurrently from several
 *   host threads.
 * - Every call returns DHFWI_OK (0) or a negative DHFWI_ERR_* code; a message
 *   is then available from dhfwi_last_error().  No C++ exception crosses this
 *   boundary.  On error, output buffers hold unspecified values.
 *
 * Discretisation (what every propagator computes)
 * -----------------------------------------------
 * Eq. 1 (Section 2.1), constant-density acoustic: m^-2 u_tt - lap(u) = f.
 * Per shot, the padded domain is the physical column window
 * [win_x0, win_x1) extended by nb cells on all four sides (velocity there is
 * the model's, indices clamped to the model).  With kappa = v^2 dt^2/h^2,
 * D the unscaled 8th-order Laplacian (zero outside the padded domain) and w
 * the Cerjan sponge factor exp(-(0.015 (nb - d))^2) per axis (d = cells from
 * the domain's outer edge, 1 inside):
 *     a^n     = D u^n + q^n          (q^n = wavelet[n] at the source node)
 *     u^{n+1} = w (2 u^n + kappa a^n) - w^2 u^{n-1},   u^0 = u^{-1} = 0
 *     d[n][r] = u^{n+1} at receiver r,                 n = 0 .. nt_s-1
 */
#ifndef DHFWI_H
#define DHFWI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DHFWI_OK 0
#define DHFWI_ERR_ARG (-1)        /* null pointer, bad size or bad config value */
#define DHFWI_ERR_GEOM (-2)       /* source, receiver or window outside the grid */
#define DHFWI_ERR_CFL (-3)        /* kappa_max * 13.0032 > 4: the scheme is unstable */
#define DHFWI_ERR_NONFINITE (-4)  /* non-finite or non-positive velocity, or non-finite result */
#define DHFWI_ERR_OOM (-5)        /* device allocation failed */
#define DHFWI_ERR_TIMEOUT (-6)    /* a bounded device-side wait ran out (a step kernel's tile copies did
                                     not land within ~1 s); reported by the call itself when it
                                     synchronises (misfit_out, data_misfit, loss_hist), else by the
                                     next call on the context */
#define DHFWI_ERR_CUDA (-7)       /* any other CUDA runtime error */
#define DHFWI_ERR_STATE (-8)      /* call made in the wrong state (e.g. apply before train) */

/* Born/migration parameterisation flags (born_demig / rtm_mig `flags`). */
#define DHFWI_ABS 0  /* dv is an absolute velocity perturbation in m/s */
#define DHFWI_REL 1  /* dv is relative, dv_abs = v0 * dv (Section 2.2, after Eq. 12) */

typedef struct dhfwi_ctx dhfwi_ctx;

/* Physical grid: nz rows (depth, row 0 at the surface) by nx columns, spacing
 * h metres in both directions, time step dt seconds, sponge width nb cells
 * (0 <= nb <= 64). */
typedef struct {
    int nz, nx, nb;
    float h, dt;
} dhfwi_grid;

/* Acquisition geometry, all HOST pointers.
 *   src_iz, src_ix [n_shots]  source node (physical row, column)
 *   nt             [n_shots]  record length of each shot (samples), 0..nt_max
 *   rec_off        [n_shots+1] CSR offsets into rec_iz / rec_ix
 *   rec_iz, rec_ix [rec_off[n_shots]] receiver nodes
 *   win_x0, win_x1 [n_shots]  physical column window [x0, x1) of each shot;
 *                             its source and receivers must lie inside it
 *   wavelet        [nt_max] if wavelet_shared, else [n_shots][nt_max]
 */
typedef struct {
    int n_shots;
    const int *src_iz, *src_ix, *nt;
    const int *rec_off;
    const int *rec_iz, *rec_ix;
    const int *win_x0, *win_x1;
    const float *wavelet;
    int nt_max;
    int wavelet_shared;
} dhfwi_geom;

/* Per-context counters of the last call (host struct filled by dhfwi_stats). */
typedef struct {
    long long cell_updates;   /* stencil cell updates of the last call (all wavefields) */
    long long kernel_launches;/* kernels this library launched in the last call */
    int checkpoint_every;     /* forward checkpoint interval used (steps) */
    int shot_groups;          /* number of shot groups the memory planner used */
    double workspace_bytes;   /* device workspace held by the context */
    /* Device time of the phases of the last call, from CUDA events recorded on
     * the call's stream around each phase (0 unless timing is on, see
     * dhfwi_set_timing).  Phase 0: forward passes (forward step kernel only,
     * storing the a^n history where it covers the step); 1: backward sweeps
     * (adjoint step kernels, plus the segment recompute for steps outside the
     * history); 2: Born joint passes. */
    double phase_ms[3];
    long long phase_launches[3];
    long long phase_cells[3];  /* cell updates in that phase (Born counts 2 per cell) */
    /* Step-kernel variant chosen by the autotuner for: forward, forward with
     * segment store, adjoint, Born (index into the library's variant table). */
    int step_variant[4];
    /* Steps whose a^n (the Laplacian term of the forward update, which the
     * gradient and migration images correlate with the adjoint field) the
     * last fwi_gradient or rtm_mig call stored during its forward pass; the
     * backward sweep recomputes the other steps from checkpoints.  The
     * history is as long as device memory allows, or as DHFWI_HISTORY_MB
     * (MiB, environment, 0 = none) caps it; results are the same bit for bit
     * either way. */
    int history_steps;
    long long history_cells;   /* phase-0 cell updates that also stored a^n */
    /* Time steps per launch (1 or 2) of the forward and the adjoint sweeps:
     * the autotuner times both depths per geometry; DHFWI_TIME_BLOCK=0
     * (environment) forces 1, any other value 2. */
    int time_block[2];
    /* What the last call took from the stored forward pass of an earlier
     * call (dhfwi_set_reuse): bit 0, rtm_mig skipped its forward pass; bit 1,
     * born_demig read the background term from the history. */
    int reused;
} dhfwi_stats_t;

/* Create a context on CUDA device `device` for grid `g`.  The context owns all
 * device workspace (wavefields, checkpoints, network weights and Adam state);
 * the caller owns every argument buffer.  Returns DHFWI_OK and *out, or an
 * error code (*out is then NULL). */
int dhfwi_create(dhfwi_ctx **out, const dhfwi_grid *g, int device);

/* Release the context and its device workspace.  Accepts NULL. */
void dhfwi_destroy(dhfwi_ctx *ctx);

/* Message of the last error on this context (never NULL; "" after success).
 * With ctx == NULL, the message of the last failed dhfwi_create. */
const char *dhfwi_last_error(const dhfwi_ctx *ctx);

/* Counters of the last call on this context.  With timing on, waits for the
 * phase events of the last call to complete. */
int dhfwi_stats(const dhfwi_ctx *ctx, dhfwi_stats_t *out);

/* Turn per-phase CUDA-event timing on (1) or off (0) for later calls. */
int dhfwi_set_timing(dhfwi_ctx *ctx, int on);

/* Reuse of the forward wavefield between calls, off by default (no
 * counterpart in the paper: an implementation choice for the FWI iteration,
 * whose gradient, Born demigration and migration all propagate the same
 * background field).  With reuse on, a backward-capable forward pass
 * (fwi_gradient, rtm_mig) leaves its a^n history and checkpoints intact
 * (the segment recompute of the backward sweep starts from copies of the
 * checkpoints), and a later rtm_mig or born_demig at the same velocity model
 * and geometry takes the background from them instead of propagating it
 * again: rtm_mig skips its forward pass, and born_demig, when the history
 * holds every step, advances only the scattered field, reading the
 * background term a^n = D u0^n + q^n.  The model is identified by a 64-bit
 * hash of its values computed on the device at every call, the geometry by
 * the plan's content hash; a changed model, geometry or workspace split
 * falls back to propagating.  Results are the same bits either way.  Calls
 * report what they reused in dhfwi_stats_t.reused. */
int dhfwi_set_reuse(dhfwi_ctx *ctx, int on);

/* Forward shot modelling (Section 2.1: "the wave equation is solved using a
 * forward modeling scheme such as the finite difference method to obtain the
 * simulated data d_s").  All shots run in one batched pass.
 *   v_dev  [nz][nx] velocity (m/s), device
 *   d_dev  packed records (see above), device, written */
int model_shots(dhfwi_ctx *ctx, const float *v_dev, const dhfwi_geom *geom, float *d_dev,
                void *stream);

/* Misfit and adjoint-state gradient (Section 2.1 Eq. 2; Section 2.3.1 Eq. 13).
 *   misfit_out (host, may be NULL)  J = 1/2 sum (d_s - d_o)^2
 *   grad_dev   [nz][nx] device, written with dJ/dv (m/s)^-1 scaled units.
 *              The paper's g = L~^T (d_o - d_s) equals -grad.
 *   d_syn_dev  optional (may be NULL) packed synthetic records d_s.
 * The forward pass stores a^n of as many steps as device memory allows (see
 * history_steps in dhfwi_stats_t); the backward sweep recomputes the others
 * from checkpoints.  Synchronises the stream when misfit_out is not NULL. */
int fwi_gradient(dhfwi_ctx *ctx, const float *v_dev, const dhfwi_geom *geom,
                 const float *d_obs_dev, float *grad_dev, double *misfit_out, float *d_syn_dev,
                 void *stream);

/* Born demigration d = L~ dv (Section 2.2 Eqs. 9-12b): the background field
 * (Eq. 9) and the scattered field (Eq. 11) advance together in one kernel, so
 * the background wavefield is never stored.  This is the exact tangent of
 * model_shots at v0.
 *   dv_dev [nz][nx] device: perturbation (absolute m/s, or relative with
 *          flags = DHFWI_REL)
 *   d_dev  packed Born records, device, written */
int born_demig(dhfwi_ctx *ctx, const float *v0_dev, const dhfwi_geom *geom, const float *dv_dev,
               float *d_dev, int flags, void *stream);

/* Migration img = L~^T d (Section 2.3.1 Eq. 13 applied to arbitrary data; the
 * exact transpose of born_demig with the same flags).  The doubly migrated
 * image of Eq. 15 is rtm_mig(born_demig(g)).  Workspace as fwi_gradient.
 *   d_dev   packed records, device
 *   img_dev [nz][nx] device, written */
int rtm_mig(dhfwi_ctx *ctx, const float *v0_dev, const dhfwi_geom *geom, const float *d_dev,
            float *img_dev, int flags, void *stream);

/* Model update along a direction (Section 2.1 Eq. 4 with the inverse Hessian
 * replaced by a scalar step, or by the network for the deblurred direction):
 *   v_out = clamp(v - alpha * dir / max|dir|, vmin, vmax),
 * with dir taken as 0 in the first mute_rows rows (source/receiver footprint;
 * those rows are also left out of the max).  v_dev, dir_dev, v_out_dev
 * [nz][nx] float32 device (v_out may equal v).  Asynchronous. */
int fwi_update(dhfwi_ctx *ctx, const float *v_dev, const float *dir_dev, float alpha, float vmin, float vmax,
               int mute_rows, float *v_out_dev, void *stream);

/* Barzilai-Borwein short step of the plain-gradient arm (Section 3.1, Eq. 17):
 *   alpha = (dx . dg) / (dg . dg),  dx = x_k - x_prev,  dg = g_k - g_prev,
 * the differences and sums in float64, over the rows from mute_rows down
 * (the rows the update leaves unchanged are left out).  The BB update is
 * x_{k+1} = x_k - alpha g_k, i.e. fwi_update with alpha * max|g_k| (the
 * normalisation of fwi_update divides by max|g_k|); gmax_out (may be NULL)
 * receives max|g_k| over the same rows.  x_*, g_* [nz][nx] float32 device.
 * DHFWI_ERR_NONFINITE when dg is zero.  Synchronises the stream. */
int bb_step(dhfwi_ctx *ctx, const float *x_k, const float *x_prev, const float *g_k, const float *g_prev,
            int mute_rows, double *alpha_out, double *gmax_out, void *stream);

/* Quality-control filter of a migrated image (Section 3.3 images the data
 * with the estimated models to validate them; the paper names no filter, so
 * this is the reading adopted): out = -(D2 img) / h^2 with D2 the 5-point
 * Laplacian, the image's edge values repeated outside the grid.  It damps
 * the low-wavenumber part of a migration image.  img_dev, out_dev
 * [nz][nx] float32 device (out must not alias img).  Asynchronous. */
int image_laplacian(dhfwi_ctx *ctx, const float *img_dev, float *out_dev, void *stream);

/* Self-test of the failure path (no counterpart in the paper): launches one
 * kernel whose bounded device-side wait (~1 s, the step kernels' limit) runs
 * out on a barrier that nothing arrives at; it records that as a timed-out
 * step kernel does, so the next call on this context returns
 * DHFWI_ERR_TIMEOUT and clears the record, and later calls work normally.
 * Nothing faults or hangs.  Asynchronous. */
int dhfwi_selftest_timeout(dhfwi_ctx *ctx, void *stream);

/* Data misfit J = 1/2 sum (a - b)^2 (Section 2.1 Eq. 2) of two device
 * vectors of n float32 values, accumulated in float64.  Synchronises. */
int data_misfit(dhfwi_ctx *ctx, const float *a_dev, const float *b_dev, long long n, double *misfit_out,
                void *stream);

/* ------------------------------------------------------------------------
 * Forward modelling without device allocation.  The paper has no
 * counterpart: this serves callers that may not call cudaMalloc (code running
 * inside a framework that owns every device allocation, memory-capped
 * services, or callers that must avoid the device synchronisation that
 * cudaMalloc/cudaFree can cause).
 *
 * model_shots_static computes what model_shots computes (the same
 * recurrence), without a context, with the one-step cp.async step kernel
 * (the variant model_shots runs with DHFWI_TIME_BLOCK=0 and
 * DHFWI_STEP_VARIANT=1, whose records it reproduces bit for bit; the
 * default model_shots path agrees to relative L2 1e-5).  All its temporary buffers
 * (padded model arrays, wavefield state, geometry tables) live in one
 * file-scope device array of DHFWI_STATIC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits; it calls no
 * cudaMalloc, cudaFree or allocating library routine.  The caller passes
 * v_dev ([nz][nx] float32, device) and d_dev (packed records, device), as for
 * model_shots.
 *   - Problems whose scratch exceeds the array return DHFWI_ERR_ARG with the
 *     sizes in model_shots_static_error().
 *   - It runs on the CURRENT device: v_dev, d_dev and stream must belong to
 *     it (make the device current first, e.g. cudaSetDevice).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it; make that
 *     first call before any stream capture.  A cudaDeviceReset of that
 *     device invalidates the kept address: do not call model_shots_static
 *     again in a process that has reset a device it used.
 *   - Every call shares the array and leaves its contents behind (each call
 *     clears what must start at zero); calls that overlap on the GPU (other
 *     streams, other host threads, other contexts of the same device) race.
 *   - Synchronises `stream` once, for the velocity/CFL check.
 * ------------------------------------------------------------------------ */
#define DHFWI_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

int model_shots_static(const dhfwi_grid *g, const float *v_dev, const dhfwi_geom *geom, float *d_dev,
                       void *stream);

/* Message of the last failed model_shots_static call of this host thread. */
const char *model_shots_static_error(void);

/* ------------------------------------------------------------------------
 * Deblurring network: an approximate inverse Hessian (Section 2.3.1 and
 * Section 2.4, architecture in Appendix A).  A UNet-like network is trained to
 * map the doubly migrated image delta m_1 (Eq. 15) to the gradient g
 * (Eq. 13), then applied to g to obtain the update direction; weights carry
 * over between training calls (transfer learning).  Convolutions run with
 * bfloat16 operands and float32 accumulation; master weights, Adam moments,
 * loss and schedule are float32.
 *
 * Parameters are one flat float32 vector, tensor after tensor: input block
 * (conv 1->B, conv B->B), `levels` down blocks (conv, conv), `levels` up blocks
 * (transposed conv, conv on [skip, up], conv), output 1x1 conv B->1.  A 3x3
 * conv stores weight [Cout][3][3][Cin] then bias [Cout]; the 2x2 stride-2
 * transposed conv weight [Cout][2][2][Cin] (output pixel (2h+a, 2w+b) gets
 * W[co][a][b][:] . x[h][w]) then bias; the 1x1 conv [Cout][Cin] then bias.
 * ------------------------------------------------------------------------ */
typedef struct {
    int base_channels;  /* channels of the input block (multiple of 8, 8..256); 32 here, 128 in the paper */
    int levels;         /* down/up blocks (4 in the paper) */
    int patch;          /* square patch size (multiple of 2^levels); 0: full-image training, the
                           paper's choice (Section 2.4): the whole image, zero-padded at the bottom
                           and right to a multiple of 2^levels, is the one sample of every step
                           (batch 1; stride and batch are ignored; the loss is the mean over the
                           padded frame) */
    int stride;         /* patch stride; the last patch of each axis touches the edge */
    int batch;          /* patches per optimiser step */
    int epochs;         /* passes over the patches (<= 4096); optimiser steps when patch is 0 */
    float lr;           /* initial learning rate of the cosine schedule */
    float beta1, beta2, eps;     /* Adam */
    unsigned long long seed;     /* initialisation (cold start) and shuffling */
    int mute_rows;               /* rows from the top taken as 0 in x and y (source/receiver
                                    footprint); also used by deblur_apply */
    float warmup_frac;           /* linear learning-rate ramp over this fraction of the call's
                                    steps (0 = none), in [0, 1] */
} dhfwi_train_cfg;

/* Fix the architecture and initialise the weights from `seed` (SplitMix64,
 * uniform in +-1/sqrt(fan_in)).  Synchronous. */
int dhfwi_net_init(dhfwi_ctx *ctx, int base_channels, int levels, unsigned long long seed);

/* Number of float32 parameters of the current network (0 if none). */
long long dhfwi_net_size(const dhfwi_ctx *ctx);

/* Copy the float32 master weights to / from HOST memory (n = dhfwi_net_size).
 * Synchronous.  net_set requires a prior dhfwi_net_init (architecture). */
int dhfwi_net_get(dhfwi_ctx *ctx, float *host, size_t n);
int dhfwi_net_set(dhfwi_ctx *ctx, const float *host, size_t n);

/* Network output for a batch: x_dev [n][h][w] float32 (one channel, device),
 * out_dev [n][h][w] float32 (device); h, w multiples of 2^levels.  No
 * normalisation.  Asynchronous on `stream`. */
int deblur_forward(dhfwi_ctx *ctx, const float *x_dev, int n, int h, int w, float *out_dev, void *stream);

/* One forward + MSE + backward on a batch: grad_dev (device, float32,
 * dhfwi_net_size values) receives dL/dtheta of L = mean((net(x) - y)^2);
 * loss_out (host, may be NULL) receives L and synchronises the stream. */
int deblur_grad(dhfwi_ctx *ctx, const float *x_dev, const float *y_dev, int n, int h, int w, float *grad_dev,
                double *loss_out, void *stream);

/* Train on the pair (x = doubly migrated image, y = gradient), both [nz][nx]
 * float32 device images, each normalised by its max |.| below the first
 * cfg->mute_rows rows (which are taken as 0), cut into patches.
 * Adam with lr_t = lr (1 + cos(pi t / T)) / 2 over the T steps of this call,
 * times min(1, (t+1)/W) for W = ceil(warmup_frac T) warm-up steps; fresh Adam
 * moments at every call; warm_start != 0 keeps the current weights (transfer
 * learning), 0 re-initialises them from cfg->seed.
 * loss_hist (host, may be NULL): cfg->epochs per-epoch mean MSE; when given,
 * the stream is synchronised.  Errors: DHFWI_ERR_ARG for a bad cfg. */
int deblur_train(dhfwi_ctx *ctx, const float *x_dev, const float *y_dev, int nz, int nx,
                 const dhfwi_train_cfg *cfg, int warm_start, float *loss_hist, void *stream);

/* One convolution layer of the network on its own, with the kernels the
 * network runs for it (Appendix A layers: the 3x3 convolutions and the 2x2
 * stride-2 transposed convolutions of the up blocks), so that each GEMM path
 * can be checked against a reference layer by layer.  All arrays float32
 * device memory, NHWC:
 *   x  [n][H][W][ci]   layer input (rounded to bfloat16 as the network does)
 *   w  weights in the parameter layout of deblur's flat vector
 *      ([co][3][3][ci] or [co][2][2][ci]; rounded to bfloat16), b [co]
 *   gy [n][Ho][Wo][co] gradient of the layer output (rounded to bfloat16),
 *      Ho, Wo = H, W (3x3) or 2H, 2W (transposed)
 *   out  DHFWI_LAYER_FWD: [n][Ho][Wo][co], the stored activation:
 *          bf16(LeakyReLU_0.2(conv(x) + b)) for the 3x3 convolution,
 *          bf16(convT(x) + b) for the transposed one (widened to float32);
 *        DHFWI_LAYER_DGRAD: [n][H][W][ci] = dL/dx for dL/dy = gy;
 *        DHFWI_LAYER_WGRAD: dL/dw (parameter layout) then dL/db [co].
 * ci and co are multiples of 8.  Kind DHFWI_LAYER_FIRST is the network's
 * first 3x3 convolution, whose input has one channel (ci = 1; co a multiple
 * of 8), on the CUDA-core kernels the network runs for it; FWD and WGRAD
 * only.  Unused pointers may be NULL.  Allocates its temporaries and
 * synchronises the stream. */
#define DHFWI_LAYER_CONV3 0
#define DHFWI_LAYER_CONVT 1
#define DHFWI_LAYER_FIRST 2
#define DHFWI_LAYER_FWD 0
#define DHFWI_LAYER_DGRAD 1
#define DHFWI_LAYER_WGRAD 2
int deblur_layer(dhfwi_ctx *ctx, int kind, int op, int n, int H, int W, int ci, int co, const float *x_dev,
                 const float *w_dev, const float *b_dev, const float *gy_dev, float *out_dev, void *stream);

/* Update direction from the gradient (Section 2.3.1): out = net(g / max|g|)
 * * max|g| on the full image, zero padded to a multiple of 2^levels and
 * cropped; the first mute_rows rows (of the last training cfg) of g are taken
 * as 0 and excluded from max|g|.  g_dev, out_dev [nz][nx] float32 device.  DHFWI_ERR_STATE before
 * the network has weights. */
int deblur_apply(dhfwi_ctx *ctx, const float *g_dev, int nz, int nx, float *out_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DHFWI_H */
