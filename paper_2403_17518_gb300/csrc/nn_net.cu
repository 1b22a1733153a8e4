// Deblurring network (Section 2.4 / Appendix A of arXiv 2403.17518) on the
// GPU: parameter state, activation workspace, forward, backward, Adam
// training with cosine annealing on image patches, and full-image apply.
//
// Per FWI iteration the network learns the map from the doubly migrated
// image (Eq. 15) to the gradient (Eq. 13) and is then applied to the
// gradient (Section 2.3.1); weights carry over between calls when
// warm_start is set (transfer learning, Section 2.3.1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dhfwi.h"
#include "nn_api.h"
#include "nn_internal.h"

namespace dhfwi {
using namespace nn;

namespace {

constexpr int CPAD = 8;          // first-layer input channels after padding
constexpr int MSE_BLOCKS = 256;
constexpr int RED_BLOCKS = 512;  // max blocks of the bias reductions

enum { K_C3 = 0, K_CT = 1, K_C1 = 2 };

struct LayerDesc {
    int kind, ci, co;
    long long off;   // offset of the weight in the flat parameter vector (bias follows)
    long long nw;    // number of weight values
};

int ilog_mult(int v, int levels) { return (v >> levels) << levels == v; }

}  // namespace

struct NetState {
    int base = 0, levels = 0;
    std::vector<LayerDesc> L;
    long long nparams = 0;
    bool have_weights = false;
    // Parameter state (device).
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *w16 = nullptr, *wt16 = nullptr, *w0pad = nullptr;
    __nv_bfloat16 *wc16 = nullptr;  // transposed convs' weights tap-major ([4][co][ci]) at their offsets
    float *g0pad = nullptr;
    // Workspace (device arena) sized for (wsN, wsH, wsW); the workspace of
    // the previous shape is kept as `prev` (training patches and the
    // full-image apply alternate every FWI iteration), so switching back
    // allocates nothing.
    int wsN = 0, wsH = 0, wsW = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    // Small buffers.
    double *mse_part = nullptr, *loss_acc = nullptr;
    float *red_part = nullptr;
    size_t red_part_floats = 0;
    float *wg_part = nullptr;
    size_t wg_part_floats = 0;
    float *fp_part = nullptr;    // split-k partials of the fprop GEMMs
    size_t fp_part_floats = 0;
    __nv_bfloat16 *ones = nullptr;  // {1, 0, ..., 0}: bias column of the weight-gradient GEMMs
    unsigned *mx = nullptr;
    unsigned *err = nullptr;     // set by a tensor-core GEMM whose bounded wait ran out
    float *scales = nullptr;  // [0..1] x scale, [2..3] y scale
    int *oz = nullptr, *ox = nullptr, *perm = nullptr;
    size_t oz_cap = 0, perm_cap = 0;
    int mute_rows = 0;           // from the last training configuration
    long long adam_t = 0;        // Adam steps of the current training call
    long long launches = 0;
    // Side stream of the backward pass: a layer's weight gradient runs there,
    // concurrently with its input gradient on the caller's stream.  ev_ready:
    // the output gradient g is written (caller -> side); ev_buf[b]: the last
    // weight gradient reading gradient buffer b (gbuf, gbuf2) is done (side ->
    // caller, before b is written again); ev_join: every weight gradient of
    // the pass is done.  DHFWI_NN_OVERLAP=0 keeps everything on one stream.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_buf[2] = {nullptr, nullptr}, ev_join = nullptr;
    bool use_side = false;  // this backward pass overlaps
    bool buf_rec[2] = {false, false};  // ev_buf[b] recorded in this backward pass

    // CUDA graphs of the fixed-shape passes (a training step's forward, loss
    // and backward; the forward of an apply): a pass seen once eagerly for a
    // (kind, batch, shape, workspace, GEMM switches) key is captured the
    // second time and replayed from then on as one graph launch.  Every
    // buffer a graph touches belongs to the network state (the workspace
    // arena, parameters, partials); drop_graphs() runs whenever one of them
    // is reallocated.  DHFWI_NN_GRAPH=0 keeps every pass eager.
    struct PassGraph {
        int kind = 0, n = 0, H = 0, W = 0;
        const char *arena = nullptr;
        std::string env;
        int seen = 0;
        bool failed = false;
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;  // kernel launches (and copies) one replay stands for
    };
    std::vector<PassGraph> graphs;
    cudaStream_t cap = nullptr;  // capture stream (the caller's may be the legacy default stream)

    // Workspace views (filled by layout()).
    struct Views {
        __nv_bfloat16 *xin, *a_inc0;
        std::vector<__nv_bfloat16 *> cat, pool, tmp, dec0, dec1;
        __nv_bfloat16 *bottom, *gbuf, *gbuf2;
        float *xf, *yf, *out, *dA, *dB;
        std::vector<float *> dskip;
    } V;
    struct Workspace {
        int wsN = 0, wsH = 0, wsW = 0;
        char *arena = nullptr;
        size_t arena_bytes = 0;
        Views V;
    } prev;
};

namespace {

void drop_graphs(NetState &N);

int layer_index_down(const NetState &N, int l, int j) { return 2 + 2 * (l - 1) + j; }
int layer_index_up(const NetState &N, int l, int j) { return 2 + 2 * N.levels + 3 * (l - 1) + j; }  // j: 0 t, 1 c0, 2 c1
int layer_index_out(const NetState &N) { return (int)N.L.size() - 1; }

void build_layers(NetState &N, int base, int levels) {
    N.base = base;
    N.levels = levels;
    N.L.clear();
    long long off = 0;
    auto add = [&](int kind, int ci, int co) {
        LayerDesc d;
        d.kind = kind;
        d.ci = ci;
        d.co = co;
        d.off = off;
        d.nw = kind == K_C3 ? 9LL * ci * co : kind == K_CT ? 4LL * ci * co : (long long)ci * co;
        off += d.nw + co;
        N.L.push_back(d);
    };
    auto C = [&](int l) { return base << l; };
    add(K_C3, 1, base);
    add(K_C3, base, base);
    for (int l = 1; l <= levels; l++) {
        add(K_C3, C(l - 1), C(l));
        add(K_C3, C(l), C(l));
    }
    for (int l = 1; l <= levels; l++) {
        const int hi = C(levels - l + 1), lo = C(levels - l);
        add(K_CT, hi, lo);
        add(K_C3, 2 * lo, lo);
        add(K_C3, lo, lo);
    }
    add(K_C1, base, 1);
    N.nparams = off;
}

// SplitMix64 (Steele, Lea, Flood 2014): state = seed + (counter+1) * golden.
unsigned long long splitmix(unsigned long long seed, unsigned long long counter) {
    unsigned long long z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void init_host(const NetState &N, unsigned long long seed, std::vector<float> &out) {
    out.assign((size_t)N.nparams, 0.f);
    for (const LayerDesc &d : N.L) {
        const int fan = d.kind == K_C3 ? 9 * d.ci : d.ci;
        const float bound = (float)(1.0 / std::sqrt((double)fan));
        const long long cnt = d.nw + d.co;
        for (long long i = 0; i < cnt; i++) {
            const unsigned long long k = (unsigned long long)(d.off + i);
            const float u = (float)(splitmix(seed, k) >> 40) * (1.0f / 16777216.0f);
            const float two_u = 2.0f * u;
            const float c = two_u - 1.0f;
            out[(size_t)(d.off + i)] = bound * c;
        }
    }
}

void permutation_host(int n, unsigned long long seed, int epoch, std::vector<int> &perm) {
    const unsigned long long key = seed ^ ((unsigned long long)(epoch + 1) * 0xD1B54A32D192ED03ull);
    perm.resize(n);
    for (int i = 0; i < n; i++) perm[i] = i;
    for (int i = n - 1; i > 0; i--) {
        const int j = (int)(splitmix(key, (unsigned long long)i) % (unsigned long long)(i + 1));
        std::swap(perm[i], perm[j]);
    }
}

std::vector<int> patch_origins(int n, int p, int stride) {
    std::vector<int> o;
    for (int v = 0; v + p <= n; v += stride) o.push_back(v);
    if (o.empty() || o.back() != n - p) o.push_back(n - p);
    return o;
}

int fail(dhfwi_ctx *ctx, int code, const char *msg) {
    ctx_set_error(ctx, msg);
    return code;
}

#define NCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            char b_[256];                                                      \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));  \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DHFWI_ERR_OOM : DHFWI_ERR_CUDA, b_); \
        }                                                                      \
    } while (0)

int dev_alloc(dhfwi_ctx *ctx, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char b[200];
        snprintf(b, sizeof b, "network allocation of %.3f GB failed: %s", bytes / 1e9, cudaGetErrorString(e));
        *p = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? DHFWI_ERR_OOM : DHFWI_ERR_CUDA, b);
    }
    return DHFWI_OK;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

void free_params(NetState &N) {
    dev_free(N.theta);
    dev_free(N.grad);
    dev_free(N.m);
    dev_free(N.v);
    dev_free(N.w16);
    dev_free(N.wt16);
    dev_free(N.wc16);
    dev_free(N.w0pad);
    dev_free(N.g0pad);
    N.theta = N.grad = N.m = N.v = nullptr;
    N.w16 = N.wt16 = N.wc16 = N.w0pad = nullptr;
    N.g0pad = nullptr;
}

int alloc_params(dhfwi_ctx *ctx, NetState &N) {
    free_params(N);
    const size_t n = (size_t)N.nparams;
    int rc;
    if ((rc = dev_alloc(ctx, (void **)&N.theta, 4 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.grad, 4 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.m, 4 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.v, 4 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.w16, 2 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.wt16, 2 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.wc16, 2 * n))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.w0pad, 2 * 9 * CPAD * (size_t)N.base))) return rc;
    if ((rc = dev_alloc(ctx, (void **)&N.g0pad, 4 * 9 * CPAD * (size_t)N.base))) return rc;
    return DHFWI_OK;
}

// bf16 shadow, transposed copies and the padded first layer from theta.
void refresh_weights(NetState &N, cudaStream_t s, bool shadow_from_theta) {
    if (shadow_from_theta) {
        launch_to_bf16(N.theta, N.nparams, N.w16, s);
        N.launches++;
    }
    // Transposed copies of the 3x3 (but the first) and transposed-conv
    // layers, in batches of up to TransposeJobs::MAX layers per launch.
    TransposeJobs jobs{};
    auto flush = [&]() {
        if (jobs.n == 0) return;
        launch_transpose_w_batch(N.w16, N.wt16, jobs, s);
        N.launches++;
        jobs.n = 0;
    };
    for (size_t i = 0; i < N.L.size(); i++) {
        const LayerDesc &d = N.L[i];
        const int taps = d.kind == K_C3 && i != 0 ? 9 : d.kind == K_CT ? 4 : 0;
        if (!taps) continue;
        jobs.off[jobs.n] = (long long)d.off;
        jobs.co[jobs.n] = d.co;
        jobs.taps[jobs.n] = taps;
        jobs.ci[jobs.n] = d.ci;
        if (++jobs.n == TransposeJobs::MAX) flush();
    }
    flush();
    // Tap-major copies of the transposed convs' weights (their forward GEMM's B^T).
    TransposeJobs ct{};
    for (size_t i = 0; i < N.L.size() && ct.n < TransposeJobs::MAX; i++) {
        const LayerDesc &d = N.L[i];
        if (d.kind != K_CT) continue;
        ct.off[ct.n] = (long long)d.off;
        ct.co[ct.n] = d.co;
        ct.taps[ct.n] = 4;
        ct.ci[ct.n] = d.ci;
        ct.n++;
    }
    launch_convt_tapmajor_batch(N.w16, N.wc16, ct, s);
    launch_pad_first_w(N.w16 + N.L[0].off, N.base, CPAD, N.w0pad, s);
    N.launches += 2;
}

// Swap the current workspace with the kept one.
void swap_workspace(NetState &N) {
    std::swap(N.wsN, N.prev.wsN);
    std::swap(N.wsH, N.prev.wsH);
    std::swap(N.wsW, N.prev.wsW);
    std::swap(N.arena, N.prev.arena);
    std::swap(N.arena_bytes, N.prev.arena_bytes);
    std::swap(N.V, N.prev.V);
}

// Activation / gradient workspace for batches of up to (n, H, W).
int layout(dhfwi_ctx *ctx, NetState &N, int n, int H, int W) {
    if (N.arena && N.wsN >= n && N.wsH == H && N.wsW == W) return DHFWI_OK;
    if (N.prev.arena && N.prev.wsN >= n && N.prev.wsH == H && N.prev.wsW == W) {
        swap_workspace(N);
        return DHFWI_OK;
    }
    // A new shape: the current workspace becomes the kept one.
    drop_graphs(N);
    if (N.prev.arena) cudaFree(N.prev.arena);
    N.prev = NetState::Workspace{};
    swap_workspace(N);
    const int Lv = N.levels;
    auto P = [&](int r) { return (size_t)n * (size_t)(H >> r) * (size_t)(W >> r); };
    auto C = [&](int r) { return (size_t)N.base << r; };
    size_t off = 0;
    std::vector<std::pair<void **, size_t>> plan;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    // Offsets first, pointers after allocation.
    std::vector<size_t> o_cat(Lv), o_pool(Lv + 1), o_tmp(Lv + 1), o_dec0(Lv), o_dec1(Lv), o_dskip(Lv);
    const size_t o_xin = take(2 * P(0) * CPAD);
    const size_t o_inc0 = take(2 * P(0) * C(0));
    size_t max_pc2 = 0;
    for (int r = 0; r < Lv; r++) {
        o_cat[r] = take(2 * P(r) * 2 * C(r));
        o_dec0[r] = take(2 * P(r) * C(r));
        o_dec1[r] = take(2 * P(r) * C(r));
        o_dskip[r] = take(4 * P(r) * C(r));
        max_pc2 = std::max(max_pc2, P(r) * 2 * C(r));
    }
    for (int r = 1; r <= Lv; r++) {
        o_pool[r] = take(2 * P(r) * C(r - 1));
        o_tmp[r] = take(2 * P(r) * C(r));
        max_pc2 = std::max(max_pc2, P(r) * 2 * C(r));
    }
    const size_t o_bottom = take(2 * P(Lv) * C(Lv));
    const size_t o_gbuf = take(2 * max_pc2);
    const size_t o_gbuf2 = take(2 * max_pc2);
    const size_t o_xf = take(4 * P(0));
    const size_t o_yf = take(4 * P(0));
    const size_t o_out = take(4 * P(0));
    const size_t o_dA = take(4 * max_pc2);
    const size_t o_dB = take(4 * max_pc2);
    if (N.arena) cudaFree(N.arena);
    N.arena = nullptr;
    int rc = dev_alloc(ctx, (void **)&N.arena, off);
    if (rc) return rc;
    N.arena_bytes = off;
    char *A = N.arena;
    auto bf = [&](size_t o) { return reinterpret_cast<__nv_bfloat16 *>(A + o); };
    auto fl = [&](size_t o) { return reinterpret_cast<float *>(A + o); };
    N.V.xin = bf(o_xin);
    N.V.a_inc0 = bf(o_inc0);
    N.V.cat.assign(Lv, nullptr);
    N.V.dec0.assign(Lv, nullptr);
    N.V.dec1.assign(Lv, nullptr);
    N.V.dskip.assign(Lv, nullptr);
    N.V.pool.assign(Lv + 1, nullptr);
    N.V.tmp.assign(Lv + 1, nullptr);
    for (int r = 0; r < Lv; r++) {
        N.V.cat[r] = bf(o_cat[r]);
        N.V.dec0[r] = bf(o_dec0[r]);
        N.V.dec1[r] = bf(o_dec1[r]);
        N.V.dskip[r] = fl(o_dskip[r]);
    }
    for (int r = 1; r <= Lv; r++) {
        N.V.pool[r] = bf(o_pool[r]);
        N.V.tmp[r] = bf(o_tmp[r]);
    }
    N.V.bottom = bf(o_bottom);
    N.V.gbuf = bf(o_gbuf);
    N.V.gbuf2 = bf(o_gbuf2);
    N.V.xf = fl(o_xf);
    N.V.yf = fl(o_yf);
    N.V.out = fl(o_out);
    N.V.dA = fl(o_dA);
    N.V.dB = fl(o_dB);
    N.wsN = n;
    N.wsH = H;
    N.wsW = W;
    // Weight-gradient partials: splits x M x N over every weight-gradient call.
    size_t need = 0;
    auto consider = [&](long long kpix, int M, int Nw) {
        const int Nn = Nw + 8;  // + bias column block
        need = std::max(need, (size_t)wgrad_splits(kpix, M, Nn) * M * Nn);
    };
    consider((long long)P(0), (int)C(0), 9 * CPAD);  // first layer (padded input)
    consider((long long)P(0), (int)C(0), 9 * (int)C(0));
    for (int l = 1; l <= Lv; l++) {
        consider((long long)P(l), (int)C(l), 9 * (int)C(l - 1));
        consider((long long)P(l), (int)C(l), 9 * (int)C(l));
    }
    for (int r = 0; r < Lv; r++) {
        consider((long long)P(r + 1), 4 * (int)C(r), (int)C(r + 1));  // transposed conv
        consider((long long)P(r), (int)C(r), 9 * 2 * (int)C(r));
        consider((long long)P(r), (int)C(r), 9 * (int)C(r));
    }
    if (N.wg_part_floats < need) {
        dev_free(N.wg_part);
        N.wg_part = nullptr;
        if ((rc = dev_alloc(ctx, (void **)&N.wg_part, 4 * need))) return rc;
        N.wg_part_floats = need;
    }
    // Split-k partials of the forward / input-gradient GEMMs: up to ~1216
    // tiles' worth of 128 x 64 outputs, and at least the deepest level's M x N x 8.
    {
        size_t fneed = (size_t)2 * 152 * 4 * 128 * 64;
        fneed = std::max(fneed, (size_t)8 * P(Lv) * 4 * C(Lv));
        if (N.fp_part_floats < fneed) {
            dev_free(N.fp_part);
            N.fp_part = nullptr;
            if ((rc = dev_alloc(ctx, (void **)&N.fp_part, 4 * fneed))) return rc;
            N.fp_part_floats = fneed;
        }
    }
    const size_t rneed = (size_t)RED_BLOCKS * (2 * C(Lv) + 2);
    if (N.red_part_floats < rneed) {
        dev_free(N.red_part);
        N.red_part = nullptr;
        if ((rc = dev_alloc(ctx, (void **)&N.red_part, 4 * rneed))) return rc;
        N.red_part_floats = rneed;
    }
    return DHFWI_OK;
}

// 3x3 conv forward with epilogue; src channel stride/offset, dst stride/offset.
void conv3_fwd(NetState &N, const LayerDesc &d, const __nv_bfloat16 *w, int nimg, int H, int W,
               const __nv_bfloat16 *src, int ss, int so, int C, void *dst, int ds, int dof, int epi, cudaStream_t s) {
    FpropArgs a{};
    a.src = src;
    a.src_stride = ss;
    a.src_off = so;
    a.Hs = H;
    a.Ws = W;
    a.C = C;
    a.ntaps = 9;
    a.scale = 1;
    for (int t = 0; t < 9; t++) {
        a.dh[t] = t / 3 - 1;
        a.dw[t] = t % 3 - 1;
    }
    a.Ho = H;
    a.Wo = W;
    a.M = nimg * H * W;
    a.N = d.co;
    a.bt = w;
    a.bias = N.theta + d.off + d.nw;
    a.slope = 0.2f;
    if (epi == EPI_F32 || epi == EPI_F32_ADD)
        a.dst_f32 = (float *)dst;
    else
        a.dst_bf16 = (__nv_bfloat16 *)dst;
    a.dst_stride = ds;
    a.dst_off = dof;
    a.part = N.fp_part;
    a.part_floats = (long long)N.fp_part_floats;
    a.err = N.err;
    launch_fprop(a, epi, s);
    N.launches += 2;
}

void forward(NetState &N, int n, int H, int W, cudaStream_t s) {
    const int Lv = N.levels;
    auto C = [&](int r) { return N.base << r; };
    NetState::Views &V = N.V;
    launch_input_pack(V.xf, (long long)n * H * W, CPAD, V.xin, s);
    N.launches++;
    // First layer: one real input channel, on CUDA cores (the GEMM would
    // spend 7 of its 8 padded channels on zeros).
    if (launch_first_conv(V.xin, CPAD, n, H, W, N.w16 + N.L[0].off, N.theta + N.L[0].off + N.L[0].nw, C(0), 0.2f,
                          V.a_inc0, C(0), s))
        N.launches++;
    else
        conv3_fwd(N, N.L[0], N.w0pad, n, H, W, V.xin, CPAD, 0, CPAD, V.a_inc0, C(0), 0, EPI_BF16_LEAKY, s);
    conv3_fwd(N, N.L[1], N.w16 + N.L[1].off, n, H, W, V.a_inc0, C(0), 0, C(0), V.cat[0], 2 * C(0), 0,
              EPI_BF16_LEAKY, s);
    for (int r = 1; r <= Lv; r++) {
        const int Hp = H >> (r - 1), Wp = W >> (r - 1), Hr = H >> r, Wr = W >> r;
        launch_avgpool_fwd(V.cat[r - 1], 2 * C(r - 1), 0, n, Hp, Wp, C(r - 1), V.pool[r], s);
        N.launches++;
        const LayerDesc &d0 = N.L[layer_index_down(N, r, 0)], &d1 = N.L[layer_index_down(N, r, 1)];
        conv3_fwd(N, d0, N.w16 + d0.off, n, Hr, Wr, V.pool[r], C(r - 1), 0, C(r - 1), V.tmp[r], C(r), 0,
                  EPI_BF16_LEAKY, s);
        if (r < Lv)
            conv3_fwd(N, d1, N.w16 + d1.off, n, Hr, Wr, V.tmp[r], C(r), 0, C(r), V.cat[r], 2 * C(r), 0,
                      EPI_BF16_LEAKY, s);
        else
            conv3_fwd(N, d1, N.w16 + d1.off, n, Hr, Wr, V.tmp[r], C(r), 0, C(r), V.bottom, C(r), 0,
                      EPI_BF16_LEAKY, s);
    }
    const __nv_bfloat16 *a = V.bottom;
    int as = C(Lv);
    for (int l = 1; l <= Lv; l++) {
        const int r = Lv - l;
        const int Hr = H >> r, Wr = W >> r;
        const LayerDesc &dt = N.L[layer_index_up(N, l, 0)];
        FpropArgs t{};
        t.src = a;
        t.src_stride = as;
        t.src_off = 0;
        t.Hs = H >> (r + 1);
        t.Ws = W >> (r + 1);
        t.C = C(r + 1);
        t.ntaps = 1;
        t.scale = 1;
        t.dh[0] = t.dw[0] = 0;
        t.Ho = H >> (r + 1);
        t.Wo = W >> (r + 1);
        t.M = n * t.Ho * t.Wo;
        t.N = 4 * C(r);
        t.bt = N.wc16 + dt.off;  // tap-major rows
        t.bias = N.theta + dt.off + dt.nw;
        t.dst_bf16 = V.cat[r];
        t.dst_stride = 2 * C(r);
        t.dst_off = C(r);
        t.part = N.fp_part;
        t.part_floats = (long long)N.fp_part_floats;
        t.err = N.err;
        launch_fprop(t, EPI_BF16_CONVT, s);
        N.launches++;
        const LayerDesc &d0 = N.L[layer_index_up(N, l, 1)], &d1 = N.L[layer_index_up(N, l, 2)];
        conv3_fwd(N, d0, N.w16 + d0.off, n, Hr, Wr, V.cat[r], 2 * C(r), 0, 2 * C(r), V.dec0[r], C(r), 0,
                  EPI_BF16_LEAKY, s);
        conv3_fwd(N, d1, N.w16 + d1.off, n, Hr, Wr, V.dec0[r], C(r), 0, C(r), V.dec1[r], C(r), 0,
                  EPI_BF16_LEAKY, s);
        a = V.dec1[r];
        as = C(r);
    }
    const LayerDesc &dout = N.L[layer_index_out(N)];
    launch_conv1x1_fwd(V.dec1[0], C(0), (long long)n * H * W, N.w16 + dout.off, N.theta + dout.off + dout.nw,
                       V.out, s);
    N.launches++;
}

bool overlap_on() {
    const char *e = getenv("DHFWI_NN_OVERLAP");
    return !(e && strcmp(e, "0") == 0);
}

// The stream the weight gradients run on (the side stream when overlapping).
cudaStream_t wgrad_stream(NetState &N, cudaStream_t s) { return N.use_side ? N.side : s; }

// Index of gradient buffer p (0 gbuf, 1 gbuf2, -1 neither).
int gbuf_index(const NetState &N, const void *p) {
    return p == (const void *)N.V.gbuf ? 0 : p == (const void *)N.V.gbuf2 ? 1 : -1;
}

// Before the caller's stream writes gradient buffer p: wait for the weight
// gradient that read it last.
void before_gbuf_write(NetState &N, const void *p, cudaStream_t s) {
    const int b = gbuf_index(N, p);
    // Only an event of this pass: the previous pass's weight gradients were
    // joined at its end (and a captured pass may wait on no outside event).
    if (N.use_side && b >= 0 && N.buf_rec[b]) cudaStreamWaitEvent(s, N.ev_buf[b], 0);
}

// A weight gradient reading g may start: the side stream waits for the
// caller's stream up to here.
void fork_wgrad(NetState &N, cudaStream_t s) {
    if (!N.use_side) return;
    cudaEventRecord(N.ev_ready, s);
    cudaStreamWaitEvent(N.side, N.ev_ready, 0);
}

// After the weight gradient that read g was launched on the side stream.
void after_wgrad(NetState &N, const void *g) {
    const int b = gbuf_index(N, g);
    if (N.use_side && b >= 0) {
        cudaEventRecord(N.ev_buf[b], N.side);
        N.buf_rec[b] = true;
    }
}

// Backward of one conv + LeakyReLU block: dA (float, dense [P][co]) is the
// gradient of its output a; x its (bf16) input.  Writes the weight and bias
// gradients and, when dx != nullptr, the input gradient (float [P][ci]).
// The layer's output gradient g (bf16) is either computed here from dA
// (f32) and the layer's activation a, or given as g_in (already computed by
// the previous block's fused epilogue).  The input gradient goes to dx (f32),
// or, when next_g is set, straight into the next block's g: times the
// LeakyReLU derivative of next_act, the input x's activation (the two give
// the same bits as storing dx and running the activation backward after).
struct FuseNext {
    const __nv_bfloat16 *act = nullptr;
    int stride = 0, off = 0;
    __nv_bfloat16 *g = nullptr;
};

void block_bwd(NetState &N, int li, const float *dA, const __nv_bfloat16 *a, int as, int ao, const __nv_bfloat16 *x,
               int xs, int xo, int ci, int nimg, int H, int W, float *dx, cudaStream_t s,
               const __nv_bfloat16 *g_in = nullptr, const FuseNext &next = FuseNext()) {
    const LayerDesc &d = N.L[li];
    const long long P = (long long)nimg * H * W;
    const __nv_bfloat16 *g = g_in;
    if (!g) {
        before_gbuf_write(N, N.V.gbuf, s);
        launch_leaky_bwd(dA, a, as, ao, P, d.co, 0.2f, N.V.gbuf, s);
        g = N.V.gbuf;
        N.launches++;
    }
    fork_wgrad(N, s);
    const cudaStream_t ws = wgrad_stream(N, s);
    WgradArgs w{};
    w.mode = WG_CONV;
    w.g = g;
    w.g_stride = d.co;
    w.x = x;
    w.x_stride = xs;
    w.x_off = xo;
    w.nimg = nimg;
    w.H = H;
    w.W = W;
    w.ci = ci;
    w.M = d.co;
    w.nw = 9 * ci;
    w.N = w.nw + 8;
    w.ones = N.ones;
    w.part = N.wg_part;
    w.err = N.err;
    const int sp = wgrad_splits(P, w.M, w.N);
    // The first layer (one real input channel): a pixel reduction on CUDA cores.
    const int first = li == 0 ? launch_first_wgrad(g, d.co, x, xs, nimg, H, W, N.wg_part, (long long)N.wg_part_floats,
                                                   N.grad + d.off, N.grad + d.off + d.nw, ws)
                              : 0;
    if (first) {
        N.launches += first;
    } else {
        float *dw = li == 0 ? N.g0pad : N.grad + d.off;
        N.launches += launch_wgrad(w, sp, dw, N.grad + d.off + d.nw, ws);
        if (li == 0) {
            launch_unpad_first_grad(N.g0pad, d.co, CPAD, N.grad + d.off, ws);
            N.launches++;
        }
    }
    after_wgrad(N, g);
    if (dx || next.g) {
        FpropArgs a{};
        a.src = g;
        a.src_stride = d.co;
        a.src_off = 0;
        a.Hs = H;
        a.Ws = W;
        a.C = d.co;
        a.ntaps = 9;
        a.scale = 1;
        for (int t = 0; t < 9; t++) {
            a.dh[t] = 1 - t / 3;
            a.dw[t] = 1 - t % 3;
        }
        a.Ho = H;
        a.Wo = W;
        a.M = (int)P;
        a.N = ci;
        a.bt = N.wt16 + d.off;
        a.dst_stride = ci;
        a.dst_off = 0;
        a.part = N.fp_part;
        a.part_floats = (long long)N.fp_part_floats;
        a.err = N.err;
        if (next.g) {
            before_gbuf_write(N, next.g, s);
            a.dst_bf16 = next.g;
            a.act = next.act;
            a.act_stride = next.stride;
            a.act_off = next.off;
            a.slope = 0.2f;
            launch_fprop(a, EPI_BF16_LEAKYBWD, s);
        } else {
            a.dst_f32 = dx;
            launch_fprop(a, EPI_F32, s);
        }
        N.launches += 2;
    }
}

// The side stream and its events (created once, on the context's device).
bool ensure_side(NetState &N) {
    if (N.side) return true;
    if (cudaStreamCreateWithFlags(&N.side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        N.side = nullptr;
        return false;
    }
    cudaEvent_t *evs[] = {&N.ev_ready, &N.ev_buf[0], &N.ev_buf[1], &N.ev_join};
    for (cudaEvent_t *e : evs)
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    return true;
}

void backward_impl(NetState &N, int n, int H, int W, cudaStream_t s);

void backward(NetState &N, int n, int H, int W, cudaStream_t s) {
    N.use_side = overlap_on() && ensure_side(N);
    N.buf_rec[0] = N.buf_rec[1] = false;
    backward_impl(N, n, H, W, s);
    if (N.use_side) {  // every weight gradient is done before the caller's stream goes on
        cudaEventRecord(N.ev_join, N.side);
        cudaStreamWaitEvent(s, N.ev_join, 0);
    }
    N.use_side = false;
}

void backward_impl(NetState &N, int n, int H, int W, cudaStream_t s) {
    const int Lv = N.levels;
    auto C = [&](int r) { return N.base << r; };
    NetState::Views &V = N.V;
    const long long P0 = (long long)n * H * W;
    // Output layer: g_out (bf16 [P0]) was written by the loss kernel into gbuf.
    const LayerDesc &dout = N.L[layer_index_out(N)];
    // Keep g_out apart from gbuf, which the blocks reuse: stage it in dB.
    __nv_bfloat16 *gout = reinterpret_cast<__nv_bfloat16 *>(V.dB);
    // Its input gradient goes, with dec1[0]'s activation backward, straight
    // into the next block's output gradient (gbuf).
    before_gbuf_write(N, V.gbuf, s);
    launch_conv1x1_bwd_leaky(gout, V.dec1[0], P0, C(0), N.w16 + dout.off, 0.2f, V.gbuf, N.red_part, RED_BLOCKS,
                             N.grad + dout.off, s);
    N.launches += 2;
    float *dA = V.dA, *dB = V.dB;
    for (int l = Lv; l >= 1; l--) {
        const int r = Lv - l;
        const int Hr = H >> r, Wr = W >> r;
        const long long Pr = (long long)n * Hr * Wr;
        // up_l.1: output dec1, input dec0; its input gradient goes straight into
        // up_l.0's output gradient (dec0's activation backward fused).
        FuseNext fu;
        fu.act = V.dec0[r];
        fu.stride = C(r);
        fu.g = V.gbuf2;
        const __nv_bfloat16 *g_top = l == Lv ? V.gbuf : nullptr;  // from the output layer's backward
        block_bwd(N, layer_index_up(N, l, 2), g_top ? nullptr : dA, V.dec1[r], C(r), 0, V.dec0[r], C(r), 0, C(r), n,
                  Hr, Wr, nullptr, s, g_top, fu);
        // up_l.0: output dec0, input cat (2C).
        block_bwd(N, layer_index_up(N, l, 1), nullptr, nullptr, 0, 0, V.cat[r], 2 * C(r), 0, 2 * C(r), n, Hr, Wr, dA,
                  s, V.gbuf2);
        // dA = d(cat) [Pr][2C]: skip half kept, up half to bf16 in
        // space-to-depth layout on the coarse grid (the transposed conv's
        // gradients are then one-tap GEMMs).
        before_gbuf_write(N, V.gbuf, s);
        const bool s2d = launch_split_cat(dA, n, Hr, Wr, C(r), V.dskip[r], V.gbuf, s);
        if (s2d) {
            N.launches++;
        } else {
            cudaMemsetAsync(V.dskip[r], 0, sizeof(float) * Pr * C(r), s);
            launch_add_slice(dA, 2 * C(r), 0, Pr, C(r), V.dskip[r], s);
            launch_f32_to_bf16_slice(dA, 2 * C(r), C(r), Pr, C(r), V.gbuf, s);
            N.launches += 2;
        }
        // Transposed conv: input is the level-(r+1) activation.
        const int li = layer_index_up(N, l, 0);
        const LayerDesc &dt = N.L[li];
        const __nv_bfloat16 *xin = l == 1 ? V.bottom : V.dec1[r + 1];
        const int Hc = H >> (r + 1), Wc = W >> (r + 1);
        WgradArgs w{};
        w.mode = WG_CONVT;
        w.g = V.gbuf;
        w.g_stride = s2d ? 4 * C(r) : C(r);
        w.g_s2d = s2d;
        w.x = xin;
        w.x_stride = C(r + 1);
        w.x_off = 0;
        w.nimg = n;
        w.H = Hc;
        w.W = Wc;
        w.co = C(r);
        w.ci = C(r + 1);
        w.M = 4 * C(r);
        w.nw = C(r + 1);
        w.N = w.nw + 8;
        w.ones = N.ones;
        w.part = N.wg_part;
        w.err = N.err;
        const int sp = wgrad_splits((long long)n * Hc * Wc, w.M, w.N);
        fork_wgrad(N, s);
        launch_wgrad(w, sp, N.grad + dt.off, N.grad + dt.off + dt.nw, wgrad_stream(N, s));
        after_wgrad(N, V.gbuf);
        FpropArgs a{};
        a.src = V.gbuf;
        a.src_off = 0;
        if (s2d) {  // input gradient: the one-tap GEMM over the 4 C(r) space-to-depth channels
            a.src_stride = 4 * C(r);
            a.Hs = Hc;
            a.Ws = Wc;
            a.C = 4 * C(r);
            a.ntaps = 1;
            a.scale = 1;
            a.dh[0] = a.dw[0] = 0;
        } else {
            a.src_stride = C(r);
            a.Hs = Hr;
            a.Ws = Wr;
            a.C = C(r);
            a.ntaps = 4;
            a.scale = 2;
            for (int t = 0; t < 4; t++) {
                a.dh[t] = t >> 1;
                a.dw[t] = t & 1;
            }
        }
        a.Ho = Hc;
        a.Wo = Wc;
        a.M = n * Hc * Wc;
        a.N = C(r + 1);
        a.bt = N.wt16 + dt.off;
        a.dst_f32 = dB;
        a.dst_stride = C(r + 1);
        a.dst_off = 0;
        a.part = N.fp_part;
        a.part_floats = (long long)N.fp_part_floats;
        a.err = N.err;
        launch_fprop(a, EPI_F32, s);
        N.launches += 5;
        std::swap(dA, dB);
    }
    // dA: gradient of the bottom activation.  gin: the next block's output
    // gradient (bf16, gbuf) when the pool's backward already produced it.
    const __nv_bfloat16 *gin = nullptr;
    for (int r = Lv; r >= 1; r--) {
        const int Hr = H >> r, Wr = W >> r;
        const long long Pr = (long long)n * Hr * Wr;
        if (r < Lv && !gin) {
            launch_add_slice(V.dskip[r], C(r), 0, Pr, C(r), dA, s);
            N.launches++;
        }
        const __nv_bfloat16 *ar = r < Lv ? V.cat[r] : V.bottom;
        const int ars = r < Lv ? 2 * C(r) : C(r);
        FuseNext fd;
        fd.act = V.tmp[r];
        fd.stride = C(r);
        fd.g = V.gbuf2;
        block_bwd(N, layer_index_down(N, r, 1), gin ? nullptr : dA, ar, ars, 0, V.tmp[r], C(r), 0, C(r), n, Hr, Wr,
                  nullptr, s, gin, fd);
        block_bwd(N, layer_index_down(N, r, 0), nullptr, nullptr, 0, 0, V.pool[r], C(r - 1), 0, C(r - 1), n, Hr, Wr,
                  dA, s, V.gbuf2);
        // Level r-1's output gradient: the pool's backward of dA plus the skip
        // gradient, times the LeakyReLU derivative of that output (cat[r-1]'s
        // first half), straight to bf16 for the next block.
        before_gbuf_write(N, V.gbuf, s);
        if (launch_avgpool_bwd_leaky(dA, n, H >> (r - 1), W >> (r - 1), C(r - 1), V.dskip[r - 1], V.cat[r - 1],
                                     2 * C(r - 1), 0, 0.2f, V.gbuf, s)) {
            gin = V.gbuf;
        } else {
            launch_avgpool_bwd(dA, n, H >> (r - 1), W >> (r - 1), C(r - 1), dB, 0, s);
            std::swap(dA, dB);
            gin = nullptr;
        }
        N.launches++;
    }
    if (!gin) {
        launch_add_slice(V.dskip[0], C(0), 0, P0, C(0), dA, s);
        N.launches++;
    }
    FuseNext f0;
    f0.act = V.a_inc0;
    f0.stride = C(0);
    f0.g = V.gbuf2;
    block_bwd(N, 1, gin ? nullptr : dA, V.cat[0], 2 * C(0), 0, V.a_inc0, C(0), 0, C(0), n, H, W, nullptr, s, gin, f0);
    block_bwd(N, 0, nullptr, nullptr, 0, 0, V.xin, CPAD, 0, CPAD, n, H, W, nullptr, s, V.gbuf2);
}

// Loss of the current batch: MSE against yf; writes g_out (bf16) to the
// staging slot read by backward().
void loss(NetState &N, int n, int H, int W, cudaStream_t s) {
    launch_mse(N.V.out, N.V.yf, (long long)n * H * W, reinterpret_cast<__nv_bfloat16 *>(N.V.dB), N.mse_part,
               MSE_BLOCKS, s);
    N.launches++;
}

void drop_graphs(NetState &N) {
    for (NetState::PassGraph &g : N.graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    N.graphs.clear();
}

bool graphs_on() {
    const char *e = getenv("DHFWI_NN_GRAPH");
    return !(e && strcmp(e, "0") == 0);
}

// The switches that change which kernels a pass launches.
std::string gemm_switches() {
    static const char *names[] = {"DHFWI_NN_GEMM", "DHFWI_NN_WGRAD", "DHFWI_NN_CONV",   "DHFWI_NN_PATCH",
                                  "DHFWI_NN_HALO", "DHFWI_NN_CONVT", "DHFWI_NN_OVERLAP", "DHFWI_NN_WGRAD_NB", "DHFWI_NN_CONV_BN"};
    std::string k;
    for (const char *n : names) {
        const char *e = getenv(n);
        k += e ? e : "-";
        k += '|';
    }
    return k;
}

enum { PASS_TRAIN = 0, PASS_FORWARD = 1 };

void pass_eager(NetState &N, int kind, int n, int H, int W, cudaStream_t s) {
    forward(N, n, H, W, s);
    if (kind == PASS_TRAIN) {
        loss(N, n, H, W, s);
        backward(N, n, H, W, s);
    }
}

// One pass of the given kind on the current workspace (see PassGraph).
// Returns a CUDA error of the capture or the launch (cudaSuccess after an
// eager run; a capture that fails marks its key eager for good).
cudaError_t run_pass(NetState &N, int kind, int n, int H, int W, cudaStream_t s) {
    if (!graphs_on()) {
        pass_eager(N, kind, n, H, W, s);
        return cudaSuccess;
    }
    const std::string env = gemm_switches();
    NetState::PassGraph *g = nullptr;
    for (NetState::PassGraph &e : N.graphs)
        if (e.kind == kind && e.n == n && e.H == H && e.W == W && e.arena == N.arena && e.env == env) g = &e;
    if (!g) {
        if (N.graphs.size() >= 16) drop_graphs(N);
        N.graphs.emplace_back();
        g = &N.graphs.back();
        g->kind = kind;
        g->n = n;
        g->H = H;
        g->W = W;
        g->arena = N.arena;
        g->env = env;
    }
    if (g->failed || g->seen++ == 0) {  // first sighting: eager (lazy attributes, streams and events settle)
        pass_eager(N, kind, n, H, W, s);
        return cudaSuccess;
    }
    if (!g->exec) {
        if (!N.cap && cudaStreamCreateWithFlags(&N.cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            N.cap = nullptr;
            g->failed = true;
            pass_eager(N, kind, n, H, W, s);
            return cudaSuccess;
        }
        const long long l0 = N.launches;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(N.cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            pass_eager(N, kind, n, H, W, N.cap);
            e = cudaStreamEndCapture(N.cap, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        g->launches = N.launches - l0;
        N.launches = l0;
        if (e != cudaSuccess) {  // nothing of the captured pass ran: run it eagerly
            cudaGetLastError();
            g->exec = nullptr;
            g->failed = true;
            pass_eager(N, kind, n, H, W, s);
            return cudaSuccess;
        }
    }
    N.launches += g->launches;
    return cudaGraphLaunch(g->exec, s);
}

int ensure_small(dhfwi_ctx *ctx, NetState &N) {
    int rc;
    if (!N.mse_part && (rc = dev_alloc(ctx, (void **)&N.mse_part, sizeof(double) * MSE_BLOCKS))) return rc;
    if (!N.loss_acc && (rc = dev_alloc(ctx, (void **)&N.loss_acc, sizeof(double) * 4096))) return rc;
    if (!N.mx && (rc = dev_alloc(ctx, (void **)&N.mx, 16))) return rc;
    if (!N.err) {
        if ((rc = dev_alloc(ctx, (void **)&N.err, 16))) return rc;
        NCK(cudaMemset(N.err, 0, 16));
    }
    if (!N.scales && (rc = dev_alloc(ctx, (void **)&N.scales, 4 * sizeof(float)))) return rc;
    if (!N.ones) {
        if ((rc = dev_alloc(ctx, (void **)&N.ones, 16))) return rc;
        __nv_bfloat16 h[8];
        for (int i = 0; i < 8; i++) h[i] = __float2bfloat16_rn(i == 0 ? 1.0f : 0.0f);
        NCK(cudaMemcpy(N.ones, h, sizeof h, cudaMemcpyHostToDevice));
    }
    return DHFWI_OK;
}

int ensure_net(dhfwi_ctx *ctx, int base, int levels) {
    NetState *&net = ctx_net(ctx);
    if (base < 8 || base > 256 || base % 8 != 0 || levels < 1 || levels > 6)
        return fail(ctx, DHFWI_ERR_ARG,
                    "network needs base_channels a multiple of 8 in [8, 256] and 1 <= levels <= 6");
    if (!net) net = new NetState();
    if (net->base != base || net->levels != levels || !net->theta) {
        drop_graphs(*net);
        build_layers(*net, base, levels);
        int rc = alloc_params(ctx, *net);
        if (rc) return rc;
        net->have_weights = false;
        if (net->arena) cudaFree(net->arena);
        net->arena = nullptr;
        net->wsN = net->wsH = net->wsW = 0;
        if (net->prev.arena) cudaFree(net->prev.arena);
        net->prev = NetState::Workspace{};
    }
    return ensure_small(ctx, *net);
}

// DHFWI_ERR_TIMEOUT if a tensor-core GEMM of this or an earlier call ran out
// its bounded wait (the word is cleared); synchronises the stream.
int check_gemm_err(dhfwi_ctx *ctx, NetState &N, cudaStream_t s) {
    if (!N.err) return DHFWI_OK;
    unsigned e = 0;
    NCK(cudaMemcpyAsync(&e, N.err, sizeof e, cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    if (!e) return DHFWI_OK;
    NCK(cudaMemsetAsync(N.err, 0, sizeof e, s));
    return fail(ctx, DHFWI_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting for its MMAs");
}

int upload_params(dhfwi_ctx *ctx, NetState &N, const float *host, cudaStream_t s) {
    NCK(cudaMemcpyAsync(N.theta, host, sizeof(float) * N.nparams, cudaMemcpyHostToDevice, s));
    NCK(cudaStreamSynchronize(s));
    refresh_weights(N, s, true);
    N.have_weights = true;
    return DHFWI_OK;
}

}  // namespace

void net_destroy(NetState *net) {
    if (!net) return;
    drop_graphs(*net);
    if (net->cap) cudaStreamDestroy(net->cap);
    if (net->side) {
        cudaStreamSynchronize(net->side);
        cudaStreamDestroy(net->side);
    }
    cudaEvent_t evs[] = {net->ev_ready, net->ev_buf[0], net->ev_buf[1], net->ev_join};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    free_params(*net);
    void *ps[] = {net->arena, net->prev.arena, net->mse_part, net->loss_acc, net->red_part, net->wg_part, net->fp_part, net->ones,
                  net->mx, net->err, net->scales, net->oz, net->ox, net->perm};
    for (void *p : ps) dev_free(p);
    delete net;
}

}  // namespace dhfwi

using namespace dhfwi;

extern "C" {

int dhfwi_net_init(dhfwi_ctx *ctx, int base_channels, int levels, unsigned long long seed) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    cudaSetDevice(ctx_device(ctx));
    int rc = ensure_net(ctx, base_channels, levels);
    if (rc) return rc;
    NetState &N = *ctx_net(ctx);
    std::vector<float> h;
    init_host(N, seed, h);
    return upload_params(ctx, N, h.data(), 0);
}

long long dhfwi_net_size(const dhfwi_ctx *ctx) {
    if (!ctx) return -1;
    NetState *net = ctx_net(const_cast<dhfwi_ctx *>(ctx));
    return net ? net->nparams : 0;
}

int dhfwi_net_get(dhfwi_ctx *ctx, float *host, size_t n) {
    if (!ctx || !host) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    NetState *net = ctx_net(ctx);
    if (!net || !net->have_weights) return fail(ctx, DHFWI_ERR_STATE, "the network has no weights yet");
    if (n != (size_t)net->nparams) return fail(ctx, DHFWI_ERR_ARG, "n must equal dhfwi_net_size()");
    cudaSetDevice(ctx_device(ctx));
    NCK(cudaMemcpy(host, net->theta, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return DHFWI_OK;
}

int dhfwi_net_set(dhfwi_ctx *ctx, const float *host, size_t n) {
    if (!ctx || !host) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    NetState *net = ctx_net(ctx);
    if (!net) return fail(ctx, DHFWI_ERR_STATE, "call dhfwi_net_init first to fix the architecture");
    if (n != (size_t)net->nparams) return fail(ctx, DHFWI_ERR_ARG, "n must equal dhfwi_net_size()");
    cudaSetDevice(ctx_device(ctx));
    return upload_params(ctx, *net, host, 0);
}

int deblur_forward(dhfwi_ctx *ctx, const float *x_dev, int n, int h, int w, float *out_dev, void *stream) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    NetState *net = ctx_net(ctx);
    if (!net || !net->have_weights) return fail(ctx, DHFWI_ERR_STATE, "the network has no weights yet");
    if (!x_dev || !out_dev || n < 1 || h < 1 || w < 1) return fail(ctx, DHFWI_ERR_ARG, "bad batch arguments");
    if (!ilog_mult(h, net->levels) || !ilog_mult(w, net->levels))
        return fail(ctx, DHFWI_ERR_ARG, "h and w must be multiples of 2^levels");
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    net->launches = 0;
    int rc = layout(ctx, *net, n, h, w);
    if (rc) return rc;
    const size_t P = (size_t)n * h * w;
    NCK(cudaMemcpyAsync(net->V.xf, x_dev, 4 * P, cudaMemcpyDeviceToDevice, s));
    NCK(run_pass(*net, PASS_FORWARD, n, h, w, s));
    NCK(cudaMemcpyAsync(out_dev, net->V.out, 4 * P, cudaMemcpyDeviceToDevice, s));
    NCK(cudaGetLastError());
    ctx_count_launches(ctx, net->launches);
    return DHFWI_OK;
}

int deblur_grad(dhfwi_ctx *ctx, const float *x_dev, const float *y_dev, int n, int h, int w, float *grad_dev,
                double *loss_out, void *stream) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    NetState *net = ctx_net(ctx);
    if (!net || !net->have_weights) return fail(ctx, DHFWI_ERR_STATE, "the network has no weights yet");
    if (!x_dev || !y_dev || !grad_dev || n < 1 || h < 1 || w < 1) return fail(ctx, DHFWI_ERR_ARG, "bad arguments");
    if ((long long)n * h * w >= (1LL << 31)) return fail(ctx, DHFWI_ERR_ARG, "n * h * w must be below 2^31");
    if (!ilog_mult(h, net->levels) || !ilog_mult(w, net->levels))
        return fail(ctx, DHFWI_ERR_ARG, "h and w must be multiples of 2^levels");
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    net->launches = 0;
    int rc = layout(ctx, *net, n, h, w);
    if (rc) return rc;
    const size_t P = (size_t)n * h * w;
    NCK(cudaMemcpyAsync(net->V.xf, x_dev, 4 * P, cudaMemcpyDeviceToDevice, s));
    NCK(cudaMemcpyAsync(net->V.yf, y_dev, 4 * P, cudaMemcpyDeviceToDevice, s));
    NCK(run_pass(*net, PASS_TRAIN, n, h, w, s));
    NCK(cudaMemcpyAsync(grad_dev, net->grad, 4 * (size_t)net->nparams, cudaMemcpyDeviceToDevice, s));
    if (loss_out) {
        double part[MSE_BLOCKS];
        NCK(cudaMemcpyAsync(part, net->mse_part, sizeof part, cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        double sum = 0.0;
        for (int i = 0; i < MSE_BLOCKS; i++) sum += part[i];
        *loss_out = sum / (double)P;
    }
    NCK(cudaGetLastError());
    ctx_count_launches(ctx, net->launches);
    return DHFWI_OK;
}

int deblur_train(dhfwi_ctx *ctx, const float *x_dev, const float *y_dev, int nz, int nx, const dhfwi_train_cfg *cfg,
                 int warm_start, float *loss_hist, void *stream) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    if (!cfg || !x_dev || !y_dev) return fail(ctx, DHFWI_ERR_ARG, "NULL argument");
    // patch == 0: full-image training (one sample: the whole image padded to
    // a multiple of 2^levels; batch and stride are not used).
    const bool full = cfg->patch == 0;
    if (cfg->patch < 0 || (!full && (cfg->stride < 1 || cfg->batch < 1)) || cfg->epochs < 1 || !(cfg->lr > 0.f) ||
        cfg->epochs > 4096 || nz < 1 || nx < 1)
        return fail(ctx, DHFWI_ERR_ARG, "bad training configuration");
    if (!full && (nz < cfg->patch || nx < cfg->patch)) return fail(ctx, DHFWI_ERR_ARG, "image smaller than the patch");
    if (!full && (long long)cfg->batch * cfg->patch * cfg->patch >= (1LL << 31))
        return fail(ctx, DHFWI_ERR_ARG, "batch * patch^2 must be below 2^31");
    if (full && ((long long)nz + 64) * ((long long)nx + 64) >= (1LL << 31))
        return fail(ctx, DHFWI_ERR_ARG, "image too large for full-image training");
    if (cfg->mute_rows < 0 || cfg->mute_rows >= nz) return fail(ctx, DHFWI_ERR_ARG, "mute_rows must be in [0, nz)");
    if (!(cfg->warmup_frac >= 0.f) || cfg->warmup_frac > 1.f)
        return fail(ctx, DHFWI_ERR_ARG, "warmup_frac must be in [0, 1]");
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_net(ctx, cfg->base_channels, cfg->levels);
    if (rc) return rc;
    NetState &N = *ctx_net(ctx);
    if (!full && !ilog_mult(cfg->patch, N.levels))
        return fail(ctx, DHFWI_ERR_ARG, "patch must be a multiple of 2^levels");
    N.launches = 0;
    if (!warm_start || !N.have_weights) {
        std::vector<float> h;
        init_host(N, cfg->seed, h);
        if ((rc = upload_params(ctx, N, h.data(), s))) return rc;
    }
    const int mult = 1 << N.levels;
    const int Hp = (nz + mult - 1) / mult * mult, Wp = (nx + mult - 1) / mult * mult;
    const int p = full ? 0 : cfg->patch;
    const int sh = full ? Hp : p, sw = full ? Wp : p;  // sample size
    const std::vector<int> oz = full ? std::vector<int>{0} : patch_origins(nz, p, cfg->stride),
                           ox = full ? std::vector<int>{0} : patch_origins(nx, p, cfg->stride);
    const int npatch = (int)(oz.size() * ox.size());
    std::vector<int> hoz(npatch), hox(npatch);
    for (size_t a = 0; a < oz.size(); a++)
        for (size_t b = 0; b < ox.size(); b++) {
            hoz[a * ox.size() + b] = oz[a];
            hox[a * ox.size() + b] = ox[b];
        }
    const int B = full ? 1 : std::min(cfg->batch, npatch);
    if ((rc = layout(ctx, N, B, sh, sw))) return rc;
    if (N.oz_cap < (size_t)npatch) {
        dev_free(N.oz);
        dev_free(N.ox);
        N.oz = N.ox = nullptr;
        if ((rc = dev_alloc(ctx, (void **)&N.oz, 4 * (size_t)npatch))) return rc;
        if ((rc = dev_alloc(ctx, (void **)&N.ox, 4 * (size_t)npatch))) return rc;
        N.oz_cap = npatch;
    }
    if (N.perm_cap < (size_t)npatch * cfg->epochs) {
        dev_free(N.perm);
        N.perm = nullptr;
        if ((rc = dev_alloc(ctx, (void **)&N.perm, 4 * (size_t)npatch * cfg->epochs))) return rc;
        N.perm_cap = (size_t)npatch * cfg->epochs;
    }
    std::vector<int> perms((size_t)npatch * cfg->epochs), one;
    for (int e = 0; e < cfg->epochs; e++) {
        permutation_host(npatch, cfg->seed, e, one);
        std::copy(one.begin(), one.end(), perms.begin() + (size_t)e * npatch);
    }
    NCK(cudaMemcpyAsync(N.oz, hoz.data(), 4 * (size_t)npatch, cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(N.ox, hox.data(), 4 * (size_t)npatch, cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(N.perm, perms.data(), 4 * perms.size(), cudaMemcpyHostToDevice, s));
    // Normalisation by max |.| of each image below the muted rows (Section
    // 2.3.1 pair: x = delta m_1, y = g).
    N.mute_rows = cfg->mute_rows;
    const long long moff = (long long)N.mute_rows * nx;
    launch_absmax(x_dev + moff, (long long)nz * nx - moff, N.mx, N.scales, s);
    launch_absmax(y_dev + moff, (long long)nz * nx - moff, N.mx + 1, N.scales + 2, s);
    N.launches += 6;
    // Fresh Adam moments for every training call; the learning rate ramps up
    // linearly over the first warmup steps so that the sign-like first
    // steps of fresh moments stay small.
    NCK(cudaMemsetAsync(N.m, 0, sizeof(float) * N.nparams, s));
    NCK(cudaMemsetAsync(N.v, 0, sizeof(float) * N.nparams, s));
    N.adam_t = 0;
    NCK(cudaMemsetAsync(N.loss_acc, 0, sizeof(double) * cfg->epochs, s));
    const int nb = (npatch + B - 1) / B;
    const long long T = (long long)cfg->epochs * nb;
    const long long warm_n = (long long)std::ceil((double)cfg->warmup_frac * (double)T);
    long long t = 0;
    if (full) {  // the one sample, normalised and padded once
        launch_pad_image(x_dev, nz, nx, Hp, Wp, N.scales, N.mute_rows, N.V.xf, s);
        launch_pad_image(y_dev, nz, nx, Hp, Wp, N.scales + 2, N.mute_rows, N.V.yf, s);
        N.launches += 2;
    }
    for (int e = 0; e < cfg->epochs; e++) {
        for (int b = 0; b < nb; b++) {
            const int cnt = std::min(B, npatch - b * B);
            if (!full) {
                const int *sel = N.perm + (size_t)e * npatch + (size_t)b * B;
                launch_gather_patches(x_dev, nx, N.oz, N.ox, sel, cnt, p, N.scales, N.mute_rows, N.V.xf, s);
                launch_gather_patches(y_dev, nx, N.oz, N.ox, sel, cnt, p, N.scales + 2, N.mute_rows, N.V.yf, s);
                N.launches += 2;
            }
            NCK(run_pass(N, PASS_TRAIN, cnt, sh, sw, s));  // forward, loss, backward
            launch_loss_accum(N.mse_part, MSE_BLOCKS, (double)cnt / ((double)cnt * sh * sw), N.loss_acc + e, s);
            double lr = 0.5 * cfg->lr * (1.0 + std::cos(M_PI * (double)t / (double)T));
            if (warm_n > 0 && t < warm_n) lr *= (double)(t + 1) / (double)warm_n;
            N.adam_t++;
            launch_adam(N.theta, N.grad, N.m, N.v, N.nparams, (float)lr, cfg->beta1, cfg->beta2, cfg->eps,
                        (int)N.adam_t, N.w16, s);
            refresh_weights(N, s, false);
            N.launches += 2;
            t++;
        }
        NCK(cudaGetLastError());
    }
    N.have_weights = true;
    if (loss_hist) {
        std::vector<double> acc(cfg->epochs);
        NCK(cudaMemcpyAsync(acc.data(), N.loss_acc, sizeof(double) * cfg->epochs, cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        // loss_acc[e] = sum_b cnt_b * mean_b(r^2); per-epoch mean over patches.
        for (int e = 0; e < cfg->epochs; e++) loss_hist[e] = (float)(acc[e] / (double)npatch);
        if ((rc = check_gemm_err(ctx, N, s))) return rc;
    }
    ctx_count_launches(ctx, N.launches);
    return DHFWI_OK;
}

int deblur_layer(dhfwi_ctx *ctx, int kind, int op, int n, int H, int W, int ci, int co, const float *x_dev,
                 const float *w_dev, const float *b_dev, const float *gy_dev, float *out_dev, void *stream) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    if (kind != DHFWI_LAYER_CONV3 && kind != DHFWI_LAYER_CONVT && kind != DHFWI_LAYER_FIRST)
        return fail(ctx, DHFWI_ERR_ARG, "bad layer kind");
    if (op != DHFWI_LAYER_FWD && op != DHFWI_LAYER_DGRAD && op != DHFWI_LAYER_WGRAD)
        return fail(ctx, DHFWI_ERR_ARG, "bad layer operation");
    const bool first = kind == DHFWI_LAYER_FIRST;
    if (first && (ci != 1 || op == DHFWI_LAYER_DGRAD))
        return fail(ctx, DHFWI_ERR_ARG, "the first layer has one input channel and no input gradient");
    if (n < 1 || H < 1 || W < 1 || co < 8 || co % 8 || (!first && (ci < 8 || ci % 8)))
        return fail(ctx, DHFWI_ERR_ARG, "need n, H, W >= 1 and ci, co positive multiples of 8");
    const bool conv = kind != DHFWI_LAYER_CONVT;
    const int taps = conv ? 9 : 4, Ho = conv ? H : 2 * H, Wo = conv ? W : 2 * W;
    const long long Pin = (long long)n * H * W, Pout = (long long)n * Ho * Wo;
    if (Pout * std::max(ci, co) >= (1LL << 31)) return fail(ctx, DHFWI_ERR_ARG, "layer too large");
    if (!out_dev || (op != DHFWI_LAYER_DGRAD && !x_dev) || (op != DHFWI_LAYER_WGRAD && !w_dev) ||
        (op == DHFWI_LAYER_FWD && !b_dev) || (op != DHFWI_LAYER_FWD && !gy_dev))
        return fail(ctx, DHFWI_ERR_ARG, "NULL argument");
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    const long long nw = (long long)taps * ci * co;
    // Temporaries of this call only (freed before it returns).
    __nv_bfloat16 *x16 = nullptr, *w16 = nullptr, *wt16 = nullptr, *g16 = nullptr, *y16 = nullptr, *ones = nullptr;
    float *part = nullptr, *wg = nullptr;
    unsigned *err = nullptr;
    const int wM = conv ? co : 4 * co, wN = (conv ? 9 * ci : ci) + 8;
    const int splits = wgrad_splits(Pin, wM, wN);  // summed over the input grid's pixels
    const long long fp_floats = std::max<long long>(2LL * 152 * 4 * 128 * 64, 8LL * Pout * std::max(ci, 4 * co));
    const long long wg_floats = std::max<long long>((long long)splits * wM * wN, 512LL * wM);
    int rc = DHFWI_OK;
    auto cleanup = [&]() {
        void *ps[] = {x16, w16, wt16, g16, y16, ones, part, wg, err};
        for (void *p : ps) dev_free(p);
    };
    if ((rc = dev_alloc(ctx, (void **)&x16, 2 * (size_t)Pin * (first ? CPAD : ci))) ||
        (rc = dev_alloc(ctx, (void **)&w16, 2 * (size_t)nw)) || (rc = dev_alloc(ctx, (void **)&wt16, 2 * (size_t)nw)) ||
        (rc = dev_alloc(ctx, (void **)&g16, 2 * (size_t)Pout * co)) ||
        (rc = dev_alloc(ctx, (void **)&y16, 2 * (size_t)Pout * co)) || (rc = dev_alloc(ctx, (void **)&ones, 16)) ||
        (rc = dev_alloc(ctx, (void **)&part, 4 * (size_t)fp_floats)) ||
        (rc = dev_alloc(ctx, (void **)&wg, 4 * (size_t)wg_floats)) || (rc = dev_alloc(ctx, (void **)&err, 16))) {
        cleanup();
        return rc;
    }
    __nv_bfloat16 h1[8];
    for (int i = 0; i < 8; i++) h1[i] = __float2bfloat16_rn(i == 0 ? 1.0f : 0.0f);
    cudaError_t e = cudaMemcpy(ones, h1, sizeof h1, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(err, 0, 16);
    if (e != cudaSuccess) {
        cleanup();
        return fail(ctx, DHFWI_ERR_CUDA, cudaGetErrorString(e));
    }
    long long launches = 0;
    if (first) {  // the network's first layer: one input channel padded to CPAD, CUDA-core kernels
        if (x_dev) launch_input_pack(x_dev, Pin, CPAD, x16, s), launches++;
        if (w_dev) launch_to_bf16(w_dev, nw, w16, s), launches++;
        if (op == DHFWI_LAYER_FWD) {
            if (!launch_first_conv(x16, CPAD, n, H, W, w16, b_dev, co, 0.2f, y16, co, s)) {
                cleanup();
                return fail(ctx, DHFWI_ERR_ARG, "first layer: unsupported shape");
            }
            launch_bf16_to_f32(y16, Pout * co, out_dev, s);
            launches += 2;
        } else {
            launch_to_bf16(gy_dev, Pout * co, g16, s);
            const int k = launch_first_wgrad(g16, co, x16, CPAD, n, H, W, wg, wg_floats, out_dev, out_dev + nw, s);
            if (!k) {
                cleanup();
                return fail(ctx, DHFWI_ERR_ARG, "first layer: scratch too small");
            }
            launches += 1 + k;
        }
    }
    if (!first) {
        // Operands rounded to bf16 where the network rounds them.
        if (x_dev) launch_to_bf16(x_dev, Pin * ci, x16, s), launches++;
        if (w_dev) {
            launch_to_bf16(w_dev, nw, w16, s);
            if (!conv && op == DHFWI_LAYER_FWD) {  // the transposed conv's forward takes tap-major rows
                TransposeJobs ct{};
                ct.n = 1;
                ct.off[0] = 0;
                ct.co[0] = co;
                ct.taps[0] = 4;
                ct.ci[0] = ci;
                launch_convt_tapmajor_batch(w16, wt16, ct, s);
            } else {
                launch_transpose_w(w16, co, taps, ci, wt16, s);
            }
            launches += 2;
        }
        // The transposed conv's output gradient in space-to-depth layout, as the
        // network's backward pass keeps it.
        if (gy_dev) {
            if (conv) launch_to_bf16(gy_dev, Pout * co, g16, s);
            else launch_to_bf16_s2d(gy_dev, n, H, W, co, g16, s);
            launches++;
        }
        if (op == DHFWI_LAYER_FWD) {
            FpropArgs a{};
            a.src = x16;
            a.src_stride = ci;
            a.C = ci;
            a.Hs = H;
            a.Ws = W;
            a.Ho = H;
            a.Wo = W;
            a.M = (int)Pin;
            a.bt = w16;
            a.bias = b_dev;
            a.slope = 0.2f;
            a.dst_bf16 = y16;
            a.dst_stride = co;
            a.part = part;
            a.part_floats = fp_floats;
            a.err = err;
            a.scale = 1;
            if (conv) {
                a.ntaps = 9;
                for (int t = 0; t < 9; t++) {
                    a.dh[t] = t / 3 - 1;
                    a.dw[t] = t % 3 - 1;
                }
                a.N = co;
                launch_fprop(a, EPI_BF16_LEAKY, s);
            } else {
                a.ntaps = 1;
                a.dh[0] = a.dw[0] = 0;
                a.N = 4 * co;
                a.bt = wt16;  // tap-major copy
                launch_fprop(a, EPI_BF16_CONVT, s);
            }
            launch_bf16_to_f32(y16, Pout * co, out_dev, s);
            launches += 3;
        } else if (op == DHFWI_LAYER_DGRAD) {
            FpropArgs a{};
            a.src = g16;
            a.src_stride = co;
            a.C = co;
            a.Hs = Ho;
            a.Ws = Wo;
            a.Ho = H;
            a.Wo = W;
            a.M = (int)Pin;
            a.N = ci;
            a.bt = wt16;
            a.dst_f32 = out_dev;
            a.dst_stride = ci;
            a.part = part;
            a.part_floats = fp_floats;
            a.err = err;
            if (conv) {
                a.ntaps = 9;
                a.scale = 1;
                for (int t = 0; t < 9; t++) {
                    a.dh[t] = 1 - t / 3;
                    a.dw[t] = 1 - t % 3;
                }
            } else {  // one tap over the 4 co space-to-depth channels of the coarse grid
                a.src_stride = 4 * co;
                a.C = 4 * co;
                a.Hs = H;
                a.Ws = W;
                a.ntaps = 1;
                a.scale = 1;
                a.dh[0] = a.dw[0] = 0;
            }
            launch_fprop(a, EPI_F32, s);
            launches += 2;
        } else {
            WgradArgs w{};
            w.mode = conv ? WG_CONV : WG_CONVT;
            w.g = g16;
            w.g_stride = conv ? co : 4 * co;
            w.g_s2d = !conv;
            w.x = x16;
            w.x_stride = ci;
            w.nimg = n;
            w.H = H;
            w.W = W;
            w.ci = ci;
            w.co = co;
            w.M = wM;
            w.nw = conv ? 9 * ci : ci;
            w.N = wN;
            w.ones = ones;
            w.part = wg;
            w.err = err;
            launches += launch_wgrad(w, splits, out_dev, out_dev + nw, s);
        }
    }
    e = cudaGetLastError();
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(ctx, DHFWI_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return fail(ctx, DHFWI_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting for its MMAs");
    ctx_count_launches(ctx, launches);
    return DHFWI_OK;
}

int deblur_apply(dhfwi_ctx *ctx, const float *g_dev, int nz, int nx, float *out_dev, void *stream) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx_begin(ctx);
    NetState *net = ctx_net(ctx);
    if (!net || !net->have_weights) return fail(ctx, DHFWI_ERR_STATE, "train or set the network first");
    if (!g_dev || !out_dev || nz < 1 || nx < 1) return fail(ctx, DHFWI_ERR_ARG, "bad arguments");
    cudaSetDevice(ctx_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    NetState &N = *net;
    N.launches = 0;
    const int mult = 1 << N.levels;
    const int Hp = (nz + mult - 1) / mult * mult, Wp = (nx + mult - 1) / mult * mult;
    int rc = layout(ctx, N, 1, Hp, Wp);
    if (rc) return rc;
    const int mute = std::min(N.mute_rows, nz - 1);
    const long long moff = (long long)mute * nx;
    launch_absmax(g_dev + moff, (long long)nz * nx - moff, N.mx, N.scales, s);
    launch_pad_image(g_dev, nz, nx, Hp, Wp, N.scales, mute, N.V.xf, s);
    NCK(run_pass(N, PASS_FORWARD, 1, Hp, Wp, s));
    launch_crop_image(N.V.out, Hp, Wp, nz, nx, N.scales + 1, out_dev, s);
    N.launches += 5;
    NCK(cudaGetLastError());
    ctx_count_launches(ctx, N.launches);
    return DHFWI_OK;
}

}  // extern "C"
