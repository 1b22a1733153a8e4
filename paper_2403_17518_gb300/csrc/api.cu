// Host side of the C ABI declared in include/dhfwi.h: context, geometry
// plans (cached by content), validation, workspace and the batched time loops
// for model_shots, fwi_gradient, born_demig and rtm_mig.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dhfwi.h"
#include "fd_internal.h"
#include "nn_api.h"

using namespace dhfwi;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Plan {
    unsigned long long hash = 0;
    int n_shots = 0, nt_max = 0;
    std::vector<ShotDesc> shots;       // by slot
    std::vector<int> slot_of_shot;
    std::vector<int> nt_sorted;        // nt by slot (non-increasing)
    std::vector<Tile> tiles;           // with a sentinel at the end
    std::vector<TileRec> recs;
    std::vector<TileInfo> infos;       // per tile, same order (no sentinel)
    std::vector<int> tiles_prefix;     // tiles of the first m slots
    std::vector<int> rtiles;           // tiles with receivers, in tile order
    std::vector<int> rtiles_prefix;    // of those, the tiles of the first m slots
    std::vector<TileRec> xrecs;        // receivers of each tile's grown region (StepCommon::xrecs)
    std::vector<int> xrec_off;         // per tile, with a final end offset
    bool xinj = false;                 // every grown region holds at most kInjCap entries
    long long pool_floats = 0;
    int pitch = 0;                     // row pitch of every window in a pool
    long long n_data = 0;
    long long cells_per_step_all = 0;  // padded cells of all shots
    DevBuf d_shots, d_tiles, d_recs, d_slot_of, d_wav, d_infos, d_rtiles, d_xrecs, d_xrec_off;
};

}  // namespace

struct dhfwi_ctx {
    int device = 0;
    dhfwi_grid g{};
    std::string err;
    int pf = 0;             // pitch of padded model arrays
    int NZ = 0, NXF = 0;
    Plan plan;
    DevBuf kap, dkap, status, partial;
    DevBuf fields;          // general wavefield pools
    DevBuf ck;              // checkpoints of the segments that are recomputed
    DevBuf abuf;            // segment buffer of a^n (recomputed segments)
    // Stored a^n of the first hist_segs segments of ck_every steps, written by
    // the forward pass and read by the backward sweep (no recompute there).
    // Step n holds the active slots only: hoff[n] is its offset in floats.
    DevBuf hist;
    std::vector<long long> hoff;
    int hist_segs = 0;
    unsigned long long hist_plan = 0;  // plan hash and limit the split was made for
    long long hist_limit = -2;
    DevBuf dtmp, rtmp;      // data-sized temporaries
    unsigned *h_status = nullptr;   // pinned
    double *h_partial = nullptr;    // pinned
    int ck_every = 50;
    dhfwi_stats_t stats{};
    dhfwi::NetState *net = nullptr;
    bool timing = false;
    // Step-kernel launch choice per kind: forward, forward+segment store,
    // adjoint, Born.  Picked by autotune() for the current plan.
    StepLaunch launch[4];
    // Time steps per launch (1 or 2) of the forward and the adjoint sweeps,
    // chosen by the autotuner.
    int depth[2] = {2, 2};
    // Reuse of the stored forward wavefield between calls (dhfwi_set_reuse):
    // the identity of the last complete backward-capable forward pass (plan
    // hash, model hash, history segments, checkpoint interval) whose a^n
    // history and checkpoints are still intact.
    bool reuse = false;
    unsigned long long model_hash = 0;  // of the velocity of the current call (prep_model)
    struct {
        bool valid = false;
        unsigned long long plan = 0, model = 0;
        int segs = 0, K = 0;
    } fws;
    unsigned long long tuned_hash = 0;
    int nsm = 1;
    cudaEvent_t ev[3][2] = {};
    bool ev_used[3] = {};
    // Tensor maps of the TMA-staged kernels by (base pointer, shape kind);
    // cleared when a new plan changes the pool layout.
    std::map<std::pair<const void *, int>, CUtensorMap> tmaps;
};

namespace {

constexpr int RESID_BLOCKS = 1024;
constexpr int TFLAG_WORD = 4;  // status word set by a timed-out TMA wait
constexpr int NPOOLS = 9;  // field pools: u (2) + D, nu (2) + D_nu, image, second D, second D_nu

int fail(dhfwi_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(dhfwi_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? DHFWI_ERR_OOM : DHFWI_ERR_CUDA, m);
}

#define CK(call)                                           \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int ensure(dhfwi_ctx *ctx, DevBuf &b, size_t bytes, const char *what) {
    if (b.bytes >= bytes && b.p) return DHFWI_OK;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof msg, "allocating %s (%.3f GB): %s", what, bytes / 1e9, cudaGetErrorString(e));
        return fail(ctx, e == cudaErrorMemoryAllocation ? DHFWI_ERR_OOM : DHFWI_ERR_CUDA, msg);
    }
    b.bytes = bytes;
    return DHFWI_OK;
}

void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

unsigned long long fnv(unsigned long long h, const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

int round_up(int a, int m) { return (a + m - 1) / m * m; }

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (no link-time dependency on the driver library); null when unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

// Host validation of the geometry against the grid.
int validate_geom(dhfwi_ctx *ctx, const dhfwi_geom *G) {
    const dhfwi_grid &g = ctx->g;
    if (!G) return fail(ctx, DHFWI_ERR_ARG, "geometry is NULL");
    if (G->n_shots < 1) return fail(ctx, DHFWI_ERR_ARG, "n_shots must be >= 1");
    if (!G->src_iz || !G->src_ix || !G->nt || !G->rec_off || !G->win_x0 || !G->win_x1 || !G->wavelet)
        return fail(ctx, DHFWI_ERR_ARG, "geometry has a NULL array");
    if (G->nt_max < 1) return fail(ctx, DHFWI_ERR_ARG, "nt_max must be >= 1");
    if (G->rec_off[0] != 0) return fail(ctx, DHFWI_ERR_ARG, "rec_off[0] must be 0");
    if (G->rec_off[G->n_shots] > 0 && (!G->rec_iz || !G->rec_ix))
        return fail(ctx, DHFWI_ERR_ARG, "receiver arrays are NULL");
    char msg[256];
    for (int s = 0; s < G->n_shots; s++) {
        if (G->nt[s] < 1 || G->nt[s] > G->nt_max) {
            snprintf(msg, sizeof msg, "shot %d: nt=%d outside [1, nt_max=%d]", s, G->nt[s], G->nt_max);
            return fail(ctx, DHFWI_ERR_ARG, msg);
        }
        if (G->rec_off[s + 1] < G->rec_off[s]) return fail(ctx, DHFWI_ERR_ARG, "rec_off not monotone");
        int x0 = G->win_x0[s], x1 = G->win_x1[s];
        if (x0 < 0 || x1 > g.nx || x1 <= x0) {
            snprintf(msg, sizeof msg, "shot %d: window [%d,%d) outside [0,%d)", s, x0, x1, g.nx);
            return fail(ctx, DHFWI_ERR_GEOM, msg);
        }
        auto inside = [&](int iz, int ix) { return iz >= 0 && iz < g.nz && ix >= x0 && ix < x1; };
        if (!inside(G->src_iz[s], G->src_ix[s])) {
            snprintf(msg, sizeof msg, "shot %d: source (%d,%d) outside its window", s, G->src_iz[s], G->src_ix[s]);
            return fail(ctx, DHFWI_ERR_GEOM, msg);
        }
        for (int r = G->rec_off[s]; r < G->rec_off[s + 1]; r++) {
            if (!inside(G->rec_iz[r], G->rec_ix[r])) {
                snprintf(msg, sizeof msg, "shot %d: receiver %d (%d,%d) outside its window", s, r - G->rec_off[s],
                         G->rec_iz[r], G->rec_ix[r]);
                return fail(ctx, DHFWI_ERR_GEOM, msg);
            }
        }
    }
    return DHFWI_OK;
}

unsigned long long geom_hash(const dhfwi_grid &g, const dhfwi_geom *G) {
    unsigned long long h = 1469598103934665603ull;
    h = fnv(h, &g, sizeof g);
    h = fnv(h, &G->n_shots, sizeof(int));
    h = fnv(h, &G->nt_max, sizeof(int));
    h = fnv(h, &G->wavelet_shared, sizeof(int));
    const int ns = G->n_shots;
    h = fnv(h, G->src_iz, sizeof(int) * ns);
    h = fnv(h, G->src_ix, sizeof(int) * ns);
    h = fnv(h, G->nt, sizeof(int) * ns);
    h = fnv(h, G->rec_off, sizeof(int) * (ns + 1));
    const int nr = G->rec_off[ns];
    if (nr > 0) {
        h = fnv(h, G->rec_iz, sizeof(int) * nr);
        h = fnv(h, G->rec_ix, sizeof(int) * nr);
    }
    h = fnv(h, G->win_x0, sizeof(int) * ns);
    h = fnv(h, G->win_x1, sizeof(int) * ns);
    size_t nw = (size_t)G->nt_max * (G->wavelet_shared ? 1 : ns);
    h = fnv(h, G->wavelet, sizeof(float) * nw);
    return h;
}

template <typename T>
int upload(dhfwi_ctx *ctx, DevBuf &b, const std::vector<T> &v, const char *what) {
    int rc = ensure(ctx, b, std::max<size_t>(sizeof(T) * v.size(), 16), what);
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return DHFWI_OK;
}

// Builds (or reuses) the plan for this geometry.
int get_plan(dhfwi_ctx *ctx, const dhfwi_geom *G) {
    int rc = validate_geom(ctx, G);
    if (rc) return rc;
    unsigned long long h = geom_hash(ctx->g, G);
    Plan &P = ctx->plan;
    if (P.hash == h && P.n_shots == G->n_shots) return DHFWI_OK;
    const int nb = ctx->g.nb, NZ = ctx->NZ, ns = G->n_shots;
    // The plan's device tables may still be read by earlier work on any stream.
    CK(cudaDeviceSynchronize());
    P.hash = 0;
    ctx->fws.valid = false;
    ctx->tmaps.clear();
    P.n_shots = ns;
    P.nt_max = G->nt_max;
    std::vector<int> order(ns);
    for (int s = 0; s < ns; s++) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return G->nt[a] > G->nt[b]; });
    std::vector<long long> doff(ns + 1, 0);
    for (int s = 0; s < ns; s++)
        doff[s + 1] = doff[s] + (long long)G->nt[s] * (G->rec_off[s + 1] - G->rec_off[s]);
    P.n_data = doff[ns];
    P.shots.assign(ns, ShotDesc{});
    P.slot_of_shot.assign(ns, 0);
    P.nt_sorted.assign(ns, 0);
    P.tiles.clear();
    P.recs.clear();
    P.tiles_prefix.assign(ns + 1, 0);
    P.rtiles.clear();
    P.rtiles_prefix.assign(ns + 1, 0);
    P.xrecs.clear();
    P.xrec_off.clear();
    P.xinj = true;
    // One row pitch for all windows: a pool is then a [slot][NZ][pitch] array
    // that a single 3-D tensor map describes.
    int pitch = POOL_ALIGN;
    for (int s = 0; s < ns; s++) pitch = std::max(pitch, round_up(G->win_x1[s] - G->win_x0[s] + 2 * nb, POOL_ALIGN));
    P.pitch = pitch;
    long long foff = 0;
    P.cells_per_step_all = 0;
    for (int k = 0; k < ns; k++) {
        const int s = order[k];
        ShotDesc &sd = P.shots[k];
        const int x0 = G->win_x0[s], x1 = G->win_x1[s];
        sd.nxw = x1 - x0 + 2 * nb;
        sd.pitch = pitch;
        sd.foff = foff;
        foff += (long long)pitch * NZ;
        sd.doff = doff[s];
        sd.x0 = x0;
        sd.sz = G->src_iz[s] + nb;
        sd.sx = G->src_ix[s] - x0 + nb;
        sd.nt = G->nt[s];
        sd.nrec = G->rec_off[s + 1] - G->rec_off[s];
        sd.wav_off = G->wavelet_shared ? 0 : s * G->nt_max;
        sd.shot = s;
        P.slot_of_shot[s] = k;
        P.nt_sorted[k] = sd.nt;
        P.cells_per_step_all += (long long)sd.nxw * NZ;
        // Tiles of this shot, and its receivers bucketed per tile.
        const int ntz = (NZ + TZ - 1) / TZ, ntx = (sd.nxw + TX - 1) / TX;
        std::vector<std::vector<TileRec>> bucket((size_t)ntz * ntx);
        for (int r = 0; r < sd.nrec; r++) {
            const int rz = G->rec_iz[G->rec_off[s] + r] + nb;
            const int rx = G->rec_ix[G->rec_off[s] + r] - x0 + nb;
            bucket[(size_t)(rz / TZ) * ntx + rx / TX].push_back(TileRec{(rz % TZ) * TX + rx % TX, r});
        }
        for (int tz = 0; tz < ntz; tz++)
            for (int tx = 0; tx < ntx; tx++) {
                P.tiles.push_back(Tile{k, tz * TZ, tx * TX, (int)P.recs.size()});
                // By cell, then receiver: the adjoint sums receivers sharing a
                // cell in this order (deterministic injection).
                std::vector<TileRec> &bk = bucket[(size_t)tz * ntx + tx];
                std::sort(bk.begin(), bk.end(), [](const TileRec &a, const TileRec &b) {
                    return a.cell < b.cell || (a.cell == b.cell && a.r < b.r);
                });
                for (const TileRec &e : bk) P.recs.push_back(e);
            }
        P.tiles_prefix[k + 1] = (int)P.tiles.size();
        // Receivers of each tile's grown region ((TX + 2 HALO)^2 cells), by
        // cell then receiver as the per-tile lists.
        {
            constexpr int EW = TX + 2 * HALO;
            std::vector<std::vector<TileRec>> xb((size_t)ntz * ntx);
            for (int r = 0; r < sd.nrec; r++) {
                const int rz = G->rec_iz[G->rec_off[s] + r] + nb;
                const int rx = G->rec_ix[G->rec_off[s] + r] - x0 + nb;
                for (int tz = 0; tz < ntz; tz++) {
                    const int ez = rz - (tz * TZ - HALO);
                    if (ez < 0 || ez >= EW) continue;
                    for (int tx = 0; tx < ntx; tx++) {
                        const int ex = rx - (tx * TX - HALO);
                        if (ex >= 0 && ex < EW) xb[(size_t)tz * ntx + tx].push_back(TileRec{ez * EW + ex, r});
                    }
                }
            }
            for (size_t t = 0; t < xb.size(); t++) {
                std::vector<TileRec> &bk = xb[t];
                std::sort(bk.begin(), bk.end(), [](const TileRec &a, const TileRec &b) {
                    return a.cell < b.cell || (a.cell == b.cell && a.r < b.r);
                });
                P.xrec_off.push_back((int)P.xrecs.size());
                if ((int)bk.size() > kInjCap) P.xinj = false;
                for (const TileRec &e : bk) P.xrecs.push_back(e);
            }
        }
        for (int ti = P.tiles_prefix[k]; ti < P.tiles_prefix[k + 1]; ti++) {
            const int rb = P.tiles[ti].rec_begin;
            const int re = ti + 1 < (int)P.tiles.size() ? P.tiles[ti + 1].rec_begin : (int)P.recs.size();
            if (re > rb) P.rtiles.push_back(ti);
        }
        P.rtiles_prefix[k + 1] = (int)P.rtiles.size();
    }
    P.xrec_off.push_back((int)P.xrecs.size());  // end of the last tile's list
    if (P.xrecs.empty()) P.xrecs.push_back(TileRec{0, 0});  // (a valid device pointer)
    P.tiles.push_back(Tile{0, 0, 0, (int)P.recs.size()});  // sentinel
    P.infos.resize(P.tiles.size() - 1);
    for (size_t i = 0; i + 1 < P.tiles.size(); i++) {
        const Tile &t = P.tiles[i];
        const ShotDesc &sd = P.shots[t.slot];
        TileInfo &T = P.infos[i];
        T = TileInfo{};
        T.slot = t.slot;
        T.z0 = t.z0;
        T.x0 = t.x0;
        T.mx = (sd.x0 & ~3) + t.x0;
        T.mc = sd.x0 & 3;
        T.nxw = sd.nxw;
        T.pitch = sd.pitch;
        T.sz = sd.sz;
        T.sx = sd.sx;
        T.wav_off = sd.wav_off;
        T.nrec = sd.nrec;
        T.rec_begin = t.rec_begin;
        T.rec_end = P.tiles[i + 1].rec_begin;
        T.foff = sd.foff;
        T.doff = sd.doff;
        const bool interior = t.z0 >= nb && t.z0 + TZ <= NZ - nb && t.x0 >= nb && t.x0 + TX <= sd.nxw - nb;
        const bool src = sd.sz >= t.z0 && sd.sz < t.z0 + TZ && sd.sx >= t.x0 && sd.sx < t.x0 + TX;
        // The same with the tile grown by HALO on every side (two-step kernel).
        const bool interior2 = t.z0 - HALO >= nb && t.z0 + TZ + HALO <= NZ - nb && t.x0 - HALO >= nb &&
                               t.x0 + TX + HALO <= sd.nxw - nb;
        const bool src2 = sd.sz >= t.z0 - HALO && sd.sz < t.z0 + TZ + HALO && sd.sx >= t.x0 - HALO &&
                          sd.sx < t.x0 + TX + HALO;
        T.flags = (interior ? TI_INTERIOR : 0) | (interior && !src ? TI_FULL_FWD : 0) |
                  (interior2 && !src2 ? TI_FULL2 : 0) | (interior2 ? TI_INTERIOR2 : 0);
        T.nt = sd.nt;
    }
    P.pool_floats = foff;
    std::vector<float> wav((size_t)G->nt_max * (G->wavelet_shared ? 1 : ns));
    std::memcpy(wav.data(), G->wavelet, sizeof(float) * wav.size());
    if ((rc = upload(ctx, P.d_shots, P.shots, "shot table"))) return rc;
    if ((rc = upload(ctx, P.d_tiles, P.tiles, "tile table"))) return rc;
    if ((rc = upload(ctx, P.d_recs, P.recs, "receiver table"))) return rc;
    if ((rc = upload(ctx, P.d_slot_of, P.slot_of_shot, "slot table"))) return rc;
    if ((rc = upload(ctx, P.d_wav, wav, "wavelets"))) return rc;
    if ((rc = upload(ctx, P.d_infos, P.infos, "tile descriptors"))) return rc;
    if ((rc = upload(ctx, P.d_rtiles, P.rtiles, "receiver tile list"))) return rc;
    if ((rc = upload(ctx, P.d_xrecs, P.xrecs, "grown-region receiver table"))) return rc;
    if ((rc = upload(ctx, P.d_xrec_off, P.xrec_off, "grown-region receiver offsets"))) return rc;
    P.hash = h;
    return DHFWI_OK;
}

// Number of active tiles at forward step n (shots with nt > n).
inline int active_tiles(const Plan &P, int n) {
    // nt_sorted is non-increasing; count slots with nt > n.
    int lo = 0, hi = P.n_shots;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (P.nt_sorted[mid] > n) lo = mid + 1;
        else hi = mid;
    }
    return P.tiles_prefix[lo];
}

// Number of slots (shots) with nt > n.
inline int active_slots(const Plan &P, int n) {
    int lo = 0, hi = P.n_shots;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (P.nt_sorted[mid] > n) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

long long active_cells(const Plan &P, int n, int NZ) {
    long long c = 0;
    for (int k = 0; k < P.n_shots && P.nt_sorted[k] > n; k++) c += (long long)P.shots[k].nxw * NZ;
    return c;
}

StepCommon common(dhfwi_ctx *ctx) {
    StepCommon c;
    c.shots = (const ShotDesc *)ctx->plan.d_shots.p;
    c.tiles = (const Tile *)ctx->plan.d_tiles.p;
    c.recs = (const TileRec *)ctx->plan.d_recs.p;
    c.infos = (const TileInfo *)ctx->plan.d_infos.p;
    c.kap = (const float *)ctx->kap.p;
    c.mstride = (long long)ctx->NZ * ctx->pf;
    c.wav = (const float *)ctx->plan.d_wav.p;
    c.pf = ctx->pf;
    c.NZ = ctx->NZ;
    c.nb = ctx->g.nb;
    c.tflag = (unsigned *)ctx->status.p + TFLAG_WORD;
    if (ctx->plan.xinj) {
        c.xrecs = (const TileRec *)ctx->plan.d_xrecs.p;
        c.xrec_off = (const int *)ctx->plan.d_xrec_off.p;
    }
    return c;
}

// Tensor-map shape kinds: field pool with halo box, field pool cell box,
// model array (4 copies) cell box.
enum { MAP_POOL_HALO = 0, MAP_POOL_CELL = 1, MAP_MODEL = 2, MAP_POOL_HALO2 = 3, MAP_MODEL_HALO = 4 };

// The tensor map of one array for the TMA-staged kernels (cached).
int tensor_map(dhfwi_ctx *ctx, const float *base, int kind, CUtensorMap *out) {
    auto key = std::make_pair((const void *)base, kind);
    auto it = ctx->tmaps.find(key);
    if (it != ctx->tmaps.end()) {
        *out = it->second;
        return DHFWI_OK;
    }
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(ctx, DHFWI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const Plan &P = ctx->plan;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3] = {TX, TZ, 1}, estr[3] = {1, 1, 1};
    if (kind == MAP_POOL_HALO || kind == MAP_MODEL_HALO) {
        box[0] = TX + 2 * HALO;
        box[1] = TZ + 2 * HALO;
    } else if (kind == MAP_POOL_HALO2) {
        box[0] = TX + 2 * HALO2;
        box[1] = TZ + 2 * HALO2;
    }
    if (kind == MAP_MODEL || kind == MAP_MODEL_HALO) {
        dims[0] = ctx->pf;
        dims[1] = ctx->NZ;
        dims[2] = 4;
        strides[0] = sizeof(float) * (cuuint64_t)ctx->pf;
        strides[1] = sizeof(float) * (cuuint64_t)ctx->NZ * ctx->pf;
    } else {
        dims[0] = P.pitch;
        dims[1] = ctx->NZ;
        dims[2] = P.n_shots;
        strides[0] = sizeof(float) * (cuuint64_t)P.pitch;
        strides[1] = sizeof(float) * (cuuint64_t)P.pitch * ctx->NZ;
    }
    CUtensorMap m;
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[128];
        snprintf(msg, sizeof msg, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
        return fail(ctx, DHFWI_ERR_CUDA, msg);
    }
    ctx->tmaps[key] = m;
    *out = m;
    return DHFWI_OK;
}

// Maps of a forward-step launch (u^n halo, D^n, kappa).
int fwd_maps(dhfwi_ctx *ctx, const FwdArgs &a, TileMaps *M) {
    int rc;
    if ((rc = tensor_map(ctx, a.u, MAP_POOL_HALO, &M->m[0]))) return rc;
    if ((rc = tensor_map(ctx, a.dd, MAP_POOL_CELL, &M->m[1]))) return rc;
    return tensor_map(ctx, a.c.kap, MAP_MODEL, &M->m[2]);
}

// Maps of an adjoint-step launch (nu^{k+1} halo, D_nu, kappa, a^{k-1}).
int adj_maps(dhfwi_ctx *ctx, const AdjArgs &b, TileMaps *M) {
    int rc;
    if ((rc = tensor_map(ctx, b.nu, MAP_POOL_HALO, &M->m[0]))) return rc;
    if ((rc = tensor_map(ctx, b.dd, MAP_POOL_CELL, &M->m[1]))) return rc;
    if ((rc = tensor_map(ctx, b.c.kap, MAP_MODEL, &M->m[2]))) return rc;
    return tensor_map(ctx, b.a, MAP_POOL_CELL, &M->m[3]);
}

// Maps of a Born-step launch (u0^n and p^n halos, D_u0, D_p, kappa, d kappa).
int born_maps(dhfwi_ctx *ctx, const BornArgs &b, TileMaps *M) {
    int rc;
    if ((rc = tensor_map(ctx, b.u, MAP_POOL_HALO, &M->m[0]))) return rc;
    if ((rc = tensor_map(ctx, b.p, MAP_POOL_HALO, &M->m[1]))) return rc;
    if ((rc = tensor_map(ctx, b.du, MAP_POOL_CELL, &M->m[2]))) return rc;
    if ((rc = tensor_map(ctx, b.dp, MAP_POOL_CELL, &M->m[3]))) return rc;
    if ((rc = tensor_map(ctx, b.c.kap, MAP_MODEL, &M->m[4]))) return rc;
    return tensor_map(ctx, b.dkap, MAP_MODEL, &M->m[5]);
}

int adj_step(dhfwi_ctx *ctx, const AdjArgs &b, int ntiles, const StepLaunch &L, cudaStream_t st) {
    if (L.variant >= FIRST_TMA_VARIANT) {
        TileMaps M;
        int rc = adj_maps(ctx, b, &M);
        if (rc) return rc;
        launch_adj_step(b, ntiles, L, &M, st);
    } else {
        launch_adj_step(b, ntiles, L, nullptr, st);
    }
    return DHFWI_OK;
}

int born_step(dhfwi_ctx *ctx, const BornArgs &b, int ntiles, const StepLaunch &L, cudaStream_t st) {
    if (L.variant >= FIRST_TMA_VARIANT) {
        TileMaps M;
        int rc = born_maps(ctx, b, &M);
        if (rc) return rc;
        launch_born_step(b, ntiles, L, &M, st);
    } else {
        launch_born_step(b, ntiles, L, nullptr, st);
    }
    return DHFWI_OK;
}

// Forward-step launch with the maps its variant needs.
int fwd_step(dhfwi_ctx *ctx, const FwdArgs &a, int ntiles, const StepLaunch &L, cudaStream_t st) {
    if (L.variant >= FIRST_TMA_VARIANT) {
        TileMaps M;
        int rc = fwd_maps(ctx, a, &M);
        if (rc) return rc;
        launch_fwd_step(a, ntiles, L, &M, st);
    } else {
        launch_fwd_step(a, ntiles, L, nullptr, st);
    }
    return DHFWI_OK;
}

// Padded model arrays from v (and dv), with the velocity / CFL check.
int prep_model(dhfwi_ctx *ctx, const float *v, const float *dv, int rel, cudaStream_t st) {
    if (!v) return fail(ctx, DHFWI_ERR_ARG, "velocity pointer is NULL");
    size_t mb = sizeof(float) * (size_t)ctx->NZ * ctx->pf;
    int rc;
    if ((rc = ensure(ctx, ctx->kap, 4 * mb, "kappa"))) return rc;
    if (dv && (rc = ensure(ctx, ctx->dkap, 4 * mb, "d kappa"))) return rc;
    CK(cudaMemsetAsync(ctx->status.p, 0, 2 * sizeof(unsigned), st));
    CK(cudaMemsetAsync((unsigned *)ctx->status.p + 8, 0, 2 * sizeof(unsigned), st));  // model hash
    const double c = ((double)ctx->g.dt * ctx->g.dt) / ((double)ctx->g.h * ctx->g.h);
    launch_prep_model(v, dv, rel, ctx->g.nz, ctx->g.nx, ctx->g.nb, c, (float *)ctx->kap.p,
                      dv ? (float *)ctx->dkap.p : nullptr, ctx->pf, (long long)ctx->NZ * ctx->pf,
                      (unsigned *)ctx->status.p, st);
    ctx->stats.kernel_launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_status, ctx->status.p, 10 * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->model_hash = (unsigned long long)ctx->h_status[8] | ((unsigned long long)ctx->h_status[9] << 32);
    if (ctx->h_status[TFLAG_WORD]) {
        CK(cudaMemset((unsigned *)ctx->status.p + TFLAG_WORD, 0, sizeof(unsigned)));
        return fail(ctx, DHFWI_ERR_TIMEOUT, "a step kernel of an earlier call timed out waiting for its tile copies");
    }
    if (ctx->h_status[0])
        return fail(ctx, DHFWI_ERR_NONFINITE, "velocity must be finite and > 0 (and dv finite)");
    float kmax;
    std::memcpy(&kmax, &ctx->h_status[1], sizeof kmax);
    // Leapfrog stability: kappa * (spectral radius of -D) <= 4, where the 2D
    // radius of the 8th-order stencil is 2 (|c0| + 2 sum |c_k|).
    const double S = 2.0 * (205.0 / 72.0 + 2.0 * (8.0 / 5.0 + 1.0 / 5.0 + 8.0 / 315.0 + 1.0 / 560.0));
    if ((double)kmax * S > 4.0) {
        char msg[160];
        snprintf(msg, sizeof msg, "CFL violated: v_max dt/h = %.4f > %.4f", std::sqrt((double)kmax),
                 std::sqrt(4.0 / S));
        return fail(ctx, DHFWI_ERR_CFL, msg);
    }
    return DHFWI_OK;
}

// Synchronises the stream and returns DHFWI_ERR_TIMEOUT (clearing the
// record) if a step kernel of this call, or of an earlier one not yet
// reported, ran out a bounded wait: calls that synchronise anyway report a
// timeout themselves instead of leaving it to the next call.
int sync_and_check_timeout(dhfwi_ctx *ctx, cudaStream_t st) {
    CK(cudaMemcpyAsync(ctx->h_status + TFLAG_WORD, (unsigned *)ctx->status.p + TFLAG_WORD, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctx->h_status[TFLAG_WORD]) {
        ctx->h_status[TFLAG_WORD] = 0;
        CK(cudaMemset((unsigned *)ctx->status.p + TFLAG_WORD, 0, sizeof(unsigned)));
        return fail(ctx, DHFWI_ERR_TIMEOUT, "a step kernel timed out waiting for its tile copies");
    }
    return DHFWI_OK;
}

int begin_call(dhfwi_ctx *ctx) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx->err.clear();
    ctx->stats.cell_updates = 0;
    ctx->stats.kernel_launches = 0;
    ctx->stats.shot_groups = 1;
    ctx->stats.history_steps = 0;
    ctx->stats.history_cells = 0;
    ctx->stats.reused = 0;
    for (int i = 0; i < 3; i++) {
        ctx->stats.phase_ms[i] = 0.0;
        ctx->stats.phase_launches[i] = 0;
        ctx->stats.phase_cells[i] = 0;
        ctx->ev_used[i] = false;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return DHFWI_OK;
}

void phase_begin(dhfwi_ctx *ctx, int ph, cudaStream_t st) {
    if (!ctx->timing) return;
    if (!ctx->ev[ph][0]) {
        cudaEventCreate(&ctx->ev[ph][0]);
        cudaEventCreate(&ctx->ev[ph][1]);
    }
    cudaEventRecord(ctx->ev[ph][0], st);
}

void phase_end(dhfwi_ctx *ctx, int ph, cudaStream_t st, long long launches, long long cells) {
    ctx->stats.phase_launches[ph] += launches;
    ctx->stats.phase_cells[ph] += cells;
    if (!ctx->timing) return;
    cudaEventRecord(ctx->ev[ph][1], st);
    ctx->ev_used[ph] = true;
}

bool time_blocking(const dhfwi_ctx *ctx, int which);

int end_call(dhfwi_ctx *ctx) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    ctx->stats.checkpoint_every = ctx->ck_every;
    for (int k = 0; k < 4; k++) ctx->stats.step_variant[k] = ctx->launch[k].variant;
    for (int k = 0; k < 2; k++) ctx->stats.time_block[k] = time_blocking(ctx, k) ? 2 : 1;
    double ws = ctx->kap.bytes + ctx->dkap.bytes + ctx->fields.bytes + ctx->ck.bytes +
                ctx->abuf.bytes + ctx->hist.bytes + ctx->dtmp.bytes + ctx->rtmp.bytes;
    ctx->stats.workspace_bytes = ws;
    return DHFWI_OK;
}

void set_variant(dhfwi_ctx *ctx, int kind, int v) {
    static const int kernel_kind[4] = {0, 0, 1, 2};
    ctx->launch[kind].variant = v;
    ctx->launch[kind].max_ctas = step_occupancy(kernel_kind[kind], v, kind == 1) * ctx->nsm;
    cudaGetLastError();
}

int tune_depth(dhfwi_ctx *ctx, cudaStream_t st, const float *one_step_ms, int reps);

// Autotuner: for the current plan, time every step-kernel variant of each
// kind on the plan's full tile list (all shots active) using the scratch
// field pools, and keep the fastest; then the time-blocking depth of the
// forward and adjoint sweeps (tune_depth).  The pools are zeroed again by the
// call that follows, so tuning leaves no trace in the results.  Runs once per
// geometry; DHFWI_STEP_VARIANT=<0..6> pins a variant instead (and the depth
// stays two unless DHFWI_TIME_BLOCK says otherwise).
int autotune(dhfwi_ctx *ctx, cudaStream_t st) {
    const Plan &P = ctx->plan;
    if (ctx->tuned_hash == P.hash) return DHFWI_OK;
    static const int kernel_kind[4] = {0, 0, 1, 2};
    const char *pin = getenv("DHFWI_STEP_VARIANT");
    if (pin && *pin) {
        // A kind without the pinned variant takes its last one (a pin past
        // every kind's range, or negative, takes the default).
        const int v = atoi(pin);
        const bool valid = v >= 0 && v < N_STEP_VARIANTS;
        for (int k = 0; k < 4; k++)
            set_variant(ctx, k, valid ? std::min(v, step_variants(kernel_kind[k]) - 1) : 1);
        ctx->tuned_hash = P.hash;
        return DHFWI_OK;
    }
    const long long pool = P.pool_floats;
    int rc = ensure(ctx, ctx->fields, NPOOLS * sizeof(float) * (size_t)pool, "wavefield pools");
    if (rc) return rc;
    if ((rc = ensure(ctx, ctx->rtmp, sizeof(float) * std::max<long long>(P.n_data, 1), "residual"))) return rc;
    if ((rc = ensure(ctx, ctx->dtmp, sizeof(float) * std::max<long long>(P.n_data, 1), "synthetic data")))
        return rc;
    float *F = (float *)ctx->fields.p;
    CK(cudaMemsetAsync(F, 0, sizeof(float) * NPOOLS * (size_t)pool, st));
    CK(cudaMemsetAsync(ctx->rtmp.p, 0, sizeof(float) * std::max<long long>(P.n_data, 1), st));
    const int ntiles = active_tiles(P, 0);
    const int reps = 4;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    long long timed = 0;
    float best_ms[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kind = 0; kind < 4; kind++) {
        float best = 1e30f;
        int best_v = 1;
        int nv = step_variants(kernel_kind[kind]);
        if (!encode_tiled()) nv = std::min(nv, (int)FIRST_TMA_VARIANT);
        for (int v = 0; v < nv; v++) {
            set_variant(ctx, kind, v);
            float ms = 0.f;
            rc = DHFWI_OK;
            for (int rep = -1; rep < reps && !rc; rep++) {
                if (rep == 0) cudaEventRecord(e0, st);
                if (kind <= 1) {
                    FwdArgs a{};
                    a.c = common(ctx);
                    a.u = F;
                    a.un = F + pool;
                    a.dd = F + 2 * pool;
                    a.a_out = kind == 1 ? F + 3 * pool : nullptr;
                    a.d = kind == 0 ? (float *)ctx->dtmp.p : nullptr;
                    a.n = 0;
                    if ((rc = fwd_step(ctx, a, ntiles, ctx->launch[kind], st))) break;
                } else if (kind == 2) {
                    AdjArgs b{};
                    b.c = common(ctx);
                    b.nu = F;
                    b.nun = F + pool;
                    b.dd = F + 2 * pool;
                    b.a = F + 3 * pool;
                    b.g = F + 4 * pool;
                    b.r = (const float *)ctx->rtmp.p;
                    b.k = 1;
                    if ((rc = adj_step(ctx, b, ntiles, ctx->launch[kind], st))) break;
                } else {
                    BornArgs b{};
                    b.c = common(ctx);
                    b.u = F;
                    b.un = F + pool;
                    b.du = F + 2 * pool;
                    b.p = F + 3 * pool;
                    b.pn = F + 4 * pool;
                    b.dp = F + 5 * pool;
                    b.dkap = (const float *)ctx->kap.p;
                    b.d = (float *)ctx->dtmp.p;
                    b.n = 0;
                    if ((rc = born_step(ctx, b, ntiles, ctx->launch[kind], st))) break;
                }
            }
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(ctx, e, "autotune");
            }
            if (rc) {  // a variant that cannot be launched here is not a candidate
                ctx->err.clear();
                continue;
            }
            timed += reps + 1;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        set_variant(ctx, kind, best_v);
        best_ms[kind] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->stats.kernel_launches += timed;
    if ((rc = tune_depth(ctx, st, best_ms, reps))) return rc;
    ctx->tuned_hash = P.hash;
    CK(cudaGetLastError());
    return DHFWI_OK;
}

// DHFWI_TIME_BLOCK=0 forces one time step per launch, any other value two;
// unset, the autotuner's choice applies (read per call).  Without tensor
// maps there are no two-step kernels.
bool time_blocking(const dhfwi_ctx *ctx, int which) {
    if (!encode_tiled()) return false;
    const char *e = getenv("DHFWI_TIME_BLOCK");
    if (e && *e) return strcmp(e, "0") != 0;
    return ctx->depth[which] == 2;
}

// Maps of a two-step forward launch (u^n with the doubled halo, D^n with
// its ring, kappa with its ring).
int pair_maps(dhfwi_ctx *ctx, const FwdArgs &a, TileMaps *M) {
    int rc;
    if ((rc = tensor_map(ctx, a.u, MAP_POOL_HALO2, &M->m[0]))) return rc;
    if ((rc = tensor_map(ctx, a.dd, MAP_POOL_HALO, &M->m[1]))) return rc;
    return tensor_map(ctx, a.c.kap, MAP_MODEL_HALO, &M->m[2]);
}

// Maps of a two-step adjoint launch (nu^{k+1} with the doubled halo, D_nu
// with its ring, kappa with its ring; the image, a^{k-1} and a^{k-2}, which
// the kernel only prefetches into L2).  A history step's map spans all
// slots from its base: the spare pool at the history's end keeps it inside
// the allocation.
int adj_pair_maps(dhfwi_ctx *ctx, const AdjArgs &b, TileMaps *M) {
    int rc;
    if ((rc = tensor_map(ctx, b.nu, MAP_POOL_HALO2, &M->m[0]))) return rc;
    if ((rc = tensor_map(ctx, b.dd, MAP_POOL_HALO, &M->m[1]))) return rc;
    if ((rc = tensor_map(ctx, b.c.kap, MAP_MODEL_HALO, &M->m[2]))) return rc;
    if ((rc = tensor_map(ctx, b.g, MAP_POOL_CELL, &M->m[3]))) return rc;
    if ((rc = tensor_map(ctx, b.a, MAP_POOL_CELL, &M->m[4]))) return rc;
    return tensor_map(ctx, b.a2, MAP_POOL_CELL, &M->m[5]);
}

// Time-blocking depth of the forward and the adjoint sweeps: `reps` launches
// of the two-step kernel on the plan's full tile list against twice the
// chosen one-step kernel's time for as many launches (one_step_ms: the
// variant loop's best time of `reps` launches per kind: forward, forward with
// store, adjoint, Born).  The faster depth is kept.
int tune_depth(dhfwi_ctx *ctx, cudaStream_t st, const float *one_step_ms, int reps) {
    if (!encode_tiled()) return DHFWI_OK;
    const Plan &P = ctx->plan;
    const long long pool = P.pool_floats;
    float *F = (float *)ctx->fields.p;
    const int ntiles = active_tiles(P, 0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = DHFWI_OK;
    for (int which = 0; which < 2 && !rc; which++) {
        float ms = 0.f;
        for (int rep = -1; rep < reps && !rc; rep++) {
            if (rep == 0) cudaEventRecord(e0, st);
            TileMaps M;
            if (which == 0) {
                FwdArgs a{};
                a.c = common(ctx);
                a.u = F;
                a.un = F + pool;
                a.dd = F + 2 * pool;
                a.dd_out = F + 7 * pool;
                a.d = (float *)ctx->dtmp.p;
                a.n = 0;
                if (!(rc = pair_maps(ctx, a, &M))) launch_fwd_pair(a, ntiles, M, st);
                ctx->stats.kernel_launches++;
            } else {
                AdjArgs b{};
                b.c = common(ctx);
                b.nu = F;
                b.nun = F + pool;
                b.dd = F + 2 * pool;
                b.dd_out = F + 8 * pool;
                b.a = F + 3 * pool;
                b.a2 = F + 5 * pool;
                b.g = F + 4 * pool;
                b.r = (const float *)ctx->rtmp.p;
                b.k = 2;
                b.inject_here = P.xinj ? 1 : 0;
                const int nrt = P.xinj ? 0 : P.rtiles_prefix[active_slots(P, 1)];
                launch_adj_inject(b, (const int *)P.d_rtiles.p, nrt, st);
                if (!(rc = adj_pair_maps(ctx, b, &M))) launch_adj_pair(b, ntiles, M, st);
                ctx->stats.kernel_launches += 1 + (nrt > 0);
            }
        }
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(ctx, e, "autotune (time-blocking depth)");
        }
        if (rc) break;
        cudaEventElapsedTime(&ms, e0, e1);
        const float one = one_step_ms[which == 0 ? 0 : 2];
        ctx->depth[which] = ms <= 2.f * one ? 2 : 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {  // no two-step launch possible here: one step per launch
        ctx->err.clear();
        ctx->depth[0] = ctx->depth[1] = 1;
    }
    return DHFWI_OK;
}

// Advances the forward state from step n: two steps with one two-step launch
// when blocking is on and n + 1 < n_end, else one.  State: u in *cur (next
// in *nxt), D in *dcur (*dnxt: the two-step kernel's output pool).  a_slot(n)
// gives the segment slot for a^n (nullptr: no segment store).  Returns the
// number of steps taken, or a negative error code.
template <typename SlotFn>
int forward_steps(dhfwi_ctx *ctx, FwdArgs &a, int n, int n_end, float *&cur, float *&nxt, float *&dcur,
                  float *&dnxt, const StepLaunch &L, bool blocking, SlotFn a_slot, cudaStream_t st) {
    const Plan &P = ctx->plan;
    a.u = cur;
    a.un = nxt;
    a.dd = dcur;
    a.n = n;
    a.a_out = a_slot(n);
    int rc;
    if (blocking && n + 1 < n_end) {
        a.dd_out = dnxt;
        a.a_out2 = a.a_out ? a_slot(n + 1) : nullptr;
        TileMaps M;
        if ((rc = pair_maps(ctx, a, &M))) return rc;
        launch_fwd_pair(a, active_tiles(P, n), M, st);
        ctx->stats.kernel_launches++;
        ctx->stats.cell_updates += active_cells(P, n, ctx->NZ) + active_cells(P, n + 1, ctx->NZ);
        std::swap(cur, nxt);
        std::swap(dcur, dnxt);
        return 2;
    }
    a.dd_out = a.a_out2 = nullptr;
    if ((rc = fwd_step(ctx, a, active_tiles(P, n), L, st))) return rc;
    ctx->stats.kernel_launches++;
    ctx->stats.cell_updates += active_cells(P, n, ctx->NZ);
    std::swap(cur, nxt);
    return 1;
}

// Forward pass over all steps.  State pools uA (u^0), uB (scratch), dd
// (D^0) and dd2 (scratch) must be zeroed by the caller.  d (nullable)
// receives samples.  With backward set (workspace from ensure_backward_ws)
// the pass also stores a^n of the steps kept in the history and, at the
// start of every other segment of K steps, the checkpoint (u^n, D^n).
int run_forward(dhfwi_ctx *ctx, float *uA, float *uB, float *dd, float *dd2, float *d, bool backward,
                cudaStream_t st) {
    const Plan &P = ctx->plan;
    FwdArgs a{};
    a.c = common(ctx);
    a.d = d;
    float *cur = uA, *nxt = uB, *dcur = dd, *dnxt = dd2;
    const long long pool = P.pool_floats;
    const bool blocking = time_blocking(ctx, 0);
    const int K = ctx->ck_every, S = backward ? ctx->hist_segs : 0;
    const int H = std::min(S * K, P.nt_max);  // steps whose a^n are stored
    float *ck = (float *)ctx->ck.p, *hist = (float *)ctx->hist.p;
    auto slot = [&](int n) -> float * { return n < H ? hist + ctx->hoff[n] : nullptr; };
    const long long l0 = ctx->stats.kernel_launches, c0 = ctx->stats.cell_updates;
    if (backward) ctx->fws.valid = false;  // the history and checkpoints are about to change
    phase_begin(ctx, 0, st);
    for (int n = 0; n < P.nt_max;) {
        // K and H are even and two-step launches start at even n: a launch
        // never straddles a segment or the end of the history.
        if (backward && n >= H && n % K == 0) {
            const long long j = n / K - S;
            a.ck_u = ck + (2 * j) * pool;
            a.ck_d = ck + (2 * j + 1) * pool;
        } else {
            a.ck_u = a.ck_d = nullptr;
        }
        const long long cn = ctx->stats.cell_updates;
        const int rc = forward_steps(ctx, a, n, P.nt_max, cur, nxt, dcur, dnxt, ctx->launch[n < H ? 1 : 0], blocking,
                                     slot, st);
        if (rc < 0) return rc;
        if (n < H) ctx->stats.history_cells += ctx->stats.cell_updates - cn;
        n += rc;
    }
    if (backward) {
        ctx->stats.history_steps = H;
        ctx->fws.valid = true;
        ctx->fws.plan = P.hash;
        ctx->fws.model = ctx->model_hash;
        ctx->fws.segs = ctx->hist_segs;
        ctx->fws.K = ctx->ck_every;
    }
    phase_end(ctx, 0, st, ctx->stats.kernel_launches - l0, ctx->stats.cell_updates - c0);
    CK(cudaGetLastError());
    return DHFWI_OK;
}

// True when the last backward-capable forward pass ran at this plan and
// model (its a^n history and checkpoints intact) and reuse is on.
bool forward_reusable(const dhfwi_ctx *ctx) {
    return ctx->reuse && ctx->fws.valid && ctx->fws.plan == ctx->plan.hash && ctx->fws.model == ctx->model_hash &&
           ctx->fws.segs == ctx->hist_segs && ctx->fws.K == ctx->ck_every;
}

// Backward sweep, segment by segment from the last: a^n of a segment comes
// from the history, or is recomputed from the segment's checkpoint (u and D
// start in the checkpoint pools and alternate with the work pools w and w2)
// into the segment buffer; then the adjoint steps over it with the data r
// injected, the image accumulated in gpool.  Adjoint state pools nuA, nuB,
// nud, nud2 must be zeroed by the caller; with time blocking the adjoint
// also advances two steps per launch.  With reuse on, a recomputed segment
// starts from copies of its checkpoint in w3 and w4 (the recompute then
// alternates w3 / w and w4 / w2), so that the checkpoints stay intact for a
// later call that reuses this forward pass; without it the recompute
// overwrites them and the forward pass can no longer be reused.
int run_backward(dhfwi_ctx *ctx, float *w, float *w2, float *w3, float *w4, float *nuA, float *nuB, float *nud,
                 float *nud2, float *gpool, const float *r, cudaStream_t st) {
    const Plan &P = ctx->plan;
    const long long pool = P.pool_floats;
    const int K = ctx->ck_every, S = ctx->hist_segs;
    const int nseg = (P.nt_max + K - 1) / K;
    const bool blocking = time_blocking(ctx, 0), blocking_adj = time_blocking(ctx, 1);
    float *ck = (float *)ctx->ck.p, *abuf = (float *)ctx->abuf.p, *hist = (float *)ctx->hist.p;
    FwdArgs f{};
    f.c = common(ctx);
    AdjArgs b{};
    b.c = f.c;
    b.r = r;
    b.g = gpool;
    float *ncur = nuA, *nnxt = nuB, *dcur_nu = nud, *dnxt_nu = nud2;
    const long long l0 = ctx->stats.kernel_launches, c0 = ctx->stats.cell_updates;
    phase_begin(ctx, 1, st);
    for (int js = nseg - 1; js >= 0; js--) {
        const int n0 = js * K, n1 = std::min(n0 + K, P.nt_max);
        const bool stored = js < S;
        auto slot = [&](int n) -> float * {
            return stored ? hist + ctx->hoff[n] : abuf + (long long)(n - n0) * pool;
        };
        if (!stored) {
            float *cur = ck + (2 * (long long)(js - S)) * pool, *nxt = w;
            float *dcur = ck + (2 * (long long)(js - S) + 1) * pool, *dnxt = w2;
            if (ctx->reuse) {
                CK(cudaMemcpyAsync(w3, cur, sizeof(float) * (size_t)pool, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(w4, dcur, sizeof(float) * (size_t)pool, cudaMemcpyDeviceToDevice, st));
                cur = w3;
                dcur = w4;
            } else {
                ctx->fws.valid = false;
            }
            f.d = nullptr;
            f.ck_u = f.ck_d = nullptr;
            for (int n = n0; n < n1;) {
                const int rc = forward_steps(ctx, f, n, n1, cur, nxt, dcur, dnxt, ctx->launch[1], blocking, slot, st);
                if (rc < 0) return rc;
                n += rc;
            }
        }
        for (int k = n1; k >= n0 + 1;) {
            b.nu = ncur;
            b.nun = nnxt;
            b.dd = dcur_nu;
            b.a = slot(k - 1);
            b.k = k;
            if (blocking_adj && k - 1 >= n0 + 1) {
                // Steps k and k-1: the data of step k go into D_nu first (in
                // the kernel's staged tiles, or by the separate pass when a
                // tile's grown region holds too many receivers).
                b.inject_here = P.xinj ? 1 : 0;
                const int nrt = P.xinj ? 0 : P.rtiles_prefix[active_slots(P, k - 1)];
                launch_adj_inject(b, (const int *)P.d_rtiles.p, nrt, st);
                b.dd_out = dnxt_nu;
                b.a2 = slot(k - 2);
                TileMaps M;
                int rc = adj_pair_maps(ctx, b, &M);
                if (rc) return rc;
                launch_adj_pair(b, active_tiles(P, k - 2), M, st);
                ctx->stats.kernel_launches += 1 + (nrt > 0);
                ctx->stats.cell_updates += active_cells(P, k - 1, ctx->NZ) + active_cells(P, k - 2, ctx->NZ);
                std::swap(ncur, nnxt);
                std::swap(dcur_nu, dnxt_nu);
                k -= 2;
                continue;
            }
            b.dd_out = nullptr;
            b.a2 = nullptr;
            int rc = adj_step(ctx, b, active_tiles(P, k - 1), ctx->launch[2], st);
            if (rc) return rc;
            ctx->stats.kernel_launches++;
            ctx->stats.cell_updates += active_cells(P, k - 1, ctx->NZ);
            std::swap(ncur, nnxt);
            k--;
        }
        CK(cudaGetLastError());
    }
    phase_end(ctx, 1, st, ctx->stats.kernel_launches - l0, ctx->stats.cell_updates - c0);
    return DHFWI_OK;
}

// Cap on the stored history in bytes from DHFWI_HISTORY_MB (MiB): -1 when
// unset (as much as device memory allows), 0 for none.
long long history_limit() {
    const char *e = std::getenv("DHFWI_HISTORY_MB");
    if (!e || !*e) return -1;
    const long long mb = std::atoll(e);
    return mb < 0 ? -1 : mb << 20;
}

// Workspace for a backward-capable pass: the field pools; the history of
// a^n for the first S segments of K steps (K even) and, for the other
// segments, a checkpoint pair each plus the K-slot segment buffer.  The
// history trades memory for the recompute of those segments: it holds the
// active slots of each step only (sum over shots of nt x NZ x pitch floats,
// plus one pool so that a tensor map over any step stays inside it).  S is
// as large as DHFWI_HISTORY_MB allows, else as device memory allows with
// max(16 GiB, 1/16 of the device) left free; chosen once per plan.
int ensure_backward_ws_impl(dhfwi_ctx *ctx);

// The workspace of ensure_backward_ws_impl; a change of the history or
// checkpoint buffers (reallocated, or a new split) ends the reuse of the
// forward pass stored in them.
int ensure_backward_ws(dhfwi_ctx *ctx) {
    const void *h0 = ctx->hist.p, *c0 = ctx->ck.p;
    const int s0 = ctx->hist_segs, k0 = ctx->ck_every;
    const int rc = ensure_backward_ws_impl(ctx);
    if (rc || ctx->hist.p != h0 || ctx->ck.p != c0 || ctx->hist_segs != s0 || ctx->ck_every != k0)
        ctx->fws.valid = false;
    return rc;
}

int ensure_backward_ws_impl(dhfwi_ctx *ctx) {
    const Plan &P = ctx->plan;
    const size_t pool = sizeof(float) * (size_t)P.pool_floats;
    int rc = ensure(ctx, ctx->fields, NPOOLS * pool, "wavefield pools");
    if (rc) return rc;
    const long long limit = history_limit();
    if (ctx->hist_plan != P.hash || ctx->hist_limit != limit) {
        const int K = ctx->ck_every;
        const int nseg = (P.nt_max + K - 1) / K;
        const size_t slot = sizeof(float) * (size_t)ctx->NZ * P.pitch;
        std::vector<size_t> seg(nseg, 0);
        for (int n = 0; n < P.nt_max; n++) seg[n / K] += (size_t)active_slots(P, n) * slot;
        release(ctx->hist);
        size_t avail;
        if (limit >= 0) {
            avail = (size_t)limit;
        } else {
            release(ctx->ck);
            release(ctx->abuf);
            size_t fr = 0, tot = 0;
            CK(cudaMemGetInfo(&fr, &tot));
            const size_t reserve = std::max<size_t>(16ull << 30, tot / 16);
            avail = fr > reserve ? fr - reserve : 0;
        }
        // Largest S whose history (and, in the automatic case, the
        // checkpoints and segment buffer of the rest) fits.
        int S = 0;
        size_t h = pool;
        for (int t = 1; t <= nseg; t++) {
            h += seg[t - 1];
            const size_t rest = t < nseg ? (2 * (size_t)(nseg - t) + (size_t)std::min(K, P.nt_max)) * pool : 0;
            if (h + (limit >= 0 ? 0 : rest) <= avail) S = t;
        }
        if (S > 0) {
            size_t hb = pool;
            for (int t = 0; t < S; t++) hb += seg[t];
            if (ensure(ctx, ctx->hist, hb, "wavefield history") != DHFWI_OK) {
                ctx->err.clear();
                S = 0;
            }
        }
        ctx->hist_segs = S;
        ctx->hoff.assign((size_t)std::min(S * K, P.nt_max), 0);
        long long off = 0;
        for (size_t n = 0; n < ctx->hoff.size(); n++) {
            ctx->hoff[n] = off;
            off += (long long)active_slots(P, (int)n) * ctx->NZ * P.pitch;
        }
        ctx->hist_plan = P.hash;
        ctx->hist_limit = limit;
    }
    // Checkpoints and segment buffer of the recomputed segments.  Out of
    // memory: drop the history first, then fall back to ~sqrt(2 nt)
    // segments, which minimises 2 nt/K + K.
    for (int attempt = 0; attempt < 3; attempt++) {
        const int K = ctx->ck_every, S = ctx->hist_segs;
        const int nseg = (P.nt_max + K - 1) / K;
        if (S >= nseg) {
            release(ctx->ck);
            release(ctx->abuf);
            return DHFWI_OK;
        }
        rc = ensure(ctx, ctx->ck, 2 * (size_t)(nseg - S) * pool, "checkpoints");
        if (!rc) rc = ensure(ctx, ctx->abuf, (size_t)std::min(K, P.nt_max) * pool, "segment buffer");
        if (rc != DHFWI_ERR_OOM) return rc;
        release(ctx->ck);
        release(ctx->abuf);
        if (attempt == 2) break;
        ctx->err.clear();
        if (S > 0) {
            release(ctx->hist);
            ctx->hist_segs = 0;
            ctx->hoff.clear();
        } else {
            int K2 = std::max(K, (int)std::ceil(std::sqrt(2.0 * P.nt_max)));
            K2 += K2 & 1;  // checkpoints at even steps: a two-step launch never straddles one
            ctx->ck_every = K2;
        }
    }
    return rc;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int dhfwi_create(dhfwi_ctx **out, const dhfwi_grid *g, int device) {
    g_create_error.clear();
    if (!out || !g) {
        g_create_error = "out and g must not be NULL";
        return DHFWI_ERR_ARG;
    }
    *out = nullptr;
    if (g->nz < 1 || g->nx < 1 || g->nb < 0 || g->nb > 64 || !(g->h > 0.f) || !(g->dt > 0.f) ||
        !std::isfinite(g->h) || !std::isfinite(g->dt)) {
        g_create_error = "bad grid: need nz, nx >= 1, 0 <= nb <= 64, finite h, dt > 0";
        return DHFWI_ERR_ARG;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = std::string("no such CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "index");
        cudaGetLastError();
        return DHFWI_ERR_CUDA;
    }
    if ((e = cudaSetDevice(device)) != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        return DHFWI_ERR_CUDA;
    }
    dhfwi_ctx *ctx = new (std::nothrow) dhfwi_ctx();
    if (!ctx) {
        g_create_error = "host allocation failed";
        return DHFWI_ERR_OOM;
    }
    ctx->device = device;
    ctx->g = *g;
    ctx->NZ = g->nz + 2 * g->nb;
    ctx->NXF = g->nx + 2 * g->nb;
    ctx->pf = round_up(ctx->NXF + 4, 32);
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    cudaGetLastError();
    for (int k = 0; k < 4; k++) set_variant(ctx, k, 1);
    if (ensure(ctx, ctx->status, 64, "status") || ensure(ctx, ctx->partial, sizeof(double) * RESID_BLOCKS, "partials") ||
        cudaMallocHost(&ctx->h_status, 64) != cudaSuccess ||
        cudaMallocHost(&ctx->h_partial, sizeof(double) * RESID_BLOCKS) != cudaSuccess) {
        g_create_error = ctx->err.empty() ? "pinned allocation failed" : ctx->err;
        dhfwi_destroy(ctx);
        return DHFWI_ERR_OOM;
    }
    *out = ctx;
    return DHFWI_OK;
}

void dhfwi_destroy(dhfwi_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    DevBuf *bufs[] = {&ctx->kap, &ctx->dkap, &ctx->status, &ctx->partial, &ctx->fields,
                      &ctx->ck, &ctx->abuf, &ctx->hist, &ctx->dtmp, &ctx->rtmp, &ctx->plan.d_shots, &ctx->plan.d_tiles,
                      &ctx->plan.d_recs, &ctx->plan.d_slot_of, &ctx->plan.d_wav, &ctx->plan.d_infos,
                      &ctx->plan.d_rtiles, &ctx->plan.d_xrecs, &ctx->plan.d_xrec_off};
    for (DevBuf *b : bufs) release(*b);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_partial) cudaFreeHost(ctx->h_partial);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 2; j++)
            if (ctx->ev[i][j]) cudaEventDestroy(ctx->ev[i][j]);
    dhfwi::net_destroy(ctx->net);
    delete ctx;
}

const char *dhfwi_last_error(const dhfwi_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

int dhfwi_stats(const dhfwi_ctx *ctx, dhfwi_stats_t *out) {
    if (!ctx || !out) return DHFWI_ERR_ARG;
    *out = ctx->stats;
    for (int i = 0; i < 3; i++) {
        out->phase_ms[i] = 0.0;
        if (ctx->timing && ctx->ev_used[i]) {
            float ms = 0.f;
            if (cudaEventSynchronize(ctx->ev[i][1]) == cudaSuccess &&
                cudaEventElapsedTime(&ms, ctx->ev[i][0], ctx->ev[i][1]) == cudaSuccess)
                out->phase_ms[i] = ms;
            cudaGetLastError();
        }
    }
    return DHFWI_OK;
}

int dhfwi_set_timing(dhfwi_ctx *ctx, int on) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx->timing = on != 0;
    return DHFWI_OK;
}

int dhfwi_set_reuse(dhfwi_ctx *ctx, int on) {
    if (!ctx) return DHFWI_ERR_ARG;
    ctx->reuse = on != 0;
    if (!ctx->reuse) ctx->fws.valid = false;
    return DHFWI_OK;
}

int model_shots(dhfwi_ctx *ctx, const float *v_dev, const dhfwi_geom *geom, float *d_dev, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!d_dev) return fail(ctx, DHFWI_ERR_ARG, "d_dev is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = get_plan(ctx, geom))) return rc;
    if ((rc = prep_model(ctx, v_dev, nullptr, 0, st))) return rc;
    if ((rc = autotune(ctx, st))) return rc;
    const size_t pool = sizeof(float) * (size_t)ctx->plan.pool_floats;
    if ((rc = ensure(ctx, ctx->fields, NPOOLS * pool, "wavefield pools"))) return rc;
    float *uA = (float *)ctx->fields.p, *uB = uA + ctx->plan.pool_floats, *ud = uB + ctx->plan.pool_floats;
    float *ud2 = ud + ctx->plan.pool_floats;
    CK(cudaMemsetAsync(uA, 0, 4 * pool, st));
    if ((rc = run_forward(ctx, uA, uB, ud, ud2, d_dev, false, st))) return rc;
    return end_call(ctx);
}

int fwi_gradient(dhfwi_ctx *ctx, const float *v_dev, const dhfwi_geom *geom, const float *d_obs_dev,
                 float *grad_dev, double *misfit_out, float *d_syn_dev, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!d_obs_dev || !grad_dev) return fail(ctx, DHFWI_ERR_ARG, "d_obs_dev and grad_dev must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = get_plan(ctx, geom))) return rc;
    if ((rc = prep_model(ctx, v_dev, nullptr, 0, st))) return rc;
    if ((rc = autotune(ctx, st))) return rc;
    const Plan &P = ctx->plan;
    if ((rc = ensure_backward_ws(ctx))) return rc;
    const size_t nd = (size_t)P.n_data;
    if ((rc = ensure(ctx, ctx->rtmp, sizeof(float) * std::max<size_t>(nd, 1), "residual"))) return rc;
    float *dsyn = d_syn_dev;
    if (!dsyn) {
        if ((rc = ensure(ctx, ctx->dtmp, sizeof(float) * std::max<size_t>(nd, 1), "synthetic data"))) return rc;
        dsyn = (float *)ctx->dtmp.p;
    }
    const long long pool = P.pool_floats;
    float *F = (float *)ctx->fields.p;
    float *uA = F, *uB = F + pool, *ud = F + 2 * pool;
    float *nuA = F + 3 * pool, *nuB = F + 4 * pool, *nud = F + 5 * pool, *gp = F + 6 * pool;
    CK(cudaMemsetAsync(F, 0, sizeof(float) * NPOOLS * (size_t)pool, st));
    // Checkpoints are staged back as halo tiles: their padding columns, which
    // no kernel writes, must read as zero.
    if (ctx->ck.p) CK(cudaMemsetAsync(ctx->ck.p, 0, ctx->ck.bytes, st));
    if ((rc = run_forward(ctx, uA, uB, ud, F + 7 * pool, dsyn, true, st))) return rc;
    float *r = (float *)ctx->rtmp.p;
    launch_residual(dsyn, d_obs_dev, r, (long long)nd, (double *)ctx->partial.p, RESID_BLOCKS, st);
    ctx->stats.kernel_launches++;
    if ((rc = run_backward(ctx, uA, uB, ud, F + 7 * pool, nuA, nuB, nud, F + 8 * pool, gp, r, st)))
        return rc;
    launch_reduce_image((const ShotDesc *)P.d_shots.p, (const int *)P.d_slot_of.p, P.n_shots, gp, ctx->g.nz,
                        ctx->g.nx, ctx->g.nb, v_dev, 0, grad_dev, st);
    ctx->stats.kernel_launches++;
    CK(cudaGetLastError());
    if (misfit_out) {
        CK(cudaMemcpyAsync(ctx->h_partial, ctx->partial.p, sizeof(double) * RESID_BLOCKS, cudaMemcpyDeviceToHost, st));
        if ((rc = sync_and_check_timeout(ctx, st))) return rc;
        double J = 0.0;
        for (int i = 0; i < RESID_BLOCKS; i++) J += ctx->h_partial[i];
        J *= 0.5;
        if (!std::isfinite(J)) return fail(ctx, DHFWI_ERR_NONFINITE, "misfit is not finite");
        *misfit_out = J;
    }
    return end_call(ctx);
}

int born_demig(dhfwi_ctx *ctx, const float *v0_dev, const dhfwi_geom *geom, const float *dv_dev, float *d_dev,
               int flags, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!dv_dev || !d_dev) return fail(ctx, DHFWI_ERR_ARG, "dv_dev and d_dev must not be NULL");
    if (flags != DHFWI_ABS && flags != DHFWI_REL) return fail(ctx, DHFWI_ERR_ARG, "flags must be DHFWI_ABS or DHFWI_REL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = get_plan(ctx, geom))) return rc;
    if ((rc = prep_model(ctx, v0_dev, dv_dev, flags == DHFWI_REL, st))) return rc;
    if ((rc = autotune(ctx, st))) return rc;
    const Plan &P = ctx->plan;
    const long long pool = P.pool_floats;
    if ((rc = ensure(ctx, ctx->fields, NPOOLS * sizeof(float) * (size_t)pool, "wavefield pools"))) return rc;
    float *F = (float *)ctx->fields.p;
    CK(cudaMemsetAsync(F, 0, sizeof(float) * 6 * (size_t)pool, st));
    BornArgs a{};
    a.c = common(ctx);
    a.dkap = (const float *)ctx->dkap.p;
    a.d = d_dev;
    float *u = F, *un = F + pool, *p = F + 2 * pool, *pn = F + 3 * pool;
    a.du = F + 4 * pool;
    a.dp = F + 5 * pool;
    const long long l0 = ctx->stats.kernel_launches, c0 = ctx->stats.cell_updates;
    phase_begin(ctx, 2, st);
    // Background from the stored forward pass at this model (every step of
    // it in the history, TMA available): only the scattered field advances.
    if (forward_reusable(ctx) && (long long)ctx->hist_segs * ctx->ck_every >= P.nt_max && encode_tiled()) {
        float *hist = (float *)ctx->hist.p;
        for (int n = 0; n < P.nt_max; n++) {
            a.p = p;
            a.pn = pn;
            a.n = n;
            a.a = hist + ctx->hoff[n];
            TileMaps M;
            if ((rc = tensor_map(ctx, a.p, MAP_POOL_HALO, &M.m[0])) || (rc = tensor_map(ctx, a.dp, MAP_POOL_CELL, &M.m[1])) ||
                (rc = tensor_map(ctx, a.c.kap, MAP_MODEL, &M.m[2])) || (rc = tensor_map(ctx, a.dkap, MAP_MODEL, &M.m[3])) ||
                (rc = tensor_map(ctx, a.a, MAP_POOL_CELL, &M.m[4])))
                return rc;
            launch_born_hist_step(a, active_tiles(P, n), M, st);
            ctx->stats.kernel_launches++;
            ctx->stats.cell_updates += active_cells(P, n, ctx->NZ);
            std::swap(p, pn);
        }
        ctx->stats.reused |= 2;
        phase_end(ctx, 2, st, ctx->stats.kernel_launches - l0, ctx->stats.cell_updates - c0);
        return end_call(ctx);
    }
    for (int n = 0; n < P.nt_max; n++) {
        a.u = u;
        a.un = un;
        a.p = p;
        a.pn = pn;
        a.n = n;
        if ((rc = born_step(ctx, a, active_tiles(P, n), ctx->launch[3], st))) return rc;
        ctx->stats.kernel_launches++;
        ctx->stats.cell_updates += 2 * active_cells(P, n, ctx->NZ);
        std::swap(u, un);
        std::swap(p, pn);
    }
    phase_end(ctx, 2, st, ctx->stats.kernel_launches - l0, ctx->stats.cell_updates - c0);
    return end_call(ctx);
}

int rtm_mig(dhfwi_ctx *ctx, const float *v0_dev, const dhfwi_geom *geom, const float *d_dev, float *img_dev,
            int flags, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!d_dev || !img_dev) return fail(ctx, DHFWI_ERR_ARG, "d_dev and img_dev must not be NULL");
    if (flags != DHFWI_ABS && flags != DHFWI_REL) return fail(ctx, DHFWI_ERR_ARG, "flags must be DHFWI_ABS or DHFWI_REL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = get_plan(ctx, geom))) return rc;
    if ((rc = prep_model(ctx, v0_dev, nullptr, 0, st))) return rc;
    if ((rc = autotune(ctx, st))) return rc;
    const Plan &P = ctx->plan;
    if ((rc = ensure_backward_ws(ctx))) return rc;
    const long long pool = P.pool_floats;
    float *F = (float *)ctx->fields.p;
    float *uA = F, *uB = F + pool, *ud = F + 2 * pool;
    float *nuA = F + 3 * pool, *nuB = F + 4 * pool, *nud = F + 5 * pool, *gp = F + 6 * pool;
    if (forward_reusable(ctx)) {
        // The forward pass stored at this model and geometry is still intact:
        // only the adjoint state and the image start from zero.
        CK(cudaMemsetAsync(nuA, 0, sizeof(float) * 6 * (size_t)pool, st));
        ctx->stats.reused |= 1;
    } else {
        CK(cudaMemsetAsync(F, 0, sizeof(float) * NPOOLS * (size_t)pool, st));
        // Checkpoints are staged back as halo tiles: their padding columns, which
        // no kernel writes, must read as zero.
        if (ctx->ck.p) CK(cudaMemsetAsync(ctx->ck.p, 0, ctx->ck.bytes, st));
        if ((rc = run_forward(ctx, uA, uB, ud, F + 7 * pool, nullptr, true, st))) return rc;
    }
    if ((rc = run_backward(ctx, uA, uB, ud, F + 7 * pool, nuA, nuB, nud, F + 8 * pool, gp, d_dev, st)))
        return rc;
    launch_reduce_image((const ShotDesc *)P.d_shots.p, (const int *)P.d_slot_of.p, P.n_shots, gp, ctx->g.nz,
                        ctx->g.nx, ctx->g.nb, v0_dev, flags == DHFWI_REL, img_dev, st);
    ctx->stats.kernel_launches++;
    return end_call(ctx);
}

int fwi_update(dhfwi_ctx *ctx, const float *v_dev, const float *dir_dev, float alpha, float vmin, float vmax,
               int mute_rows, float *v_out_dev, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!v_dev || !dir_dev || !v_out_dev) return fail(ctx, DHFWI_ERR_ARG, "NULL model pointer");
    if (!(vmin > 0.f) || !(vmax >= vmin) || !std::isfinite(alpha) || mute_rows < 0)
        return fail(ctx, DHFWI_ERR_ARG, "need 0 < vmin <= vmax, finite alpha, mute_rows >= 0");
    launch_update_model(v_dev, dir_dev, ctx->g.nz, ctx->g.nx, std::min(mute_rows, ctx->g.nz), alpha, vmin, vmax,
                        (unsigned *)ctx->status.p + 2, v_out_dev, (cudaStream_t)stream);
    ctx->stats.kernel_launches += 2;
    return end_call(ctx);
}

int bb_step(dhfwi_ctx *ctx, const float *x_k, const float *x_prev, const float *g_k, const float *g_prev,
            int mute_rows, double *alpha_out, double *gmax_out, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!x_k || !x_prev || !g_k || !g_prev || !alpha_out || mute_rows < 0)
        return fail(ctx, DHFWI_ERR_ARG, "NULL pointer or negative mute_rows");
    cudaStream_t st = (cudaStream_t)stream;
    const long long off = (long long)std::min(mute_rows, ctx->g.nz) * ctx->g.nx;
    const long long n = (long long)ctx->g.nz * ctx->g.nx - off;
    constexpr int NB = RESID_BLOCKS / 2;  // two sums per block in the partial buffer
    launch_bb_partials(x_k + off, x_prev + off, g_k + off, g_prev + off, n, (double *)ctx->partial.p, NB,
                       (unsigned *)ctx->status.p + 2, st);
    ctx->stats.kernel_launches += 2;
    CK(cudaMemcpyAsync(ctx->h_partial, ctx->partial.p, sizeof(double) * 2 * NB, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_status + 2, (unsigned *)ctx->status.p + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       st));
    if ((rc = sync_and_check_timeout(ctx, st))) return rc;
    double sxg = 0.0, sgg = 0.0;
    for (int i = 0; i < NB; i++) {
        sxg += ctx->h_partial[2 * i];
        sgg += ctx->h_partial[2 * i + 1];
    }
    if (!(sgg > 0.0) || !std::isfinite(sxg) || !std::isfinite(sgg))
        return fail(ctx, DHFWI_ERR_NONFINITE, "the gradient difference is zero or not finite");
    *alpha_out = sxg / sgg;
    if (gmax_out) {
        float gm;
        std::memcpy(&gm, &ctx->h_status[2], sizeof gm);
        *gmax_out = gm;
    }
    return end_call(ctx);
}

int dhfwi_selftest_timeout(dhfwi_ctx *ctx, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    launch_wait_timeout_selftest((unsigned *)ctx->status.p + TFLAG_WORD, (cudaStream_t)stream);
    ctx->stats.kernel_launches++;
    return end_call(ctx);
}

int image_laplacian(dhfwi_ctx *ctx, const float *img_dev, float *out_dev, void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!img_dev || !out_dev) return fail(ctx, DHFWI_ERR_ARG, "NULL image pointer");
    if (img_dev == out_dev) return fail(ctx, DHFWI_ERR_ARG, "out must not alias img");
    launch_image_laplacian(img_dev, ctx->g.nz, ctx->g.nx, ctx->g.h, out_dev, (cudaStream_t)stream);
    ctx->stats.kernel_launches++;
    return end_call(ctx);
}

int data_misfit(dhfwi_ctx *ctx, const float *a_dev, const float *b_dev, long long n, double *misfit_out,
                void *stream) {
    int rc = begin_call(ctx);
    if (rc) return rc;
    if (!a_dev || !b_dev || !misfit_out || n < 0) return fail(ctx, DHFWI_ERR_ARG, "bad misfit arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure(ctx, ctx->rtmp, sizeof(float) * std::max<long long>(n, 1), "residual"))) return rc;
    launch_residual(a_dev, b_dev, (float *)ctx->rtmp.p, n, (double *)ctx->partial.p, RESID_BLOCKS, st);
    ctx->stats.kernel_launches++;
    CK(cudaMemcpyAsync(ctx->h_partial, ctx->partial.p, sizeof(double) * RESID_BLOCKS, cudaMemcpyDeviceToHost, st));
    if ((rc = sync_and_check_timeout(ctx, st))) return rc;
    double J = 0.0;
    for (int i = 0; i < RESID_BLOCKS; i++) J += ctx->h_partial[i];
    *misfit_out = 0.5 * J;
    return end_call(ctx);
}

}  // extern "C"

// Accessors used by the network code in the same library.
namespace dhfwi {
NetState *&ctx_net(dhfwi_ctx *ctx) { return ctx->net; }
int ctx_device(dhfwi_ctx *ctx) { return ctx->device; }
void ctx_set_error(dhfwi_ctx *ctx, const char *msg) { ctx->err = msg; }
void ctx_begin(dhfwi_ctx *ctx) {
    ctx->err.clear();
    ctx->stats.kernel_launches = 0;
    ctx->stats.cell_updates = 0;
}
void ctx_count_launches(dhfwi_ctx *ctx, long long n) { ctx->stats.kernel_launches += n; }
}  // namespace dhfwi
