// Forward shot modelling for callers that cannot allocate device memory.
//
// Some callers run where cudaMalloc is off limits: code inside a host
// framework that owns every device allocation (a custom allocator or a
// memory-capped service), callbacks that must not synchronise the device the
// way cudaMalloc/cudaFree can, or processes whose allocation budget is
// already spent.  model_shots_static serves them: it computes exactly what
// model_shots computes, but every temporary buffer (padded model arrays,
// wavefield state, geometry tables) lives in one file-scope device array of
// fixed size that the library reserves when it is loaded.  The caller still
// passes the velocity model and the output buffer.
//
// Cost of the convenience: every GPU that loads this library holds the array
// (DHFWI_STATIC_SCRATCH_BYTES) until the process exits, problems larger than
// it are rejected, and all calls share it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/dhfwi.h"
#include "fd_internal.h"

using namespace dhfwi;

namespace {

constexpr size_t kScratchBytes = (size_t)DHFWI_STATIC_SCRATCH_BYTES;

// The scratch array.  Host code must not use its name as an address: the
// device address comes from cudaGetSymbolAddress, once per device.
__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

thread_local char g_err[256] = "";

int err(int code, const char *msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

// Device address of the scratch array on the current device (set-up on the
// first call per device, with that device current).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(DHFWI_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(DHFWI_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(DHFWI_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DHFWI_OK;
}

int round_up(long long a, long long m) { return (int)((a + m - 1) / m * m); }

// Bump allocator over the scratch array (offsets only; 256-byte aligned).
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

}  // namespace

extern "C" {

const char *model_shots_static_error(void) { return g_err; }

int model_shots_static(const dhfwi_grid *g, const float *v_dev, const dhfwi_geom *G, float *d_dev, void *stream) {
    g_err[0] = 0;
    if (!g || !G || !v_dev || !d_dev) return err(DHFWI_ERR_ARG, "NULL argument");
    if (g->nz < 1 || g->nx < 1 || g->nb < 0 || g->nb > 64 || !(g->h > 0.f) || !(g->dt > 0.f))
        return err(DHFWI_ERR_ARG, "bad grid");
    if (G->n_shots < 1 || G->nt_max < 1 || !G->src_iz || !G->src_ix || !G->nt || !G->rec_off || !G->win_x0 ||
        !G->win_x1 || !G->wavelet || G->rec_off[0] != 0)
        return err(DHFWI_ERR_ARG, "bad geometry arrays");
    const int ns = G->n_shots, nb = g->nb, NZ = g->nz + 2 * nb, NXF = g->nx + 2 * nb;
    if (G->rec_off[ns] > 0 && (!G->rec_iz || !G->rec_ix)) return err(DHFWI_ERR_ARG, "receiver arrays are NULL");
    for (int s = 0; s < ns; s++) {
        const int x0 = G->win_x0[s], x1 = G->win_x1[s];
        if (G->nt[s] < 1 || G->nt[s] > G->nt_max || G->rec_off[s + 1] < G->rec_off[s])
            return err(DHFWI_ERR_ARG, "bad record length or receiver offsets");
        if (x0 < 0 || x1 > g->nx || x1 <= x0) return err(DHFWI_ERR_GEOM, "window outside the grid");
        auto in = [&](int iz, int ix) { return iz >= 0 && iz < g->nz && ix >= x0 && ix < x1; };
        if (!in(G->src_iz[s], G->src_ix[s])) return err(DHFWI_ERR_GEOM, "source outside its window");
        for (int r = G->rec_off[s]; r < G->rec_off[s + 1]; r++)
            if (!in(G->rec_iz[r], G->rec_ix[r])) return err(DHFWI_ERR_GEOM, "receiver outside its window");
    }

    // Host tables: shots sorted by record length (longest first), tiles per
    // shot, receivers bucketed per tile (same layout the step kernels read).
    std::vector<int> order(ns);
    for (int s = 0; s < ns; s++) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return G->nt[a] > G->nt[b]; });
    std::vector<long long> doff(ns + 1, 0);
    for (int s = 0; s < ns; s++) doff[s + 1] = doff[s] + (long long)G->nt[s] * (G->rec_off[s + 1] - G->rec_off[s]);
    std::vector<ShotDesc> shots(ns);
    std::vector<Tile> tiles;
    std::vector<TileRec> recs;
    std::vector<int> prefix(ns + 1, 0), nt_sorted(ns);
    long long foff = 0;
    for (int k = 0; k < ns; k++) {
        const int s = order[k];
        ShotDesc &sd = shots[k];
        sd.nxw = G->win_x1[s] - G->win_x0[s] + 2 * nb;
        sd.pitch = round_up(sd.nxw, POOL_ALIGN);
        sd.foff = foff;
        foff += (long long)sd.pitch * NZ;
        sd.doff = doff[s];
        sd.x0 = G->win_x0[s];
        sd.sz = G->src_iz[s] + nb;
        sd.sx = G->src_ix[s] - G->win_x0[s] + nb;
        sd.nt = G->nt[s];
        sd.nrec = G->rec_off[s + 1] - G->rec_off[s];
        sd.wav_off = G->wavelet_shared ? 0 : s * G->nt_max;
        sd.shot = s;
        nt_sorted[k] = sd.nt;
        const int ntz = (NZ + TZ - 1) / TZ, ntx = (sd.nxw + TX - 1) / TX;
        std::vector<std::vector<TileRec>> bucket((size_t)ntz * ntx);
        for (int r = 0; r < sd.nrec; r++) {
            const int rz = G->rec_iz[G->rec_off[s] + r] + nb;
            const int rx = G->rec_ix[G->rec_off[s] + r] - sd.x0 + nb;
            bucket[(size_t)(rz / TZ) * ntx + rx / TX].push_back(TileRec{(rz % TZ) * TX + rx % TX, r});
        }
        for (int tz = 0; tz < ntz; tz++)
            for (int tx = 0; tx < ntx; tx++) {
                tiles.push_back(Tile{k, tz * TZ, tx * TX, (int)recs.size()});
                for (const TileRec &e : bucket[(size_t)tz * ntx + tx]) recs.push_back(e);
            }
        prefix[k + 1] = (int)tiles.size();
    }
    tiles.push_back(Tile{0, 0, 0, (int)recs.size()});
    const size_t nwav = (size_t)G->nt_max * (G->wavelet_shared ? 1 : ns);

    // Scratch layout.
    const int pf = round_up(NXF + 4, 32);
    const long long mstride = (long long)NZ * pf;
    Carve cv;
    const size_t o_kap = cv.take(sizeof(float) * 4 * mstride);
    const size_t o_status = cv.take(64);  // the model kernel's status words (0, 1 and the hash at 8-9)
    const size_t o_shots = cv.take(sizeof(ShotDesc) * shots.size());
    const size_t o_tiles = cv.take(sizeof(Tile) * tiles.size());
    const size_t o_recs = cv.take(sizeof(TileRec) * std::max<size_t>(recs.size(), 1));
    const size_t o_wav = cv.take(sizeof(float) * nwav);
    const size_t o_u = cv.take(sizeof(float) * 3 * (size_t)foff);
    if (cv.off > kScratchBytes) {
        char b[200];
        snprintf(b, sizeof b, "problem needs %.1f MiB of scratch, the static array holds %.1f MiB", cv.off / 1048576.0,
                 kScratchBytes / 1048576.0);
        return err(DHFWI_ERR_ARG, b);
    }
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    char *S = (char *)base;
    cudaStream_t st = (cudaStream_t)stream;
#define SCK(call)                                                            \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return err(DHFWI_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)
    // Copies from pageable host memory are staged before the call returns.
    SCK(cudaMemcpyAsync(S + o_shots, shots.data(), sizeof(ShotDesc) * shots.size(), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(S + o_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, st));
    if (!recs.empty())
        SCK(cudaMemcpyAsync(S + o_recs, recs.data(), sizeof(TileRec) * recs.size(), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(S + o_wav, G->wavelet, sizeof(float) * nwav, cudaMemcpyHostToDevice, st));
    // The array keeps the previous call's contents: clear the status words and
    // the wavefield state, which must start at zero.
    SCK(cudaMemsetAsync(S + o_status, 0, 64, st));
    SCK(cudaMemsetAsync(S + o_u, 0, sizeof(float) * 3 * (size_t)foff, st));
    const double c = ((double)g->dt * g->dt) / ((double)g->h * g->h);
    launch_prep_model(v_dev, nullptr, 0, g->nz, g->nx, nb, c, (float *)(S + o_kap), nullptr, pf, mstride,
                      (unsigned *)(S + o_status), st);
    SCK(cudaGetLastError());
    unsigned status[2] = {0, 0};
    SCK(cudaMemcpyAsync(status, S + o_status, sizeof status, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (status[0]) return err(DHFWI_ERR_NONFINITE, "velocity must be finite and > 0");
    float kmax;
    std::memcpy(&kmax, &status[1], sizeof kmax);
    const double Srad = 2.0 * (205.0 / 72.0 + 2.0 * (8.0 / 5.0 + 1.0 / 5.0 + 8.0 / 315.0 + 1.0 / 560.0));
    if ((double)kmax * Srad > 4.0) return err(DHFWI_ERR_CFL, "CFL violated");

    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    StepLaunch L;
    L.variant = 1;
    L.max_ctas = step_occupancy(0, L.variant, 0) * nsm;
    FwdArgs a{};
    a.c.shots = (const ShotDesc *)(S + o_shots);
    a.c.tiles = (const Tile *)(S + o_tiles);
    a.c.recs = (const TileRec *)(S + o_recs);
    a.c.kap = (const float *)(S + o_kap);
    a.c.mstride = mstride;
    a.c.wav = (const float *)(S + o_wav);
    a.c.pf = pf;
    a.c.NZ = NZ;
    a.c.nb = nb;
    float *U = (float *)(S + o_u);
    float *cur = U, *nxt = U + foff;
    a.dd = U + 2 * foff;
    a.d = d_dev;
    for (int n = 0; n < G->nt_max; n++) {
        // Shots with nt > n are the first m slots.
        int m = 0;
        while (m < ns && nt_sorted[m] > n) m++;
        a.u = cur;
        a.un = nxt;
        a.n = n;
        launch_fwd_step(a, prefix[m], L, nullptr, st);
        std::swap(cur, nxt);
    }
    SCK(cudaGetLastError());
#undef SCK
    return DHFWI_OK;
}

}  // extern "C"
