// Internal declarations shared by the host orchestration (api.cu) and the
// finite-difference kernels (fd_kernels.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dhfwi {

// Stencil tile handled by one CTA: TZ rows x TX columns of one shot window.
constexpr int TX = 64;
constexpr int TZ = 32;
constexpr int HALO = 4;          // radius of the 8th-order stencil
constexpr int NTHR_X = 64;       // threads per CTA along x (one column each)
constexpr int NTHR_Z = 4;        // threads per CTA along z
constexpr int ROWS_PER_THR = TZ / NTHR_Z;
constexpr int SROW = TX + 2 * HALO;   // shared-memory row length (floats)
constexpr int SROWS = TZ + 2 * HALO;

// Per-shot descriptor, indexed by "slot" (shots sorted by record length,
// longest first, so that the shots still running at step n are a prefix).
struct ShotDesc {
    long long foff;   // offset (floats) of this shot's window inside a field pool
    long long doff;   // offset of this shot's block in the packed data vector
    int nxw;          // padded window width (cells) = win_x1 - win_x0 + 2 nb
    int pitch;        // row pitch of the window in a field pool (floats)
    int x0;           // padded-model column of the window's column 0 (= win_x0)
    int sz, sx;       // source node, padded window coordinates
    int nt;           // record length
    int nrec;         // receivers of this shot
    int wav_off;      // offset of this shot's wavelet in the wavelet array
    int shot;         // original shot index
};

// One CTA work item: tile origin inside a shot window.
struct Tile {
    int slot;
    int z0, x0;
    int rec_begin;    // first receiver entry of this tile (entries are [rec_begin, next tile's))
};

// A receiver that falls inside a tile.
struct TileRec {
    int cell;         // (lz * TX + lx) inside the tile
    int r;            // receiver index within its shot
};

struct StepCommon {
    const ShotDesc *shots;
    const Tile *tiles;
    const TileRec *recs;
    const float *kap;     // [NZ][pf] padded model, kappa = v^2 dt^2/h^2
    const float *vpad;    // [NZ][pf] padded model velocity
    const float *wav;     // wavelets
    int pf;               // pitch of the padded model arrays
    int NZ;               // padded rows = nz + 2 nb
    int nb;
};

// Forward step n over the active tiles (grid = number of active tiles).
struct FwdArgs {
    StepCommon c;
    const float *u;   // pool: u^n
    float *uo;        // pool: u^{n-1}, overwritten with u^{n+1}
    float *ck_old;    // nullable: store u^{n-1} here (checkpoint)
    float *ck_cur;    // nullable: store u^n here (checkpoint)
    float *a_out;     // nullable: store a^n = D u^n + q^n here (segment buffer slot)
    float *d;         // nullable: packed records, sample n written from u^{n+1}
    int n;
};

// Adjoint step k (scaled field nu = kappa w lambda, which obeys the forward
// recurrence with the data injected like the source).
struct AdjArgs {
    StepCommon c;
    const float *nu;      // pool: nu^{k+1}
    float *nuo;           // pool: nu^{k+2}, overwritten with nu^k
    const float *r;       // packed data injected at the receivers (sample k-1)
    const float *a;       // pool: a^{k-1} of the background forward field
    float *g;             // pool: per-shot image accumulator, += (2/v) a^{k-1} nu^k
    int k;
};

// Born joint step n: background u0 and scattered p advance together.
struct BornArgs {
    StepCommon c;
    const float *u;   float *uo;     // background pools (u0^n, u0^{n-1} -> u0^{n+1})
    const float *p;   float *po;     // scattered pools
    const float *dkap;               // [NZ][pf] padded d kappa = 2 kappa dv / v
    float *d;                        // packed Born records (sample n from p^{n+1})
    int n;
};

void launch_fwd_step(const FwdArgs &a, int ntiles, cudaStream_t s);
void launch_adj_step(const AdjArgs &a, int ntiles, cudaStream_t s);
void launch_born_step(const BornArgs &a, int ntiles, cudaStream_t s);

// Padded model preparation: kap, vpad (and dkap when dv != nullptr) from the
// physical [nz][nx] model; also checks v (finite, > 0) and records max kappa.
// status[0] |= 1 for a bad velocity; status[1] = bits of max kappa (float).
void launch_prep_model(const float *v, const float *dv, int rel, int nz, int nx, int nb, float c,
                       float *kap, float *vpad, float *dkap, int pf, unsigned *status,
                       cudaStream_t s);

// r = d_syn - d_obs, and per-block partial sums of r^2 (double).
void launch_residual(const float *ds, const float *dobs, float *r, long long n, double *partial,
                     int nblocks, cudaStream_t s);

// Sum of the per-shot image accumulators into the physical [nz][nx] grid,
// folding the sponge cells onto the edge cells they copy (transpose of the
// extension), shots in original order; rel != 0 multiplies by v.
void launch_reduce_image(const ShotDesc *shots, const int *slot_of_shot, int n_shots,
                         const float *gpool, int nz, int nx, int nb, const float *v, int rel,
                         float *out, cudaStream_t s);

}  // namespace dhfwi
