// Internal declarations shared by the host orchestration (api.cu) and the
// finite-difference kernels (fd_kernels.cu).  Not part of the C ABI.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; maps are encoded in api.cu)
#include <cuda_runtime.h>
#include <stdint.h>

namespace dhfwi {

// Stencil tile handled by one CTA: TZ rows x TX columns of one shot window.
// A CTA has 32 x (TZ/R) threads; each thread owns two adjacent columns and
// R consecutive rows (R is a property of the kernel variant).  Tiles are
// staged through double-buffered shared memory with cp.async.
constexpr int TX = 64;
constexpr int TZ = 64;
constexpr int HALO = 4;          // radius of the 8th-order stencil
constexpr int SROW = TX + 2 * HALO;   // shared-memory row length (floats)
constexpr int SROWS = TZ + 2 * HALO;
constexpr int POOL_ALIGN = TX;   // row pitch of a window is a multiple of this

// Per-shot descriptor, indexed by "slot" (shots sorted by record length,
// longest first, so that the shots still running at step n are a prefix).
struct ShotDesc {
    long long foff;   // offset (floats) of this shot's window inside a field pool
    long long doff;   // offset of this shot's block in the packed data vector
    int nxw;          // padded window width (cells) = win_x1 - win_x0 + 2 nb
    int pitch;        // row pitch of the window in a field pool (floats, multiple of TX)
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

// Per-tile descriptor of the TMA-staged kernels: the tile and the fields of
// its shot they read, denormalised so that one 80-byte copy gives them all
// (no dependent shot-table load on a kernel's critical path).
enum { TI_INTERIOR = 1, TI_FULL_FWD = 2, TI_FULL2 = 4, TI_INTERIOR2 = 8 };
struct alignas(16) TileInfo {
    int slot, z0, x0;
    int mx;             // model-array column of the tile: (shot x0 & ~3) + x0, in copy mc
    int mc;             // shot x0 & 3
    int nxw, pitch;
    int sz, sx;         // source node, window coordinates
    int wav_off, nrec;
    int rec_begin, rec_end;
    int flags;          // TI_INTERIOR: inside the sponge-free interior (all cells valid);
                        // TI_FULL_FWD: interior and without the source node;
                        // TI_FULL2: the tile grown by HALO on every side is interior
                        //           and holds no source node (two-step kernel);
                        // TI_INTERIOR2: the grown tile is interior (two-step adjoint)
    int nt;             // record length of the shot
    int pad1;
    long long foff, doff;
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
    // Padded model arrays [NZ][pf]; kap and dkap hold four copies (mstride
    // floats apart): copy r is copy 0 shifted left by r columns.
    const float *kap;     // kappa = v^2 dt^2/h^2
    long long mstride;    // floats between consecutive copies
    const TileInfo *infos;  // per-tile descriptors (TMA-staged kernels)
    const float *wav;     // wavelets
    int pf;               // pitch of the padded model arrays
    int NZ;               // padded rows = nz + 2 nb
    int nb;
    unsigned *tflag;      // set to 1 by a TMA-staged kernel whose bounded wait ran out
    // Receivers of each tile's grown region (the tile and its HALO ring, a
    // (TX + 2 HALO)^2 square, cell = ez * (TX + 2 HALO) + ex), by cell then
    // receiver: tile t's are xrecs[xrec_off[t] .. xrec_off[t + 1]).  The
    // two-step adjoint applies the data injection of its first step to the
    // staged D_nu from them (nullable: no such lists, separate injection).
    const TileRec *xrecs = nullptr;
    const int *xrec_off = nullptr;
};
// Most grown-region receiver entries the two-step adjoint's shared-memory
// list holds; plans with more use the separate injection pass.
constexpr int kInjCap = 256;

// Tensor maps of one TMA-staged step launch (kernel parameters).  A field
// pool is a 3-D float array [slot][NZ][pitch] (x = column, y = row, z =
// slot), a model array [copy][NZ][pf] (z = copy).  Halo maps have a
// (TX + 8) x (TZ + 8) box, cell maps TX x TZ; elements outside the array read
// as zero.  Slot use per kind:
//   forward: 0 u^n (halo), 1 D^n, 2 kappa
//   adjoint: 0 nu^{k+1} (halo), 1 D_nu, 2 kappa, 3 a^{k-1}, 4 image
//   Born:    0 u0^n (halo), 1 p^n (halo), 2 D_u0, 3 D_p, 4 kappa, 5 d kappa
struct TileMaps {
    CUtensorMap m[6];
};

// Every propagated field is kept in "summed" form: the field u^n and its
// damped time difference D^n = u^n - w u^{n-1}.  The recurrence
//   u^{n+1} = w (2 u^n + kappa a^n) - w^2 u^{n-1}
// is then, exactly,
//   D^{n+1} = w (D^n + kappa a^n),   u^{n+1} = w u^n + D^{n+1}.
// u is double buffered (neighbours read u^n while u^{n+1} is written); D is
// updated in place.

// Forward step n over the active tiles (grid = number of active tiles).
struct FwdArgs {
    StepCommon c;
    const float *u;   // pool: u^n
    float *un;        // pool: u^{n+1} (written)
    float *dd;        // pool: D^n, overwritten with D^{n+1}
    float *ck_u;      // nullable: store u^n here (checkpoint; ignored when a_out is set)
    float *ck_d;      // nullable: store D^n here (checkpoint)
    float *a_out;     // nullable: store a^n = D u^n + q^n (history or segment buffer slot)
    float *d;         // nullable: packed records, sample n written from u^{n+1}
    int n;
    // Two-step kernel only (steps n and n+1 in one launch): D^n is read with a
    // ring of neighbour cells, so D^{n+2} goes to another pool; u^{n+2} goes
    // to un; a^{n+1} to a_out2; tiles of shots with nt = n+1 take one step.
    float *dd_out;
    float *a_out2;
};

// Adjoint step k for the scaled multiplier nu = kappa w lambda, which obeys
// the forward recurrence with the data injected like the source, in the same
// summed form.
struct AdjArgs {
    StepCommon c;
    const float *nu;      // pool: nu^{k+1}
    float *nun;           // pool: nu^k (written)
    float *dd;            // pool: D_nu^{k+1}, overwritten with D_nu^k
    const float *r;       // packed data injected at the receivers (sample k-1)
    const float *a;       // pool: a^{k-1} of the background forward field
    float *g;             // pool: per-shot image accumulator, += a^{k-1} nu^k
    int k;
    // Two-step kernel only (steps k and k-1 in one launch): dd holds D_nu^{k+1}
    // with the data of step k already injected (launch_adj_inject), D_nu^{k-1}
    // goes to dd_out, nu^{k-1} to nun, a2 = a^{k-2}.  With inject_here set
    // the data of step k are not in dd: each tile adds them to its staged
    // D_nu from c.xrecs (same arithmetic as launch_adj_inject).
    float *dd_out;
    const float *a2;
    int inject_here = 0;
};

// Born joint step n: background u0 and scattered p advance together.
struct BornArgs {
    StepCommon c;
    const float *u;  float *un;  float *du;   // background: u0^n, u0^{n+1}, D_u0 in place
    const float *p;  float *pn;  float *dp;   // scattered:  p^n,  p^{n+1},  D_p in place
    const float *dkap;                         // padded d kappa = 2 kappa dv / v (four copies)
    float *d;                                  // packed Born records (sample n from p^{n+1})
    int n;
    // Background term a^n = D u0^n + q^n read from a stored forward history
    // (launch_born_hist_step; the u fields are then not used).
    const float *a = nullptr;
};

// Step-kernel variants.  Variants 0-2: tiles staged by per-thread cp.async,
// R = 2, 4, 8 rows per thread (CTA = 32 x 64/R threads).  Variants 3-5:
// tiles staged by TMA (cp.async.bulk.tensor issued by one thread, mbarrier
// completion), R = 4, 8, 16; the adjoint and Born kernels stop at R = 8
// (step_variants()).  Born only: variants 5 and 6 are its TMA kernel with
// R = 4 and 8 and ONE stage (refilled after each tile) instead of two, so
// that two CTAs fit on an SM.  The autotuner in api.cu times them per
// geometry.
constexpr int N_STEP_VARIANTS = 7;
constexpr int FIRST_TMA_VARIANT = 3;
int step_variant_rows(int v);
// Variants available for a kernel kind (0 forward, 1 adjoint, 2 Born).
int step_variants(int kind);
// Resident CTAs per SM of a step kernel; kind 0 forward, 1 adjoint, 2 Born.
int step_occupancy(int kind, int variant, int store_a);

// Two-step (time-blocked) TMA forward kernel (fd_tma2.cu): steps n and n+1
// of the tiles active at step n.  maps: 0 u^n (HALO2 box), 1 D^n (halo box),
// 2 kappa (model halo box).
constexpr int HALO2 = 2 * HALO;
void launch_fwd_pair(const FwdArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s);
int fwd_pair_occupancy();
// Two-step adjoint (fd_tma2.cu): steps k and k-1 of the tiles active at step
// k-1; maps: 0 nu^{k+1} (HALO2 box), 1 D_nu (halo box), 2 kappa (model halo
// box).  Before it, launch_adj_inject adds kappa r^{k-1} (the data of step k,
// receivers sharing a cell summed in order) to D_nu at the receiver cells of
// the first nrtiles tiles listed in rtiles (tiles with receivers, by slot).
void launch_adj_pair(const AdjArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s);
void launch_adj_inject(const AdjArgs &a, const int *rtiles, int nrtiles, cudaStream_t s);

// TMA-staged step kernels (fd_tma.cu); variant >= FIRST_TMA_VARIANT.
void launch_fwd_step_tma(const FwdArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s);
void launch_adj_step_tma(const AdjArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s);
void launch_born_step_tma(const BornArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s);
// Born step with the background's a^n read from the forward history (maps:
// 0 p^n halo, 1 D_p, 2 kappa, 3 d kappa, 4 a^n cell box): only the
// scattered field is advanced; the same bits as the joint step.
void launch_born_hist_step(const BornArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s);
int tma_occupancy(int kind, int variant);

struct StepLaunch {
    int variant = 1;     // index into the variant table
    int max_ctas = 152;  // persistent grid cap = resident CTAs per SM x SMs
};

// Persistent launches: grid = min(ntiles, max_ctas); each CTA walks the tile
// list with a stride of gridDim.x.  maps: the launch's tensor maps, required
// by the TMA variants, ignored (may be null) by the others.
void launch_fwd_step(const FwdArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s);
void launch_adj_step(const AdjArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s);
void launch_born_step(const BornArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s);

// Padded model preparation: kap (and dkap when dv != nullptr) from the
// physical [nz][nx] model, columns [0, pf) (clamped beyond the model); also
// checks v (finite, > 0) and records max kappa.
// status[0] |= 1 for a bad velocity; status[1] = bits of max kappa (float);
// status[8..9] (64-bit, 8-byte aligned, cleared by the caller) += a hash of
// v's values and positions.
void launch_prep_model(const float *v, const float *dv, int rel, int nz, int nx, int nb, double c,
                       float *kap, float *dkap, int pf, long long mstride,
                       unsigned *status, cudaStream_t s);

// r = d_syn - d_obs, and per-block partial sums of r^2 (double).
void launch_residual(const float *ds, const float *dobs, float *r, long long n, double *partial,
                     int nblocks, cudaStream_t s);

// vout = clamp(v - alpha * dir / max|dir|, vmin, vmax), dir taken as 0 in the
// first mute_rows rows (also excluded from the max); mxbits: 1 word scratch.
// Partial sums of Eq. 17 (dx.dg, dg.dg per block into partial[2 * nblocks])
// and max |g_k| (float bits into *mxbits) over n values.
void launch_bb_partials(const float *xk, const float *xp, const float *gk, const float *gp, long long n,
                        double *partial, int nblocks, unsigned *mxbits, cudaStream_t s);
void launch_update_model(const float *v, const float *dir, int nz, int nx, int mute_rows, float alpha, float vmin,
                         float vmax, unsigned *mxbits, float *vout, cudaStream_t s);

// One kernel whose bounded wait runs out (on a barrier nothing arrives at)
// and sets *tflag, as a step kernel's timed-out wait does.
void launch_wait_timeout_selftest(unsigned *tflag, cudaStream_t s);

// out = -(5-point Laplacian of img) / h^2 on [nz][nx], edge values repeated
// outside the grid; out must not alias img.
void launch_image_laplacian(const float *img, int nz, int nx, float h, float *out, cudaStream_t s);

// Sum of the per-shot image accumulators into the physical [nz][nx] grid,
// folding the sponge cells onto the edge cells they copy (transpose of the
// extension), shots in original order, times the imaging factor 2/v (rel !=
// 0: times v as well, i.e. times 2).
void launch_reduce_image(const ShotDesc *shots, const int *slot_of_shot, int n_shots,
                         const float *gpool, int nz, int nx, int nb, const float *v, int rel,
                         float *out, cudaStream_t s);

}  // namespace dhfwi
