// Two-step (time-blocked) forward kernel for sm_103a: one launch advances
// every active tile by the steps n and n+1 of the recurrence of Section 2.1
// (Eq. 1, summed form, difference-form Laplacian; see fd_kernels.cu), so
// u and D cross HBM once per two updates.
//
// Per 64 x 64 tile the TMA stages u^n with an 8-cell halo (80 x 80) and D^n
// and kappa with a 4-cell ring (72 x 72).  Step n is computed on the tile
// grown by the ring (36 column pairs x 72 rows, 9 rows per thread), giving
// u^{n+1} and D^{n+1} on 72 x 72 in shared memory (zero outside the window:
// the Dirichlet boundary); step n+1 is then computed on the core from them.
// The ring cells are recomputed by each tile that needs them, so tiles
// never exchange data within the launch; since they read D^n on their
// neighbours' cells, D^{n+2} goes to a second pool.  Every cell goes through
// the same floating-point operations in the same order as in the one-step
// kernels, so the results are bit-identical.
//
// Sources: injected at both steps (q^n, q^{n+1}), also on ring cells.
// Receivers: sample n from u^{n+1} in shared memory, sample n+1 from the
// pool after the tile's stores.  Checkpoints (u^n, D^n) at even n, segment
// stores of a^n and a^{n+1} for the backward recompute.  Tiles of a shot
// whose record ends at n+1 take step n only.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fd_tma.cuh"

namespace dhfwi {
namespace {

constexpr int E = TX + 2 * HALO;    // 72: core + ring
constexpr int U2 = TX + 2 * HALO2;  // 80: u^n box
static_assert(TX == TZ, "square tiles");
typedef float UTile2[U2][U2];  // u^n: rows z0-8 .., cols x0-8 ..
typedef float ETile[E][E];     // rows z0-4 .., cols x0-4 ..

struct Fwd2Stage {
    UTile2 u;
    ETile d, k;
};
constexpr unsigned kFwd2StageBytes = sizeof(UTile2) + 2 * sizeof(ETile);
static_assert(sizeof(Fwd2Stage) == kFwd2StageBytes && sizeof(Fwd2Stage) % 128 == 0, "stage layout");
constexpr size_t kFwd2Smem = sizeof(Fwd2Stage) + 2 * sizeof(ETile) + sizeof(PipeTail);
// The two-step adjoint's list of its next tile's data injection (grown
// region, step k): offset of the cell in the staged D_nu (-1: a further
// receiver of the cell before, already summed), kappa there, summed data.
struct InjEntry {
    int off;
    float kap, sum;
};
struct InjBuf {
    int n, pad[3];
    InjEntry e[kInjCap];
};
constexpr size_t kAdj2Smem = kFwd2Smem + sizeof(InjBuf);
static_assert(kFwd2Smem % 16 == 0, "injection list alignment");
// Thread layout: 288 threads.  Step n covers the 72 x 72 grown tile with
// 36 column pairs x 8 blocks of R1 = 9 rows; step n+1 covers the 64 x 64
// core with the first 256 threads, 32 column pairs x 8 blocks of R2 = 8 rows.
constexpr int NT2 = 288, R1 = 9, R2 = 8, PAIRS1 = E / 2;
static_assert(PAIRS1 * (E / R1) == NT2 && (TX / 2) * (TZ / R2) == 256, "thread layout");

// mid(): called by every thread after the barrier that ends step n (the
// stage is no longer read; kappa of the core is in registers): the leader
// refills the stage.
template <bool STORE_A, bool FULL, class MidFn>
__device__ __forceinline__ void pair_tile(const FwdArgs &A, const Fwd2Stage &S, ETile &V, ETile &Dn, const TileInfo &T,
                                          int tid, bool two, MidFn mid) {
    const int NZ = A.c.NZ, nb = A.c.nb, nxw = T.nxw, pitch = T.pitch, n = A.n;
    float q0 = 0.f, q1 = 0.f;
    if constexpr (!FULL) {
        q0 = A.c.wav[T.wav_off + n];
        q1 = two ? A.c.wav[T.wav_off + n + 1] : 0.f;
    }

    // ---- step n on the grown tile -----------------------------------------
    {
        const int ex = 2 * (tid % PAIRS1), ez0 = R1 * (tid / PAIRS1);
        const int jj = T.x0 - HALO + ex;  // window column of lane 0
        const bool core_x = ex >= HALO && ex < TX + HALO;
        float wx0 = 1.f, wx1 = 1.f;
        bool c0ok = true, c1ok = true;
        if constexpr (!FULL) {
            c0ok = jj >= 0 && jj < nxw;
            c1ok = jj + 1 >= 0 && jj + 1 < nxw;
            wx0 = sponge1(jj, nxw, nb);
            wx1 = sponge1(jj + 1, nxw, nb);
        }
        float2 zc[R1 + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R1 + 2 * HALO; r++) zc[r] = *reinterpret_cast<const float2 *>(&S.u[ez0 + r][ex + HALO]);
#pragma unroll
        for (int rr = 0; rr < R1; rr++) {
            const int ez = ez0 + rr;
            const int i = T.z0 - HALO + ez;
            f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&S.u[ez + HALO][ex]), zc + rr);
            const f2 u = pk(zc[rr + HALO]);
            const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[ez][ex]));
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[ez][ex]));
            f2 dn, un;
            bool v0 = true, v1 = true;
            if constexpr (FULL) {
                dn = fma2(kv, a, dv);
                un = add2(u, dn);
            } else {
                const bool rok = i >= 0 && i < NZ;
                v0 = rok && c0ok;
                v1 = rok && c1ok;
                a = inject(a, i, jj, T.sz, T.sx, q0);
                const float wz = sponge1(i, NZ, nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                dn = keep_lo(mul2(w, fma2(kv, a, dv)), v1);
                un = keep_lo(fma2(w, u, dn), v1);
                if (!v0) dn = un = 0ull;
            }
            *reinterpret_cast<f2 *>(&V[ez][ex]) = un;
            *reinterpret_cast<f2 *>(&Dn[ez][ex]) = dn;
            if (core_x && ez >= HALO && ez < TZ + HALO && v0) {
                const long long c = T.foff + (long long)i * pitch + jj;
                if (!STORE_A && A.ck_u) {
                    *reinterpret_cast<f2 *>(A.ck_u + c) = keep_lo(u, v1);
                    *reinterpret_cast<f2 *>(A.ck_d + c) = keep_lo(dv, v1);
                }
                if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out + c) = keep_lo(a, v1);
            }
        }
    }
    // kappa of this thread's core cells for step n+1; after the barrier the
    // stage is no longer read and u^{n+1}, D^{n+1} are complete.
    const int lxp = 2 * (tid % 32), lz0 = R2 * (tid / 32);
    const bool worker = tid < 256;
    f2 kv2[R2];
#pragma unroll
    for (int rr = 0; rr < R2; rr++)
        kv2[rr] = worker ? *reinterpret_cast<const f2 *>(&S.k[lz0 + rr + HALO][lxp + HALO]) : 0ull;
    __syncthreads();
    mid();

    // Receivers: sample n is u^{n+1}.
    if (A.d) {
        for (int e = T.rec_begin + tid; e < T.rec_end; e += NT2) {
            const TileRec tr = A.c.recs[e];
            A.d[T.doff + (long long)n * T.nrec + tr.r] = V[tr.cell / TX + HALO][tr.cell % TX + HALO];
        }
    }

    // ---- step n+1 on the core (threads 0..255) ---------------------------------
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R2 : min(R2, NZ - i0);
    const bool ok = worker && (FULL || j < nxw), hi = FULL || j + 1 < nxw;
    if (!two) {  // the record ends at n+1: store u^{n+1}, D^{n+1}
#pragma unroll
        for (int rr = 0; rr < R2; rr++) {
            if (ok && rr < nrow) {
                const long long c = cbase + (long long)rr * pitch;
                *reinterpret_cast<f2 *>(A.un + c) = *reinterpret_cast<const f2 *>(&V[lz0 + rr + HALO][lxp + HALO]);
                *reinterpret_cast<f2 *>(A.dd_out + c) = *reinterpret_cast<const f2 *>(&Dn[lz0 + rr + HALO][lxp + HALO]);
            }
        }
        return;
    }
    if (worker) {
        float wx0 = 1.f, wx1 = 1.f;
        if constexpr (!FULL) {
            wx0 = sponge1(j, nxw, nb);
            wx1 = sponge1(j + 1, nxw, nb);
        }
        float2 zc[R2 + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R2 + 2 * HALO; r++) zc[r] = *reinterpret_cast<const float2 *>(&V[lz0 + r][lxp + HALO]);
#pragma unroll
        for (int rr = 0; rr < R2; rr++) {
            if (!(ok && rr < nrow)) continue;
            f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&V[lz0 + rr + HALO][lxp]), zc + rr);
            if constexpr (!FULL) a = inject(a, i0 + rr, j, T.sz, T.sx, q1);
            const f2 u = pk(zc[rr + HALO]);
            const f2 kv = kv2[rr];
            const f2 d1 = *reinterpret_cast<const f2 *>(&Dn[lz0 + rr + HALO][lxp + HALO]);
            f2 dn, un;
            if constexpr (FULL) {
                dn = fma2(kv, a, d1);
                un = add2(u, dn);
            } else {
                const float wz = sponge1(i0 + rr, NZ, nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                dn = keep_lo(mul2(w, fma2(kv, a, d1)), hi);
                un = keep_lo(fma2(w, u, dn), hi);
            }
            const long long c = cbase + (long long)rr * pitch;
            *reinterpret_cast<f2 *>(A.dd_out + c) = dn;
            *reinterpret_cast<f2 *>(A.un + c) = un;
            if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out2 + c) = keep_lo(a, hi);
        }
    }
    // Receivers: sample n+1 is u^{n+2}, read back from the pool.
    if (A.d && T.rec_end > T.rec_begin) sample_from_pool<NT2>(A.c, T, A.un, A.d, n + 1);
}

// Tile loop: one stage, refilled in the middle of a tile (see mid() in
// pair_tile) so that the next tile's loads overlap step n+1; the descriptor
// slot is refilled at the end of the tile.  Waits bounded as in run_tiles.
template <bool STORE_A>
__global__ void __launch_bounds__(NT2, 2) fwd_pair_kernel(FwdArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Fwd2Stage &S = *reinterpret_cast<Fwd2Stage *>(smem_raw);
    ETile &V = *reinterpret_cast<ETile *>(smem_raw + sizeof(Fwd2Stage));
    ETile &Dn = *reinterpret_cast<ETile *>(smem_raw + sizeof(Fwd2Stage) + sizeof(ETile));
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + sizeof(Fwd2Stage) + 2 * sizeof(ETile));
    const int tid = threadIdx.x + threadIdx.y * 32;
    const bool leader = tid == 0;
    const unsigned bar = smem_u32(&tail->bar[0]);
    const int b = blockIdx.x, g = gridDim.x;
    int4 co = make_int4(0, 0, 0, 0);
    int mc = 0;
    if (smem_u32(&S) & 127u) {
        if (leader) atomicExch(A.c.tflag, 2u);
        return;
    }
    if (leader) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fetch_coords(A.c.infos, b, co, mc);
        copy_desc(&tail->desc[0], &A.c.infos[b]);
    }
    griddep_wait();
    griddep_launch_dependents();
    auto issue = [&]() {
        fence_proxy_async();
        mbar_expect_tx(bar, kFwd2StageBytes);
        tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO2, co.y - HALO2, co.x, bar);
        tma_load_3d(smem_u32(&S.d), &M.m[1], co.z - HALO, co.y - HALO, co.x, bar);
        tma_load_3d(smem_u32(&S.k), &M.m[2], co.w - HALO, co.y - HALO, mc, bar);
    };
    if (leader) {
        issue();
        if (b + g < ntiles) fetch_coords(A.c.infos, b + g, co, mc);
    }
    __syncthreads();
    unsigned phase = 0;
    for (int tix = b; tix < ntiles; tix += g) {
        const bool landed = mbar_wait(bar, phase);
        phase ^= 1u;
        if (leader) cp_async_wait_all();
        if (__syncthreads_or(!landed)) {
            if (leader) {
                mbar_wait(bar, phase ^ 1u);  // copies in flight: a second bounded wait before leaving
                atomicExch(A.c.tflag, 1u);
            }
            return;
        }
        const bool more = tix + g < ntiles;
        auto mid = [&]() {  // after a barrier: every thread is done with the stage
            if (leader && more) issue();
        };
        const TileInfo &T = tail->desc[0];
        const bool two = T.nt > A.n + 1;
        if ((T.flags & TI_FULL2) && two) pair_tile<STORE_A, true>(A, S, V, Dn, T, tid, true, mid);
        else pair_tile<STORE_A, false>(A, S, V, Dn, T, tid, two, mid);
        __syncthreads();  // the descriptor, V and Dn are free
        if (leader && more) {
            copy_desc(&tail->desc[0], &A.c.infos[tix + g]);
            if (tix + 2 * g < ntiles) fetch_coords(A.c.infos, tix + 2 * g, co, mc);
        }
    }
}

// ---------------------------------------------------------------------------
// Two-step adjoint: steps k (nu^{k+1} -> nu^k) and k-1 in one launch, the
// same layout and stage refill as fwd_pair_kernel.  The data of step k are
// already in the staged D_nu (D' = D + kappa r^{k-1}, launch_adj_inject, so
// ring cells need no injection tile); the data of step k-1 are added to the
// core's D_nu^k in shared memory after step k.  The image accumulator takes
// a^{k-1} nu^k (tiles whose record reaches step k) and then a^{k-2} nu^{k-1},
// in that order, as two one-step launches would.
// ---------------------------------------------------------------------------
template <bool FULL, class MidFn>
__device__ __forceinline__ void adj_pair_tile(const AdjArgs &A, const Fwd2Stage &S, ETile &V, ETile &Dn,
                                              const TileInfo &T, int tid, MidFn mid) {
    const int NZ = A.c.NZ, nb = A.c.nb, nxw = T.nxw, pitch = T.pitch, k = A.k;

    // ---- step k on the grown tile -------------------------------------------
    {
        const int ex = 2 * (tid % PAIRS1), ez0 = R1 * (tid / PAIRS1);
        const int jj = T.x0 - HALO + ex;
        float wx0 = 1.f, wx1 = 1.f;
        bool c0ok = true, c1ok = true;
        if constexpr (!FULL) {
            c0ok = jj >= 0 && jj < nxw;
            c1ok = jj + 1 >= 0 && jj + 1 < nxw;
            wx0 = sponge1(jj, nxw, nb);
            wx1 = sponge1(jj + 1, nxw, nb);
        }
        float2 zc[R1 + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R1 + 2 * HALO; r++) zc[r] = *reinterpret_cast<const float2 *>(&S.u[ez0 + r][ex + HALO]);
#pragma unroll
        for (int rr = 0; rr < R1; rr++) {
            const int ez = ez0 + rr;
            const int i = T.z0 - HALO + ez;
            const f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&S.u[ez + HALO][ex]), zc + rr);
            const f2 nu = pk(zc[rr + HALO]);
            const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[ez][ex]));
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[ez][ex]));
            f2 dn, nn;
            if constexpr (FULL) {
                dn = fma2(kv, a, dv);
                nn = add2(nu, dn);
            } else {
                const bool rok = i >= 0 && i < NZ;
                const bool v0 = rok && c0ok, v1 = rok && c1ok;
                const float wz = sponge1(i, NZ, nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                dn = keep_lo(mul2(w, fma2(kv, a, dv)), v1);
                nn = keep_lo(fma2(w, nu, dn), v1);
                if (!v0) dn = nn = 0ull;
            }
            *reinterpret_cast<f2 *>(&V[ez][ex]) = nn;
            *reinterpret_cast<f2 *>(&Dn[ez][ex]) = dn;
        }
    }
    const int lxp = 2 * (tid % 32), lz0 = R2 * (tid / 32);
    const bool worker = tid < 256;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R2 : min(R2, NZ - i0);
    const bool ok = worker && (FULL || j < nxw), hi = FULL || j + 1 < nxw;
    // Global operands of the second step (image accumulator, a^{k-1},
    // a^{k-2}; prefetched into L2 a tile ahead) kept PF rows ahead of the
    // arithmetic, the first rows requested before the barrier.  a^{k-1}
    // exists only where the record reaches step k (a stored history holds
    // the shots active at each step only).
    const bool image_k = T.nt > k - 1;
    constexpr int PF = 2;
    f2 gq[PF], a1q[PF], a2q[PF];
    auto fetch = [&](int rr, int q) {
        const bool v = ok && rr < nrow;
        const long long c = cbase + (long long)rr * pitch;
        gq[q] = v ? *reinterpret_cast<const f2 *>(A.g + c) : 0ull;
        a1q[q] = v && image_k ? *reinterpret_cast<const f2 *>(A.a + c) : 0ull;
        a2q[q] = v ? *reinterpret_cast<const f2 *>(A.a2 + c) : 0ull;
    };
#pragma unroll
    for (int q = 0; q < PF; q++) fetch(q, q);
    __syncthreads();  // nu^k, D_nu^k complete on the grown tile

    // Data of step k-1 at the tile's receivers: D' = D_nu^k + kappa r^{k-2}.
    if (T.rec_end > T.rec_begin) {
        const float *rk = A.r + T.doff + (long long)(k - 2) * T.nrec;
        for (int e = T.rec_begin + tid; e < T.rec_end; e += NT2)
            if (e == T.rec_begin || A.c.recs[e - 1].cell != A.c.recs[e].cell) {
                const int cell = A.c.recs[e].cell;
                const int lz = cell / TX + HALO, lx = cell % TX + HALO;
                Dn[lz][lx] = fmaf(S.k[lz][lx], receiver_sum(A.c.recs, e, T.rec_end, rk), Dn[lz][lx]);
            }
        __syncthreads();
    }
    mid();  // u and D_nu of the stage are no longer read (kappa is: it is refilled at the tile's end)

    // ---- step k-1 on the core (threads 0..255), imaging of both steps -----
    if (!worker) return;
    float wx0 = 1.f, wx1 = 1.f;
    if constexpr (!FULL) {
        wx0 = sponge1(j, nxw, nb);
        wx1 = sponge1(j + 1, nxw, nb);
    }
    float2 zc[R2 + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R2 + 2 * HALO; r++) zc[r] = *reinterpret_cast<const float2 *>(&V[lz0 + r][lxp + HALO]);
#pragma unroll
    for (int rr = 0; rr < R2; rr++) {
        const int q = rr % PF;
        f2 g = gq[q];
        const f2 a1 = a1q[q], a2 = a2q[q];
        if (rr + PF < R2) fetch(rr + PF, q);
        if (!(ok && rr < nrow)) continue;
        const long long c = cbase + (long long)rr * pitch;
        const f2 kv = *reinterpret_cast<const f2 *>(&S.k[lz0 + rr + HALO][lxp + HALO]);
        const f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&V[lz0 + rr + HALO][lxp]), zc + rr);
        const f2 nu = pk(zc[rr + HALO]);  // nu^k
        const f2 d1 = *reinterpret_cast<const f2 *>(&Dn[lz0 + rr + HALO][lxp + HALO]);
        f2 dn, nn;
        if constexpr (FULL) {
            dn = fma2(kv, a, d1);
            nn = add2(nu, dn);
        } else {
            const float wz = sponge1(i0 + rr, NZ, nb);
            const f2 w = pk2(wz * wx0, wz * wx1);
            dn = keep_lo(mul2(w, fma2(kv, a, d1)), hi);
            nn = keep_lo(fma2(w, nu, dn), hi);
        }
        if (image_k) g = keep_lo(fma2(a1, nu, g), hi);
        g = keep_lo(fma2(a2, nn, g), hi);
        *reinterpret_cast<f2 *>(A.dd_out + c) = dn;
        *reinterpret_cast<f2 *>(A.nun + c) = nn;
        *reinterpret_cast<f2 *>(A.g + c) = g;
    }
}

__global__ void __launch_bounds__(NT2, 2) adj_pair_kernel(AdjArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Fwd2Stage &S = *reinterpret_cast<Fwd2Stage *>(smem_raw);
    ETile &V = *reinterpret_cast<ETile *>(smem_raw + sizeof(Fwd2Stage));
    ETile &Dn = *reinterpret_cast<ETile *>(smem_raw + sizeof(Fwd2Stage) + sizeof(ETile));
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + sizeof(Fwd2Stage) + 2 * sizeof(ETile));
    InjBuf &IB = *reinterpret_cast<InjBuf *>(smem_raw + kFwd2Smem);
    const int tid = threadIdx.x + threadIdx.y * 32;
    const bool leader = tid == 0;
    const unsigned bar = smem_u32(&tail->bar[0]);
    const int b = blockIdx.x, g = gridDim.x;
    int4 co = make_int4(0, 0, 0, 0);
    int mc = 0;
    if (smem_u32(&S) & 127u) {
        if (leader) atomicExch(A.c.tflag, 2u);
        return;
    }
    if (leader) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fetch_coords(A.c.infos, b, co, mc);
        copy_desc(&tail->desc[0], &A.c.infos[b]);
    }
    griddep_wait();
    griddep_launch_dependents();
    // The stage is refilled in two parts on one mbarrier phase: u and D_nu
    // once the first step is done, kappa (read by the second step too) at
    // the end of the tile.  The same tile's image, a^{k-1} and a^{k-2},
    // which the second step loads from global memory, are prefetched into L2
    // then, a tile ahead of their use.
    auto issue_ud = [&]() {
        fence_proxy_async();
        mbar_expect_tx(bar, kFwd2StageBytes);
        tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO2, co.y - HALO2, co.x, bar);
        tma_load_3d(smem_u32(&S.d), &M.m[1], co.z - HALO, co.y - HALO, co.x, bar);
        tma_prefetch_l2_3d(&M.m[3], co.z, co.y, co.x);
        tma_prefetch_l2_3d(&M.m[4], co.z, co.y, co.x);
        tma_prefetch_l2_3d(&M.m[5], co.z, co.y, co.x);
    };
    auto issue_k = [&]() {
        fence_proxy_async();
        tma_load_3d(smem_u32(&S.k), &M.m[2], co.w - HALO, co.y - HALO, mc, bar);
    };
    // Data of step k injected here (inject_here): warp 8, which has no cells
    // in the second step, lists the next tile's grown-region injection
    // (kappa and the receivers' summed data, from global memory) while the
    // other warps run that step; after the tile's stage lands every thread
    // adds the list to the staged D_nu, D' = fmaf(kappa, sum, D) as the
    // separate pass computes it.  Shots whose record ends before step k take
    // none.
    const bool inj = A.inject_here && A.c.xrec_off != nullptr;
    auto build = [&](int t) {
        const int lane = tid - 256;
        const int xb = A.c.xrec_off[t], xe = A.c.xrec_off[t + 1];
        const TileInfo &Tg = A.c.infos[t];
        const bool has = Tg.nt > A.k - 1;
        const float *rk = A.r + Tg.doff + (long long)(A.k - 1) * Tg.nrec;
        for (int e = xb + lane; has && e < xe; e += 32) {
            InjEntry en{-1, 0.f, 0.f};
            if (e == xb || A.c.xrecs[e - 1].cell != A.c.xrecs[e].cell) {
                const int cell = A.c.xrecs[e].cell, ez = cell / E, ex = cell % E;
                en.off = cell;
                en.kap = A.c.kap[(long long)Tg.mc * A.c.mstride + (long long)(Tg.z0 - HALO + ez) * A.c.pf + Tg.mx +
                                 ex - HALO];
                en.sum = receiver_sum(A.c.xrecs, e, xe, rk);
            }
            IB.e[e - xb] = en;
        }
        if (lane == 0) IB.n = has ? xe - xb : 0;
    };
    if (leader) {
        issue_ud();
        issue_k();
        if (b + g < ntiles) fetch_coords(A.c.infos, b + g, co, mc);
    }
    if (inj && tid >= 256) build(b);
    __syncthreads();
    unsigned phase = 0;
    for (int tix = b; tix < ntiles; tix += g) {
        const bool landed = mbar_wait(bar, phase);
        phase ^= 1u;
        if (leader) cp_async_wait_all();
        if (__syncthreads_or(!landed)) {
            if (leader) {
                mbar_wait(bar, phase ^ 1u);  // copies in flight: a second bounded wait before leaving
                atomicExch(A.c.tflag, 1u);
            }
            return;
        }
        if (inj) {
            const int n = IB.n;  // uniform: written before the last barrier
            float *dflat = &S.d[0][0];
            for (int e = tid; e < n; e += NT2) {
                const InjEntry en = IB.e[e];
                if (en.off >= 0) dflat[en.off] = fmaf(en.kap, en.sum, dflat[en.off]);
            }
            if (n > 0) __syncthreads();
        }
        const bool more = tix + g < ntiles;
        auto mid = [&]() {  // after a barrier: every thread is done with u and D_nu
            if (leader && more) issue_ud();
        };
        const TileInfo &T = tail->desc[0];
        if (T.flags & TI_INTERIOR2) adj_pair_tile<true>(A, S, V, Dn, T, tid, mid);
        else adj_pair_tile<false>(A, S, V, Dn, T, tid, mid);
        if (inj && tid >= 256 && more) build(tix + g);  // warp 8, during the other warps' second step
        __syncthreads();  // kappa, the descriptor, V and Dn are free
        if (leader && more) {
            issue_k();
            copy_desc(&tail->desc[0], &A.c.infos[tix + g]);
            if (tix + 2 * g < ntiles) fetch_coords(A.c.infos, tix + 2 * g, co, mc);
        }
    }
}

// D' = D_nu + kappa r^{k-1} at the receiver cells of the listed tiles (one
// CTA per tile; receivers sharing a cell summed in order, as in
// build_injection).
__global__ void adj_inject_kernel(AdjArgs A, const int *__restrict__ rtiles) {
    // Launched as a programmatic dependent: it may start before the step
    // kernel that writes D_nu has finished, so it waits for it here, and lets
    // the next step kernel start its prologue at once.
    griddep_wait();
    griddep_launch_dependents();
    const TileInfo &T = A.c.infos[rtiles[blockIdx.x]];
    const float *rk = A.r + T.doff + (long long)(A.k - 1) * T.nrec;
    for (int e = T.rec_begin + threadIdx.x; e < T.rec_end; e += blockDim.x)
        if (e == T.rec_begin || A.c.recs[e - 1].cell != A.c.recs[e].cell) {
            const int cell = A.c.recs[e].cell;
            const int z = T.z0 + cell / TX, lx = cell % TX;
            const float kap = A.c.kap[(long long)T.mc * A.c.mstride + (long long)z * A.c.pf + T.mx + lx];
            float *d = A.dd + T.foff + (long long)z * T.pitch + T.x0 + lx;
            *d = fmaf(kap, receiver_sum(A.c.recs, e, T.rec_end, rk), *d);
        }
}

template <typename K, typename Args>
void launch_pdl2(K kernel, int grid, const Args &a, const TileMaps &maps, int ntiles, cudaStream_t s,
                 size_t smem = kFwd2Smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, NT2 / 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, a, maps, ntiles);
}

int occupancy_of(const void *fn, size_t smem = kFwd2Smem) {
    int n = 0;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NT2, smem);
    return n < 1 ? 1 : n;
}

}  // namespace

void launch_adj_pair(const AdjArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    static int sms = 0, occ = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        occ = occupancy_of((const void *)adj_pair_kernel, kAdj2Smem);
    }
    const int cap = occ * sms;
    launch_pdl2(adj_pair_kernel, ntiles < cap ? ntiles : cap, a, maps, ntiles, s, kAdj2Smem);
}

void launch_adj_inject(const AdjArgs &a, const int *rtiles, int nrtiles, cudaStream_t s) {
    if (nrtiles <= 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nrtiles);
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, adj_inject_kernel, a, rtiles);
}

int fwd_pair_occupancy() {
    const int a = occupancy_of((const void *)fwd_pair_kernel<true>);
    const int b = occupancy_of((const void *)fwd_pair_kernel<false>);
    return a < b ? a : b;
}

void launch_fwd_pair(const FwdArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    static int sms = 0, occ = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        occ = fwd_pair_occupancy();
    }
    const int cap = occ * sms;
    const int grid = ntiles < cap ? ntiles : cap;
    if (a.a_out) launch_pdl2(fwd_pair_kernel<true>, grid, a, maps, ntiles, s);
    else launch_pdl2(fwd_pair_kernel<false>, grid, a, maps, ntiles, s);
}

}  // namespace dhfwi
