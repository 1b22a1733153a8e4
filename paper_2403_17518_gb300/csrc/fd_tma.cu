// TMA-staged step kernels for sm_103a: forward, adjoint and Born.  Each has
// the arithmetic of its cp.async counterpart in fd_kernels.cu (Section 2.1
// Eq. 1 in summed form with the difference-form Laplacian, the adjoint for
// Eq. 13, the Born system of Section 2.2), in the same order, so every
// variant gives bit-identical results.  What differs is how the tiles reach
// shared memory: one thread issues a few cp.async.bulk.tensor loads per tile
// (fields with their halo, state differences, kappa, ...) that complete on
// an mbarrier, instead of every thread computing and issuing ~13 cp.async
// chunks.  Out-of-range rows and columns read as zero from the tensor map,
// which requires the padding columns of a pool (past a window's width) to
// hold zero: every step kernel writes them as zero (keep_lo), and the host
// zeroes pools and checkpoints before a pass.
//
// Tiles fully inside the sponge-free interior (and, where there is one, away
// from the source) take a path with no sponge factor, no bounds masks and no
// injection test; the sponge factor there is exactly 1, so both paths round
// identically.  Receivers are sampled from the pool after the tile's stores.
//
// Pipeline: two stages; at tile i every thread waits for stage i mod 2, a
// barrier then certifies that all threads are done with tile i-1, and the
// leader issues tile i+1 into the freed stage.  Waits are bounded: a tile
// whose copies have not landed after about one second makes the whole CTA
// leave the kernel after setting *tflag = 1 (2: a misaligned shared-memory
// base, checked before any copy), which the host reports as
// DHFWI_ERR_TIMEOUT.  Before leaving, the leader waits once more (again
// bounded) for the copies it issued, so that a late copy does not land in
// shared memory another CTA owns; if even that wait runs out, the results of
// the launch and of the context's later calls are not to be trusted.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fd_tma.cuh"

namespace dhfwi {
namespace {
// ---------------------------------------------------------------------------
// Forward step (see fwd_step_kernel): u^n with halo, D^n and kappa by TMA.
// ---------------------------------------------------------------------------
struct TmaFwdStage {
    STile u;
    CTile d, k;
};
constexpr unsigned kFwdStageBytes = sizeof(STile) + 2 * sizeof(CTile);
static_assert(sizeof(TmaFwdStage) == kFwdStageBytes, "stage layout");
static_assert(sizeof(STile) % 128 == 0 && sizeof(CTile) % 128 == 0, "TMA destinations stay 128-byte aligned");
constexpr size_t kFwdSmem = 2 * sizeof(TmaFwdStage) + sizeof(PipeTail);

// R rows x 2 columns of one tile for this thread.  FULL: the tile lies in
// the sponge-free interior, holds no source and needs no bounds masks.
template <int R, bool STORE_A, bool FULL>
__device__ __forceinline__ void fwd_rows(const FwdArgs &A, const TmaFwdStage &S, const TileInfo &T, int lxp,
                                         int lz0) {
    const int NZ = A.c.NZ;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const int nxw = T.nxw, pitch = T.pitch;
    float2 zc[R + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++)
        zc[r] = *reinterpret_cast<const float2 *>(&S.u[lz0 + r][lxp + HALO]);
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    if constexpr (FULL) {
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            const f2 a = lap8x2(S.u, zc + rr, lz0 + rr, lxp);
            const f2 u = pk(zc[rr + HALO]);
            const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[lz0 + rr][lxp]));
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr][lxp]));
            const f2 dn = fma2(kv, a, dv);
            const long long c = cbase + (long long)rr * pitch;
            *reinterpret_cast<f2 *>(A.dd + c) = dn;
            *reinterpret_cast<f2 *>(A.un + c) = add2(u, dn);
            if (!STORE_A && A.ck_u) {
                *reinterpret_cast<f2 *>(A.ck_u + c) = u;
                *reinterpret_cast<f2 *>(A.ck_d + c) = dv;
            }
            if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out + c) = a;
        }
    } else {
        const int nrow = min(R, NZ - i0);
        const bool ok = j < nxw, hi = j + 1 < nxw;
        const float q = A.c.wav[T.wav_off + A.n];
        const float wx0 = sponge1(j, nxw, A.c.nb), wx1 = sponge1(j + 1, nxw, A.c.nb);
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            if (ok && rr < nrow) {
                const int i = i0 + rr;
                const f2 a = inject(lap8x2(S.u, zc + rr, lz0 + rr, lxp), i, j, T.sz, T.sx, q);
                const float wz = sponge1(i, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                const f2 u = pk(zc[rr + HALO]);
                const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[lz0 + rr][lxp]));
                const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr][lxp]));
                const f2 dn = keep_lo(mul2(w, fma2(kv, a, dv)), hi);
                const long long c = cbase + (long long)rr * pitch;
                *reinterpret_cast<f2 *>(A.dd + c) = dn;
                *reinterpret_cast<f2 *>(A.un + c) = keep_lo(fma2(w, u, dn), hi);
                if (!STORE_A && A.ck_u) {
                    *reinterpret_cast<f2 *>(A.ck_u + c) = keep_lo(u, hi);
                    *reinterpret_cast<f2 *>(A.ck_d + c) = keep_lo(dv, hi);
                }
                if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out + c) = keep_lo(a, hi);
            }
        }
    }
}

template <int R, bool STORE_A>
__global__ void __launch_bounds__(32 * (TZ / R), 1)
    fwd_tma_kernel(FwdArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaFwdStage *st = reinterpret_cast<TmaFwdStage *>(smem_raw);
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + 2 * sizeof(TmaFwdStage));
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;
    run_tiles<2>(
        A.c, kFwdStageBytes, ntiles, st, tail,
        [&](TmaFwdStage &S, unsigned bar, int4 co, int mc) {
            tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.d), &M.m[1], co.z, co.y, co.x, bar);
            tma_load_3d(smem_u32(&S.k), &M.m[2], co.w, co.y, mc, bar);
        },
        [&](const TmaFwdStage &S, const TileInfo &T) {
            if (T.flags & TI_FULL_FWD) fwd_rows<R, STORE_A, true>(A, S, T, lxp, lz0);
            else fwd_rows<R, STORE_A, false>(A, S, T, lxp, lz0);
            if (A.d && T.rec_end > T.rec_begin) sample_from_pool<NT>(A.c, T, A.un, A.d, A.n);
        });
}

// ---------------------------------------------------------------------------
// Adjoint step (see adj_step_kernel): nu^{k+1} with halo, D_nu, kappa and the
// stored a^{k-1} by TMA; the image accumulator is read with plain loads
// issued before the arithmetic (a fifth staged tile would leave room for only
// one stage), the receiver injection tile is built per tile
// (build_injection).
// ---------------------------------------------------------------------------
struct TmaAdjStage {
    STile u;
    CTile d, k, a;
};
constexpr unsigned kAdjStageBytes = sizeof(STile) + 3 * sizeof(CTile);
static_assert(sizeof(TmaAdjStage) == kAdjStageBytes, "stage layout");
constexpr size_t kAdjSmem = 2 * sizeof(TmaAdjStage) + sizeof(PipeTail) + sizeof(CTile);

template <int R, bool FULL>
__device__ __forceinline__ void adj_rows(const AdjArgs &A, const TmaAdjStage &S, const CTile &inj, bool has_rec,
                                         const TileInfo &T, int lxp, int lz0) {
    const int NZ = A.c.NZ;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const int nxw = T.nxw, pitch = T.pitch;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R : min(R, NZ - i0);
    const bool ok = FULL || j < nxw, hi = FULL || j + 1 < nxw;
    float2 gv[R];
#pragma unroll
    for (int rr = 0; rr < R; rr++)
        gv[rr] = (ok && rr < nrow) ? *reinterpret_cast<const float2 *>(A.g + cbase + (long long)rr * pitch)
                                   : make_float2(0.f, 0.f);
    float2 zc[R + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++)
        zc[r] = *reinterpret_cast<const float2 *>(&S.u[lz0 + r][lxp + HALO]);
    float wx0 = 1.f, wx1 = 1.f;
    if constexpr (!FULL) {
        wx0 = sponge1(j, nxw, A.c.nb);
        wx1 = sponge1(j + 1, nxw, A.c.nb);
    }
#pragma unroll
    for (int rr = 0; rr < R; rr++) {
        if (ok && rr < nrow) {
            const f2 a = lap8x2(S.u, zc + rr, lz0 + rr, lxp);
            const f2 nu = pk(zc[rr + HALO]);
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr][lxp]));
            f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[lz0 + rr][lxp]));
            if (has_rec) dv = fma2(kv, pk(*reinterpret_cast<const float2 *>(&inj[lz0 + rr][lxp])), dv);
            const f2 av = pk(*reinterpret_cast<const float2 *>(&S.a[lz0 + rr][lxp]));
            f2 dn, nn;
            if constexpr (FULL) {
                dn = fma2(kv, a, dv);
                nn = add2(nu, dn);
            } else {
                const float wz = sponge1(i0 + rr, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                dn = keep_lo(mul2(w, fma2(kv, a, dv)), hi);
                nn = keep_lo(fma2(w, nu, dn), hi);
            }
            const long long c = cbase + (long long)rr * pitch;
            *reinterpret_cast<f2 *>(A.dd + c) = dn;
            *reinterpret_cast<f2 *>(A.nun + c) = nn;
            *reinterpret_cast<f2 *>(A.g + c) = keep_lo(fma2(av, nn, pk(gv[rr])), hi);
        }
    }
}

template <int R>
__global__ void __launch_bounds__(32 * (TZ / R), 1)
    adj_tma_kernel(AdjArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaAdjStage *st = reinterpret_cast<TmaAdjStage *>(smem_raw);
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + 2 * sizeof(TmaAdjStage));
    CTile &inj = *reinterpret_cast<CTile *>(smem_raw + 2 * sizeof(TmaAdjStage) + sizeof(PipeTail));
    const int tid = threadIdx.x + threadIdx.y * 32;
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;
    run_tiles<2>(
        A.c, kAdjStageBytes, ntiles, st, tail,
        [&](TmaAdjStage &S, unsigned bar, int4 co, int mc) {
            tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.d), &M.m[1], co.z, co.y, co.x, bar);
            tma_load_3d(smem_u32(&S.k), &M.m[2], co.w, co.y, mc, bar);
            tma_load_3d(smem_u32(&S.a), &M.m[3], co.z, co.y, co.x, bar);
        },
        [&](const TmaAdjStage &S, const TileInfo &T) {
            const bool has_rec = T.rec_end > T.rec_begin;
            if (has_rec)
                build_injection<NT>(inj, A.c.recs, T.rec_begin, T.rec_end,
                                    A.r + T.doff + (long long)(A.k - 1) * T.nrec, tid);
            if (T.flags & TI_INTERIOR) adj_rows<R, true>(A, S, inj, has_rec, T, lxp, lz0);
            else adj_rows<R, false>(A, S, inj, has_rec, T, lxp, lz0);
        });
}

// ---------------------------------------------------------------------------
// Born joint step (see born_step_kernel): u0^n and p^n with halos, D_u0,
// D_p, kappa and d kappa by TMA.
// ---------------------------------------------------------------------------
struct TmaBornStage {
    STile u, p;
    CTile du, dp, k, dk;
};
constexpr unsigned kBornStageBytes = 2 * sizeof(STile) + 4 * sizeof(CTile);
static_assert(sizeof(TmaBornStage) == kBornStageBytes, "stage layout");
// NS stages (2: double-buffered, one CTA per SM; 1: two CTAs per SM).
template <int NS>
constexpr size_t born_smem() { return NS * sizeof(TmaBornStage) + sizeof(PipeTail); }
constexpr size_t kBornSmem = born_smem<2>();

template <int R, bool FULL>
__device__ __forceinline__ void born_rows(const BornArgs &A, const TmaBornStage &S, const TileInfo &T, int lxp,
                                          int lz0) {
    const int NZ = A.c.NZ;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const int nxw = T.nxw, pitch = T.pitch;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R : min(R, NZ - i0);
    const bool ok = FULL || j < nxw, hi = FULL || j + 1 < nxw;
    float2 zu[R + 2 * HALO], zp[R + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++) {
        zu[r] = *reinterpret_cast<const float2 *>(&S.u[lz0 + r][lxp + HALO]);
        zp[r] = *reinterpret_cast<const float2 *>(&S.p[lz0 + r][lxp + HALO]);
    }
    float wx0 = 1.f, wx1 = 1.f, q = 0.f;
    if constexpr (!FULL) {
        wx0 = sponge1(j, nxw, A.c.nb);
        wx1 = sponge1(j + 1, nxw, A.c.nb);
        q = A.c.wav[T.wav_off + A.n];
    }
#pragma unroll
    for (int rr = 0; rr < R; rr++) {
        if (ok && rr < nrow) {
            f2 a0 = lap8x2(S.u, zu + rr, lz0 + rr, lxp);
            if constexpr (!FULL) a0 = inject(a0, i0 + rr, j, T.sz, T.sx, q);
            const f2 ap = lap8x2(S.p, zp + rr, lz0 + rr, lxp);
            const f2 duv = pk(*reinterpret_cast<const float2 *>(&S.du[lz0 + rr][lxp]));
            const f2 dpv = pk(*reinterpret_cast<const float2 *>(&S.dp[lz0 + rr][lxp]));
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr][lxp]));
            const f2 dkv = pk(*reinterpret_cast<const float2 *>(&S.dk[lz0 + rr][lxp]));
            f2 du, dp, un, pn;
            if constexpr (FULL) {
                du = fma2(kv, a0, duv);
                dp = fma2(dkv, a0, fma2(kv, ap, dpv));
                un = add2(pk(zu[rr + HALO]), du);
                pn = add2(pk(zp[rr + HALO]), dp);
            } else {
                const float wz = sponge1(i0 + rr, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                du = keep_lo(mul2(w, fma2(kv, a0, duv)), hi);
                dp = keep_lo(mul2(w, fma2(dkv, a0, fma2(kv, ap, dpv))), hi);
                un = keep_lo(fma2(w, pk(zu[rr + HALO]), du), hi);
                pn = keep_lo(fma2(w, pk(zp[rr + HALO]), dp), hi);
            }
            const long long c = cbase + (long long)rr * pitch;
            *reinterpret_cast<f2 *>(A.du + c) = du;
            *reinterpret_cast<f2 *>(A.dp + c) = dp;
            *reinterpret_cast<f2 *>(A.un + c) = un;
            *reinterpret_cast<f2 *>(A.pn + c) = pn;
        }
    }
}

template <int R, int NS>
__global__ void __launch_bounds__(32 * (TZ / R), NS == 1 ? 2 : 1)
    born_tma_kernel(BornArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaBornStage *st = reinterpret_cast<TmaBornStage *>(smem_raw);
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + NS * sizeof(TmaBornStage));
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;
    run_tiles<NS>(
        A.c, kBornStageBytes, ntiles, st, tail,
        [&](TmaBornStage &S, unsigned bar, int4 co, int mc) {
            tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.p), &M.m[1], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.du), &M.m[2], co.z, co.y, co.x, bar);
            tma_load_3d(smem_u32(&S.dp), &M.m[3], co.z, co.y, co.x, bar);
            tma_load_3d(smem_u32(&S.k), &M.m[4], co.w, co.y, mc, bar);
            tma_load_3d(smem_u32(&S.dk), &M.m[5], co.w, co.y, mc, bar);
        },
        [&](const TmaBornStage &S, const TileInfo &T) {
            if (T.flags & TI_FULL_FWD) born_rows<R, true>(A, S, T, lxp, lz0);
            else born_rows<R, false>(A, S, T, lxp, lz0);
            if (T.rec_end > T.rec_begin) sample_from_pool<NT>(A.c, T, A.pn, A.d, A.n);
        });
}

// ---------------------------------------------------------------------------
// Born step from the forward history: the background term a^n = D u0^n + q^n
// that the joint step computes from u0 is read from the a^n the forward pass
// of fwi_gradient / rtm_mig stored at the same model, so only the scattered
// field p is staged and advanced (p^n with its halo, D_p, kappa, d kappa and
// the a^n tile by TMA).  The arithmetic on p is the joint step's, in the same
// order, and the stored a^n has the bits the joint step recomputes, so the
// records are identical.
// ---------------------------------------------------------------------------
struct TmaBornHistStage {
    STile p;
    CTile dp, k, dk, a;
};
constexpr unsigned kBornHistStageBytes = sizeof(STile) + 4 * sizeof(CTile);
static_assert(sizeof(TmaBornHistStage) == kBornHistStageBytes, "stage layout");
constexpr size_t kBornHistSmem = 2 * sizeof(TmaBornHistStage) + sizeof(PipeTail);

template <int R, bool FULL>
__device__ __forceinline__ void born_hist_rows(const BornArgs &A, const TmaBornHistStage &S, const TileInfo &T,
                                               int lxp, int lz0) {
    const int NZ = A.c.NZ;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const int nxw = T.nxw, pitch = T.pitch;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R : min(R, NZ - i0);
    const bool ok = FULL || j < nxw, hi = FULL || j + 1 < nxw;
    float2 zp[R + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++) zp[r] = *reinterpret_cast<const float2 *>(&S.p[lz0 + r][lxp + HALO]);
    float wx0 = 1.f, wx1 = 1.f;
    if constexpr (!FULL) {
        wx0 = sponge1(j, nxw, A.c.nb);
        wx1 = sponge1(j + 1, nxw, A.c.nb);
    }
#pragma unroll
    for (int rr = 0; rr < R; rr++) {
        if (ok && rr < nrow) {
            const f2 a0 = pk(*reinterpret_cast<const float2 *>(&S.a[lz0 + rr][lxp]));
            const f2 ap = lap8x2(S.p, zp + rr, lz0 + rr, lxp);
            const f2 dpv = pk(*reinterpret_cast<const float2 *>(&S.dp[lz0 + rr][lxp]));
            const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr][lxp]));
            const f2 dkv = pk(*reinterpret_cast<const float2 *>(&S.dk[lz0 + rr][lxp]));
            f2 dp, pn;
            if constexpr (FULL) {
                dp = fma2(dkv, a0, fma2(kv, ap, dpv));
                pn = add2(pk(zp[rr + HALO]), dp);
            } else {
                const float wz = sponge1(i0 + rr, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                dp = keep_lo(mul2(w, fma2(dkv, a0, fma2(kv, ap, dpv))), hi);
                pn = keep_lo(fma2(w, pk(zp[rr + HALO]), dp), hi);
            }
            const long long c = cbase + (long long)rr * pitch;
            *reinterpret_cast<f2 *>(A.dp + c) = dp;
            *reinterpret_cast<f2 *>(A.pn + c) = pn;
        }
    }
}

template <int R>
__global__ void __launch_bounds__(32 * (TZ / R), 1)
    born_hist_tma_kernel(BornArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaBornHistStage *st = reinterpret_cast<TmaBornHistStage *>(smem_raw);
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + 2 * sizeof(TmaBornHistStage));
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;
    run_tiles<2>(
        A.c, kBornHistStageBytes, ntiles, st, tail,
        [&](TmaBornHistStage &S, unsigned bar, int4 co, int mc) {
            tma_load_3d(smem_u32(&S.p), &M.m[0], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.dp), &M.m[1], co.z, co.y, co.x, bar);
            tma_load_3d(smem_u32(&S.k), &M.m[2], co.w, co.y, mc, bar);
            tma_load_3d(smem_u32(&S.dk), &M.m[3], co.w, co.y, mc, bar);
            tma_load_3d(smem_u32(&S.a), &M.m[4], co.z, co.y, co.x, bar);
        },
        [&](const TmaBornHistStage &S, const TileInfo &T) {
            // The interior path needs no source test: a^n already holds q^n.
            if (T.flags & TI_INTERIOR) born_hist_rows<R, true>(A, S, T, lxp, lz0);
            else born_hist_rows<R, false>(A, S, T, lxp, lz0);
            if (T.rec_end > T.rec_begin) sample_from_pool<NT>(A.c, T, A.pn, A.d, A.n);
        });
}

// ---------------------------------------------------------------------------
// Self-test of the failure path: one warp waits, with the step kernels'
// bounded wait (~1 s), on an mbarrier that nothing arrives at, and reports
// the timeout in tflag as they do.  Nothing faults and nothing hangs.
// ---------------------------------------------------------------------------
__global__ void wait_timeout_selftest_kernel(unsigned *tflag) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool landed = mbar_wait(b, 0);
    if (!landed && threadIdx.x == 0) atomicExch(tflag, 1u);
}

// ---------------------------------------------------------------------------
// Launchers and occupancy per variant (R = 4, 8, 16 for variants 3, 4, 5).
// ---------------------------------------------------------------------------
// Launch as a programmatic dependent of the previous kernel in the stream.
template <typename Args>
void launch_pdl(void (*kernel)(Args, TileMaps, int), int grid, int R, size_t smem, cudaStream_t s, const Args &a,
                const TileMaps &maps, int ntiles) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, TZ / R);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, a, maps, ntiles);
}

template <int R>
void fwd_launch_r(const FwdArgs &a, int ntiles, int grid, const TileMaps &maps, cudaStream_t s) {
    if (a.a_out) launch_pdl(fwd_tma_kernel<R, true>, grid, R, kFwdSmem, s, a, maps, ntiles);
    else launch_pdl(fwd_tma_kernel<R, false>, grid, R, kFwdSmem, s, a, maps, ntiles);
}

int occupancy(const void *fn, int threads, size_t smem) {
    int n = 0;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
    return n < 1 ? 1 : n;
}

template <int R>
int occ_r(int kind) {
    const int nt = 32 * (TZ / R);
    if (kind == 0) {
        const int a = occupancy((const void *)fwd_tma_kernel<R, true>, nt, kFwdSmem);
        const int b = occupancy((const void *)fwd_tma_kernel<R, false>, nt, kFwdSmem);
        return a < b ? a : b;
    }
    if constexpr (R <= 8) {  // the adjoint and Born kernels have no R = 16 variant
        if (kind == 1) return occupancy((const void *)adj_tma_kernel<R>, nt, kAdjSmem);
        return occupancy((const void *)born_tma_kernel<R, 2>, nt, kBornSmem);
    }
    return 1;
}

}  // namespace

void launch_fwd_step_tma(const FwdArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s) {
    switch (variant) {
    case FIRST_TMA_VARIANT: fwd_launch_r<4>(a, ntiles, grid, maps, s); break;
    case FIRST_TMA_VARIANT + 1: fwd_launch_r<8>(a, ntiles, grid, maps, s); break;
    default: fwd_launch_r<16>(a, ntiles, grid, maps, s); break;
    }
}

void launch_adj_step_tma(const AdjArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s) {
    switch (variant) {
    case FIRST_TMA_VARIANT: launch_pdl(adj_tma_kernel<4>, grid, 4, kAdjSmem, s, a, maps, ntiles); break;
    default: launch_pdl(adj_tma_kernel<8>, grid, 8, kAdjSmem, s, a, maps, ntiles); break;
    }
}

void launch_born_step_tma(const BornArgs &a, int ntiles, int variant, int grid, const TileMaps &maps, cudaStream_t s) {
    switch (variant) {
    case FIRST_TMA_VARIANT: launch_pdl(born_tma_kernel<4, 2>, grid, 4, kBornSmem, s, a, maps, ntiles); break;
    case FIRST_TMA_VARIANT + 1: launch_pdl(born_tma_kernel<8, 2>, grid, 8, kBornSmem, s, a, maps, ntiles); break;
    case FIRST_TMA_VARIANT + 2:
        launch_pdl(born_tma_kernel<4, 1>, grid, 4, born_smem<1>(), s, a, maps, ntiles);
        break;
    default: launch_pdl(born_tma_kernel<8, 1>, grid, 8, born_smem<1>(), s, a, maps, ntiles); break;
    }
}

void launch_born_hist_step(const BornArgs &a, int ntiles, const TileMaps &maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    static int cap = 0;
    if (!cap) {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cap = occupancy((const void *)born_hist_tma_kernel<4>, 32 * (TZ / 4), kBornHistSmem) * nsm;
    }
    launch_pdl(born_hist_tma_kernel<4>, ntiles < cap ? ntiles : cap, 4, kBornHistSmem, s, a, maps, ntiles);
}

void launch_wait_timeout_selftest(unsigned *tflag, cudaStream_t s) {
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(tflag);
}

int tma_occupancy(int kind, int variant) {
    if (kind == 2 && variant == FIRST_TMA_VARIANT + 2)
        return occupancy((const void *)born_tma_kernel<4, 1>, 32 * (TZ / 4), born_smem<1>());
    if (kind == 2 && variant == FIRST_TMA_VARIANT + 3)
        return occupancy((const void *)born_tma_kernel<8, 1>, 32 * (TZ / 8), born_smem<1>());
    switch (variant) {
    case FIRST_TMA_VARIANT: return occ_r<4>(kind);
    case FIRST_TMA_VARIANT + 1: return occ_r<8>(kind);
    default: return kind == 0 ? occ_r<16>(0) : occ_r<8>(kind);
    }
}

}  // namespace dhfwi
