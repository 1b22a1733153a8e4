// Finite-difference kernels for sm_103a: forward step (with source injection,
// receiver sampling, checkpoint and segment stores fused), adjoint step (with
// receiver injection and imaging condition fused), Born joint step, model
// preparation, residual/misfit and the shot-ordered image reduction.
//
// Discretisation (Section 2.1 Eq. 1 of arXiv 2403.17518, constant-density
// acoustic): with kappa = v^2 dt^2/h^2, D the unscaled 8th-order Laplacian,
// q^n the source sample at the source node and w the Cerjan sponge factor,
//     a^n = D u^n + q^n,  u^{n+1} = w (2u^n + kappa a^n) - w^2 u^{n-1}.
// Computed in FP32 in two algebraically exact rearrangements that keep the
// rounding error of long records small:
//  * summed form: D^{n+1} = w (D^n + kappa a^n), u^{n+1} = w u^n + D^{n+1},
//    with D^n = u^n - w u^{n-1} stored instead of u^{n-1} (the small time
//    difference is never recovered from two nearly equal fields);
//  * difference-form Laplacian: since c0 + 2 sum c_k = 0 on each axis,
//    D u = sum_k c_k [(u_{+k} - u) + (u_{-k} - u)] over both axes, a sum of
//    small terms for smooth fields instead of large cancelling ones.
//
// Adjoint: the exact transpose of the recurrence, written for the scaled
// field nu = kappa w lambda, obeys the same recurrence with the data injected
// where the source is, and gives the velocity gradient (Eq. 13 with the sign
// of dJ/dv) as (2/v) sum_k a^{k-1} nu^k: the step kernels accumulate the sum,
// the image reduction applies 2/v.  The injected data r enter the state
// difference first, D' = D + kappa r (one fma), then D_nu = w (D' + kappa D nu)
// (an exact rearrangement of w (D + kappa (D nu + r))), so that a launch can
// also take the injection from a separate pass over the receivers.
//
// Born (Section 2.2 Eqs. 9-11, solved jointly): the tangent of the recurrence
// in v, secondary source w dkappa a0^n with dkappa = 2 kappa dv / v.
#include <cuda_runtime.h>
#include <math.h>

#include "fd_device.cuh"
#include "fd_internal.h"

namespace dhfwi {

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (16 bytes, zero-filled past src_bytes)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Field tile with halo: rows [z0-4, z0+TZ+4) x columns [x0-4, x0+TX+4) of a
// shot window, zero outside [0,NZ) x [0,nxw).  x0 and the pitch are
// multiples of TX, so every 16-byte chunk is aligned.
template <int NT>
__device__ __forceinline__ void issue_halo_tile(STile &s, const float *__restrict__ f, const ShotDesc &sd,
                                                int NZ, int z0, int x0) {
    const float *base = f + sd.foff;
    const int tid = threadIdx.x + threadIdx.y * 32;
    constexpr int Q = SROW / 4;
    for (int idx = tid; idx < SROWS * Q; idx += NT) {
        const int r = idx / Q;
        const int q = idx - r * Q;
        const int gz = z0 - HALO + r;
        const int gx = x0 - HALO + 4 * q;
        const bool in = gz >= 0 && gz < NZ && gx >= 0 && gx < sd.nxw;
        const int bytes = in ? min(16, 4 * (sd.nxw - gx)) : 0;
        cp_async16(&s[r][4 * q], in ? base + gz * sd.pitch + gx : f, bytes);
    }
}

// Interior tile (rows [z0, z0+TZ), columns [x0, x0+TX)) of a per-shot pool
// (window layout) or of a padded-model array (mcol0 = first model column of
// the window rounded down to a multiple of 4, in the copy shifted by the rest).
template <int NT>
__device__ __forceinline__ void issue_cell_tile(CTile &s, const float *__restrict__ base, int pitch, int NZ,
                                                int nxw, int z0, int x0) {
    const int tid = threadIdx.x + threadIdx.y * 32;
    constexpr int Q = TX / 4;
    for (int idx = tid; idx < TZ * Q; idx += NT) {
        const int r = idx / Q;
        const int q = idx - r * Q;
        const int gz = z0 + r;
        const int gx = x0 + 4 * q;
        const bool in = gz < NZ && gx < nxw;
        const int bytes = in ? min(16, 4 * (nxw - gx)) : 0;
        cp_async16(&s[r][4 * q], in ? base + (long long)gz * pitch + gx : base, bytes);
    }
}


// ---------------------------------------------------------------------------
// Step kernels.  Persistent CTAs walk tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...; the shared-memory stages are double buffered so that the
// asynchronous copies of the next tile overlap the arithmetic of the current
// one.  A warp covers the 64 columns of a tile (two per thread, float2
// shared/global accesses); each thread owns R rows.
// ---------------------------------------------------------------------------
struct FwdStage {
    STile u;
    CTile d, k;
};

template <int R, bool STORE_A>
__global__ void __launch_bounds__(32 * (TZ / R), 1) fwd_step_kernel(FwdArgs A, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdStage *st = reinterpret_cast<FwdStage *>(smem_raw);
    const int NZ = A.c.NZ;
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;

    auto issue = [&](FwdStage &S, int tix) {
        const Tile t = A.c.tiles[tix];
        const ShotDesc sd = A.c.shots[t.slot];
        issue_halo_tile<NT>(S.u, A.u, sd, NZ, t.z0, t.x0);
        issue_cell_tile<NT>(S.d, A.dd + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.k, model_base(A.c.kap, A.c, sd.x0), A.c.pf, NZ, sd.nxw, t.z0, t.x0);
    };

    int k = 0;
    if (blockIdx.x < ntiles) issue(st[0], blockIdx.x);
    cp_async_commit();
    for (int tix = blockIdx.x; tix < ntiles; tix += gridDim.x, k ^= 1) {
        if (tix + (int)gridDim.x < ntiles) issue(st[k ^ 1], tix + gridDim.x);
        cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
        FwdStage &S = st[k];
        const Tile t = A.c.tiles[tix];
        const ShotDesc sd = A.c.shots[t.slot];
        const int j = t.x0 + lxp;
        const int i0 = t.z0 + lz0;
        const int nrow = min(R, NZ - i0);
        const bool ok = j < sd.nxw, hi = j + 1 < sd.nxw;
        const float q = A.c.wav[sd.wav_off + A.n];
        const float wx0 = sponge1(j, sd.nxw, A.c.nb), wx1 = sponge1(j + 1, sd.nxw, A.c.nb);
        float2 zc[R + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R + 2 * HALO; r++) zc[r] = sm2<float2>(&S.u[lz0 + r][lxp + HALO]);
        const long long cbase = sd.foff + (long long)i0 * sd.pitch + j;
        float2 out[R];
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            out[rr] = make_float2(0.f, 0.f);
            if (ok && rr < nrow) {
                const int i = i0 + rr;
                const f2 a = inject(lap8x2(S.u, zc + rr, lz0 + rr, lxp), i, j, sd.sz, sd.sx, q);
                const float wz = sponge1(i, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                const f2 u = pk(zc[rr + HALO]);
                const f2 dv = pk(sm2<float2>(&S.d[lz0 + rr][lxp]));
                const f2 kv = pk(sm2<float2>(&S.k[lz0 + rr][lxp]));
                const f2 dn = keep_lo(mul2(w, fma2(kv, a, dv)), hi);
                const f2 un = keep_lo(fma2(w, u, dn), hi);
                const long long c = cbase + (long long)rr * sd.pitch;
                *reinterpret_cast<f2 *>(A.dd + c) = dn;
                *reinterpret_cast<f2 *>(A.un + c) = un;
                if (!STORE_A && A.ck_u) {
                    *reinterpret_cast<f2 *>(A.ck_u + c) = u;
                    *reinterpret_cast<f2 *>(A.ck_d + c) = dv;
                }
                if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out + c) = keep_lo(a, hi);
                out[rr] = upk(un);
            }
        }
        const Tile tn = A.c.tiles[tix + 1];
        __syncthreads();
        if (A.d && tn.rec_begin > t.rec_begin) {
#pragma unroll
            for (int rr = 0; rr < R; rr++) sm2<float2>(&S.u[lz0 + rr + HALO][lxp + HALO]) = out[rr];
            __syncthreads();
            sample_receivers<NT>(S.u, t, tn, A.c.recs, sd, A.d, A.n);
            __syncthreads();
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

struct AdjStage {
    STile u;
    CTile d, k, a, g;
};

template <int R>
__global__ void __launch_bounds__(32 * (TZ / R), 1) adj_step_kernel(AdjArgs A, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjStage *st = reinterpret_cast<AdjStage *>(smem_raw);
    CTile &inj = *reinterpret_cast<CTile *>(smem_raw + 2 * sizeof(AdjStage));
    const int NZ = A.c.NZ;
    const int tid = threadIdx.x + threadIdx.y * 32;
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;

    auto issue = [&](AdjStage &S, int tix) {
        const Tile t = A.c.tiles[tix];
        const ShotDesc sd = A.c.shots[t.slot];
        issue_halo_tile<NT>(S.u, A.nu, sd, NZ, t.z0, t.x0);
        issue_cell_tile<NT>(S.d, A.dd + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.a, A.a + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.g, A.g + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.k, model_base(A.c.kap, A.c, sd.x0), A.c.pf, NZ, sd.nxw, t.z0, t.x0);
    };

    int k = 0;
    if (blockIdx.x < ntiles) issue(st[0], blockIdx.x);
    cp_async_commit();
    for (int tix = blockIdx.x; tix < ntiles; tix += gridDim.x, k ^= 1) {
        if (tix + (int)gridDim.x < ntiles) issue(st[k ^ 1], tix + gridDim.x);
        cp_async_commit();
        const Tile t = A.c.tiles[tix];
        const Tile tn = A.c.tiles[tix + 1];
        const ShotDesc sd = A.c.shots[t.slot];
        const bool has_rec = tn.rec_begin > t.rec_begin;
        if (has_rec)
            build_injection<NT>(inj, A.c.recs, t.rec_begin, tn.rec_begin,
                                A.r + sd.doff + (long long)(A.k - 1) * sd.nrec, tid);
        cp_async_wait_prev();
        __syncthreads();
        AdjStage &S = st[k];
        const int j = t.x0 + lxp;
        const int i0 = t.z0 + lz0;
        const int nrow = min(R, NZ - i0);
        const bool ok = j < sd.nxw, hi = j + 1 < sd.nxw;
        const float wx0 = sponge1(j, sd.nxw, A.c.nb), wx1 = sponge1(j + 1, sd.nxw, A.c.nb);
        float2 zc[R + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R + 2 * HALO; r++) zc[r] = sm2<float2>(&S.u[lz0 + r][lxp + HALO]);
        const long long cbase = sd.foff + (long long)i0 * sd.pitch + j;
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            if (ok && rr < nrow) {
                const int i = i0 + rr;
                const f2 a = lap8x2(S.u, zc + rr, lz0 + rr, lxp);
                const float wz = sponge1(i, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                const f2 nu = pk(zc[rr + HALO]);
                const f2 kv = pk(sm2<float2>(&S.k[lz0 + rr][lxp]));
                f2 dv = pk(sm2<float2>(&S.d[lz0 + rr][lxp]));
                if (has_rec) dv = fma2(kv, pk(sm2<float2>(&inj[lz0 + rr][lxp])), dv);
                const f2 av = pk(sm2<float2>(&S.a[lz0 + rr][lxp]));
                const f2 gv = pk(sm2<float2>(&S.g[lz0 + rr][lxp]));
                const f2 dn = keep_lo(mul2(w, fma2(kv, a, dv)), hi);
                const f2 nn = keep_lo(fma2(w, nu, dn), hi);
                const long long c = cbase + (long long)rr * sd.pitch;
                *reinterpret_cast<f2 *>(A.dd + c) = dn;
                *reinterpret_cast<f2 *>(A.nun + c) = nn;
                *reinterpret_cast<f2 *>(A.g + c) = keep_lo(fma2(av, nn, gv), hi);
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

struct BornStage {
    STile u, p;
    CTile du, dp, k, dk;
};

template <int R>
__global__ void __launch_bounds__(32 * (TZ / R), 1) born_step_kernel(BornArgs A, int ntiles) {
    constexpr int NT = 32 * (TZ / R);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BornStage *st = reinterpret_cast<BornStage *>(smem_raw);
    const int NZ = A.c.NZ;
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;

    auto issue = [&](BornStage &S, int tix) {
        const Tile t = A.c.tiles[tix];
        const ShotDesc sd = A.c.shots[t.slot];
        issue_halo_tile<NT>(S.u, A.u, sd, NZ, t.z0, t.x0);
        issue_halo_tile<NT>(S.p, A.p, sd, NZ, t.z0, t.x0);
        issue_cell_tile<NT>(S.du, A.du + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.dp, A.dp + sd.foff, sd.pitch, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.k, model_base(A.c.kap, A.c, sd.x0), A.c.pf, NZ, sd.nxw, t.z0, t.x0);
        issue_cell_tile<NT>(S.dk, model_base(A.dkap, A.c, sd.x0), A.c.pf, NZ, sd.nxw, t.z0, t.x0);
    };

    int k = 0;
    if (blockIdx.x < ntiles) issue(st[0], blockIdx.x);
    cp_async_commit();
    for (int tix = blockIdx.x; tix < ntiles; tix += gridDim.x, k ^= 1) {
        if (tix + (int)gridDim.x < ntiles) issue(st[k ^ 1], tix + gridDim.x);
        cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
        BornStage &S = st[k];
        const Tile t = A.c.tiles[tix];
        const ShotDesc sd = A.c.shots[t.slot];
        const int j = t.x0 + lxp;
        const int i0 = t.z0 + lz0;
        const int nrow = min(R, NZ - i0);
        const bool ok = j < sd.nxw, hi = j + 1 < sd.nxw;
        const float q = A.c.wav[sd.wav_off + A.n];
        const float wx0 = sponge1(j, sd.nxw, A.c.nb), wx1 = sponge1(j + 1, sd.nxw, A.c.nb);
        float2 zu[R + 2 * HALO], zp[R + 2 * HALO];
#pragma unroll
        for (int r = 0; r < R + 2 * HALO; r++) {
            zu[r] = sm2<float2>(&S.u[lz0 + r][lxp + HALO]);
            zp[r] = sm2<float2>(&S.p[lz0 + r][lxp + HALO]);
        }
        const long long cbase = sd.foff + (long long)i0 * sd.pitch + j;
        float2 out[R];
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            out[rr] = make_float2(0.f, 0.f);
            if (ok && rr < nrow) {
                const int i = i0 + rr;
                const f2 a0 = inject(lap8x2(S.u, zu + rr, lz0 + rr, lxp), i, j, sd.sz, sd.sx, q);
                const f2 ap = lap8x2(S.p, zp + rr, lz0 + rr, lxp);
                const float wz = sponge1(i, NZ, A.c.nb);
                const f2 w = pk2(wz * wx0, wz * wx1);
                const f2 duv = pk(sm2<float2>(&S.du[lz0 + rr][lxp]));
                const f2 dpv = pk(sm2<float2>(&S.dp[lz0 + rr][lxp]));
                const f2 kv = pk(sm2<float2>(&S.k[lz0 + rr][lxp]));
                const f2 dkv = pk(sm2<float2>(&S.dk[lz0 + rr][lxp]));
                const f2 du = keep_lo(mul2(w, fma2(kv, a0, duv)), hi);
                const f2 dp = keep_lo(mul2(w, fma2(dkv, a0, fma2(kv, ap, dpv))), hi);
                const f2 pn = keep_lo(fma2(w, pk(zp[rr + HALO]), dp), hi);
                const long long c = cbase + (long long)rr * sd.pitch;
                *reinterpret_cast<f2 *>(A.du + c) = du;
                *reinterpret_cast<f2 *>(A.dp + c) = dp;
                *reinterpret_cast<f2 *>(A.un + c) = keep_lo(fma2(w, pk(zu[rr + HALO]), du), hi);
                *reinterpret_cast<f2 *>(A.pn + c) = pn;
                out[rr] = upk(pn);
            }
        }
        const Tile tn = A.c.tiles[tix + 1];
        __syncthreads();
        if (tn.rec_begin > t.rec_begin) {
#pragma unroll
            for (int rr = 0; rr < R; rr++) sm2<float2>(&S.p[lz0 + rr + HALO][lxp + HALO]) = out[rr];
            __syncthreads();
            sample_receivers<NT>(S.p, t, tn, A.c.recs, sd, A.d, A.n);
            __syncthreads();
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

// ---------------------------------------------------------------------------
// Variants (rows per thread) and their launchers.
// ---------------------------------------------------------------------------
namespace {
constexpr int kRows[N_STEP_VARIANTS] = {2, 4, 8, 4, 8, 16, 8};  // the Born kernel's variant 5 has R = 4

constexpr size_t fwd_smem() { return 2 * sizeof(FwdStage); }
constexpr size_t adj_smem() { return 2 * sizeof(AdjStage) + sizeof(CTile); }
constexpr size_t born_smem() { return 2 * sizeof(BornStage); }

template <int R>
void fwd_launch(const FwdArgs &a, int ntiles, int grid, cudaStream_t s) {
    if (a.a_out)
        fwd_step_kernel<R, true><<<grid, dim3(32, TZ / R), fwd_smem(), s>>>(a, ntiles);
    else
        fwd_step_kernel<R, false><<<grid, dim3(32, TZ / R), fwd_smem(), s>>>(a, ntiles);
}
template <int R>
void adj_launch(const AdjArgs &a, int ntiles, int grid, cudaStream_t s) {
    adj_step_kernel<R><<<grid, dim3(32, TZ / R), adj_smem(), s>>>(a, ntiles);
}
template <int R>
void born_launch(const BornArgs &a, int ntiles, int grid, cudaStream_t s) {
    born_step_kernel<R><<<grid, dim3(32, TZ / R), born_smem(), s>>>(a, ntiles);
}

#define DHFWI_DISPATCH(fn, v, ...)        \
    switch (v) {                          \
    case 0: fn<2>(__VA_ARGS__); break;    \
    case 1: fn<4>(__VA_ARGS__); break;    \
    default: fn<8>(__VA_ARGS__); break;   \
    }

template <int R>
int occ_of(int kind, int store_a) {
    int n = 0;
    const int nt = 32 * (TZ / R);
    const void *fn;
    size_t sm;
    if (kind == 0) {
        fn = store_a ? (const void *)fwd_step_kernel<R, true> : (const void *)fwd_step_kernel<R, false>;
        sm = store_a ? fwd_smem() : fwd_smem();
    } else if (kind == 1) {
        fn = (const void *)adj_step_kernel<R>;
        sm = adj_smem();
    } else {
        fn = (const void *)born_step_kernel<R>;
        sm = born_smem();
    }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, sm);
    return n < 1 ? 1 : n;
}
}  // namespace

int step_variant_rows(int v) { return kRows[v]; }

int step_variants(int kind) { return kind == 0 ? 6 : kind == 1 ? 5 : 7; }

int step_occupancy(int kind, int variant, int store_a) {
    if (variant >= FIRST_TMA_VARIANT) return tma_occupancy(kind, variant);
    switch (variant) {
    case 0: return occ_of<2>(kind, store_a);
    case 1: return occ_of<4>(kind, store_a);
    default: return occ_of<8>(kind, store_a);
    }
}

void launch_fwd_step(const FwdArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    const int grid = ntiles < L.max_ctas ? ntiles : L.max_ctas;
    if (L.variant >= FIRST_TMA_VARIANT) {
        launch_fwd_step_tma(a, ntiles, L.variant, grid, *maps, s);
        return;
    }
    DHFWI_DISPATCH(fwd_launch, L.variant, a, ntiles, grid, s);
}
void launch_adj_step(const AdjArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    const int grid = ntiles < L.max_ctas ? ntiles : L.max_ctas;
    if (L.variant >= FIRST_TMA_VARIANT) {
        launch_adj_step_tma(a, ntiles, L.variant, grid, *maps, s);
        return;
    }
    DHFWI_DISPATCH(adj_launch, L.variant, a, ntiles, grid, s);
}
void launch_born_step(const BornArgs &a, int ntiles, const StepLaunch &L, const TileMaps *maps, cudaStream_t s) {
    if (ntiles <= 0) return;
    const int grid = ntiles < L.max_ctas ? ntiles : L.max_ctas;
    if (L.variant >= FIRST_TMA_VARIANT) {
        launch_born_step_tma(a, ntiles, L.variant, grid, *maps, s);
        return;
    }
    DHFWI_DISPATCH(born_launch, L.variant, a, ntiles, grid, s);
}

// ---------------------------------------------------------------------------
// Model preparation
// ---------------------------------------------------------------------------
__global__ void prep_model_kernel(const float *__restrict__ v, const float *__restrict__ dv, int rel,
                                  int nz, int nx, int nb, double c, float *kap, float *dkap, int pf,
                                  long long mstride, unsigned *status) {
    const int NZ = nz + 2 * nb, NXF = nx + 2 * nb;
    const int pc = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    float kmax = 0.f;
    bool bad = false;
    unsigned long long hsum = 0ull;  // identity of v (reuse of a stored forward wavefield)
    if (pc < pf && i < NZ) {
        const int iz = min(max(i - nb, 0), nz - 1);
        // Copy r holds padded-model column pc + r, so that a window starting
        // at any model column reads 16-byte aligned rows from one copy.
        for (int copy = 0; copy < 4; copy++) {
            const int ix = min(max(pc + copy - nb, 0), nx - 1);
            const float vv = v[(long long)iz * nx + ix];
            const bool inside = copy == 0 && pc < NXF;
            bad = bad || (inside && (!(vv > 0.f) || !isfinite(vv)));
            // kappa rounded once from a double product.
            const float k = (float)((double)vv * (double)vv * c);
            const long long o = copy * mstride + (long long)i * pf + pc;
            kap[o] = k;
            if (dkap) {
                const float dd = dv[(long long)iz * nx + ix];
                bad = bad || (inside && !isfinite(dd));
                dkap[o] = rel ? (float)(2.0 * (double)k * (double)dd)
                              : (float)(2.0 * (double)vv * c * (double)dd);
            }
            if (inside && !bad) kmax = k;
            // Each physical cell once: SplitMix64 of (index, value bits),
            // summed mod 2^64 (an order-independent, deterministic total).
            if (copy == 0 && i >= nb && i < nb + nz && pc >= nb && pc < nb + nx) {
                unsigned long long z = ((unsigned long long)((long long)iz * nx + ix) << 32) ^ __float_as_uint(vv);
                z += 0x9E3779B97F4A7C15ull;
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                hsum += z ^ (z >> 31);
            }
        }
    }
    // Warp reduction of the max, the bad flag and the hash, one atomic per warp.
    for (int off = 16; off > 0; off >>= 1) {
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
        bad = __any_sync(0xffffffffu, bad);
        hsum += __shfl_xor_sync(0xffffffffu, hsum, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(status, 1u);
        atomicMax(status + 1, __float_as_uint(kmax));
        atomicAdd(reinterpret_cast<unsigned long long *>(status + 8), hsum);
    }
}

void launch_prep_model(const float *v, const float *dv, int rel, int nz, int nx, int nb, double c,
                       float *kap, float *dkap, int pf, long long mstride, unsigned *status, cudaStream_t s) {
    const int NZ = nz + 2 * nb;
    dim3 grid((pf + 127) / 128, NZ);
    prep_model_kernel<<<grid, 128, 0, s>>>(v, dv, rel, nz, nx, nb, c, kap, dkap, pf, mstride, status);
}

// ---------------------------------------------------------------------------
// Residual and misfit partial sums
// ---------------------------------------------------------------------------
__global__ void residual_kernel(const float *__restrict__ ds, const float *__restrict__ dobs,
                                float *r, long long n, double *partial) {
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = ds[i] - dobs[i];
        r[i] = x;
        acc += (double)x * (double)x;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (threadIdx.x == 0) partial[blockIdx.x] = x;
    }
}

void launch_residual(const float *ds, const float *dobs, float *r, long long n, double *partial,
                     int nblocks, cudaStream_t s) {
    residual_kernel<<<nblocks, 256, 0, s>>>(ds, dobs, r, n, partial);
}

// ---------------------------------------------------------------------------
// Model update along a direction normalised by its max |.|
// ---------------------------------------------------------------------------
__global__ void absmax_bits_kernel(const float *__restrict__ x, long long n, unsigned *out) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void update_model_kernel(const float *__restrict__ v, const float *__restrict__ dir, int nz, int nx,
                                    int mute_rows, float alpha, float vmin, float vmax, const unsigned *mxbits,
                                    float *__restrict__ vout) {
    const long long n = (long long)nz * nx;
    const float mx = __uint_as_float(*mxbits);
    const float sc = mx > 0.f ? alpha / mx : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(i / nx);
        const float d = iz < mute_rows ? 0.f : dir[i];
        vout[i] = fminf(fmaxf(v[i] - sc * d, vmin), vmax);
    }
}

void launch_update_model(const float *v, const float *dir, int nz, int nx, int mute_rows, float alpha, float vmin,
                         float vmax, unsigned *mxbits, float *vout, cudaStream_t s) {
    const long long n = (long long)nz * nx;
    cudaMemsetAsync(mxbits, 0, sizeof(unsigned), s);
    // The normalisation ignores the muted rows.
    const long long off = (long long)mute_rows * nx;
    if (n > off) absmax_bits_kernel<<<512, 256, 0, s>>>(dir + off, n - off, mxbits);
    update_model_kernel<<<512, 256, 0, s>>>(v, dir, nz, nx, mute_rows, alpha, vmin, vmax, mxbits, vout);
}

// ---------------------------------------------------------------------------
// Barzilai-Borwein short step (Eq. 17): per-block float64 partial sums of
// dx . dg and dg . dg (dx = x_k - x_{k-1}, dg = g_k - g_{k-1}, the
// differences taken in float64, so exactly), summed on the host in block
// order.
// ---------------------------------------------------------------------------
__global__ void bb_partials_kernel(const float *__restrict__ xk, const float *__restrict__ xp,
                                   const float *__restrict__ gk, const float *__restrict__ gp, long long n,
                                   double *__restrict__ partial) {
    double sxg = 0.0, sgg = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double dx = (double)xk[i] - (double)xp[i], dg = (double)gk[i] - (double)gp[i];
        sxg += dx * dg;
        sgg += dg * dg;
    }
    for (int off = 16; off > 0; off >>= 1) {
        sxg += __shfl_xor_sync(0xffffffffu, sxg, off);
        sgg += __shfl_xor_sync(0xffffffffu, sgg, off);
    }
    __shared__ double ws[2][32];
    if ((threadIdx.x & 31) == 0) {
        ws[0][threadIdx.x >> 5] = sxg;
        ws[1][threadIdx.x >> 5] = sgg;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < (blockDim.x >> 5);
        double a = in ? ws[0][threadIdx.x] : 0.0, b = in ? ws[1][threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (threadIdx.x == 0) {
            partial[2 * blockIdx.x] = a;
            partial[2 * blockIdx.x + 1] = b;
        }
    }
}

void launch_bb_partials(const float *xk, const float *xp, const float *gk, const float *gp, long long n,
                        double *partial, int nblocks, unsigned *mxbits, cudaStream_t s) {
    bb_partials_kernel<<<nblocks, 256, 0, s>>>(xk, xp, gk, gp, n, partial);
    cudaMemsetAsync(mxbits, 0, sizeof(unsigned), s);
    if (n > 0) absmax_bits_kernel<<<512, 256, 0, s>>>(gk, n, mxbits);
}

// ---------------------------------------------------------------------------
// Image QC filter: out = -(5-point Laplacian of img) / h^2, the grid's edge
// values repeated outside it (zero normal derivative).
// ---------------------------------------------------------------------------
__global__ void image_laplacian_kernel(const float *__restrict__ img, int nz, int nx, float inv_h2,
                                       float *__restrict__ out) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    if (ix >= nx || iz >= nz) return;
    const long long c = (long long)iz * nx + ix;
    const float v = img[c];
    const float up = img[c - (iz > 0 ? nx : 0)], dn = img[c + (iz < nz - 1 ? nx : 0)];
    const float lf = img[c - (ix > 0 ? 1 : 0)], rt = img[c + (ix < nx - 1 ? 1 : 0)];
    out[c] = -(((up - v) + (dn - v)) + ((lf - v) + (rt - v))) * inv_h2;
}

void launch_image_laplacian(const float *img, int nz, int nx, float h, float *out, cudaStream_t s) {
    dim3 grid((nx + 255) / 256, nz);
    image_laplacian_kernel<<<grid, 256, 0, s>>>(img, nz, nx, 1.0f / (h * h), out);
}

// ---------------------------------------------------------------------------
// Image reduction: shots in original order, sponge folded onto edge cells.
// ---------------------------------------------------------------------------
__global__ void reduce_image_kernel(const ShotDesc *__restrict__ shots, const int *__restrict__ slot_of,
                                    int n_shots, const float *__restrict__ gpool, int nz, int nx, int nb,
                                    const float *__restrict__ v, int rel, float *out) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    if (ix >= nx || iz >= nz) return;
    // Padded rows / model columns whose clamped index is (iz, ix).
    const int i_lo = iz == 0 ? 0 : iz + nb;
    const int i_hi = iz == nz - 1 ? nz + 2 * nb - 1 : iz + nb;
    const int c_lo = ix == 0 ? 0 : ix + nb;
    const int c_hi = ix == nx - 1 ? nx + 2 * nb - 1 : ix + nb;
    float acc = 0.f;
    for (int s = 0; s < n_shots; s++) {
        const ShotDesc sd = shots[slot_of[s]];
        const int j_lo = max(c_lo - sd.x0, 0);
        const int j_hi = min(c_hi - sd.x0, sd.nxw - 1);
        if (j_lo > j_hi) continue;
        const float *g = gpool + sd.foff;
        for (int i = i_lo; i <= i_hi; i++)
            for (int j = j_lo; j <= j_hi; j++) acc += g[(long long)i * sd.pitch + j];
    }
    // The imaging factor 2/v is constant in time and equal on the sponge
    // cells folded here (they copy this cell's velocity), so it is applied
    // once; for the relative perturbation v dJ/dv it cancels to 2.
    const float vv = v[(long long)iz * nx + ix];
    out[(long long)iz * nx + ix] = rel ? 2.0f * acc : acc * (float)(2.0 / (double)vv);
}

void launch_reduce_image(const ShotDesc *shots, const int *slot_of_shot, int n_shots,
                         const float *gpool, int nz, int nx, int nb, const float *v, int rel,
                         float *out, cudaStream_t s) {
    dim3 grid((nx + 127) / 128, nz);
    reduce_image_kernel<<<grid, 128, 0, s>>>(shots, slot_of_shot, n_shots, gpool, nz, nx, nb, v, rel,
                                             out);
}

}  // namespace dhfwi
