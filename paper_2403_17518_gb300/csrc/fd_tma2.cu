// Two-step (time-blocked) forward kernel for sm_103a: one launch advances
// every active tile by the steps n and n+1 of the recurrence of Section 2.1
// (Eq. 1, summed form, difference-form Laplacian; see fd_kernels.cu), so
// u and D cross HBM once per two updates.
//
// Per 64 x 64 tile the TMA stages u^n with an 8-cell halo (80 x 80) and D^n
// and kappa with a 4-cell ring (72 x 72).  Step n is computed on the tile
// grown by the ring (the core with two columns per thread and R rows, the
// ring as 544 column pairs spread over the CTA), giving u^{n+1} on 72 x 72
// in shared memory (zero outside the window: the Dirichlet boundary) and
// D^{n+1} of the core in registers; step n+1 is then computed on the core
// from them.  The ring cells are recomputed by each tile that needs them, so
// tiles never exchange data within the launch; since they read D^n on their
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
constexpr int NS2 = 1;  // one stage per CTA; two CTAs per SM cover each other's loads
constexpr size_t kFwd2Smem = NS2 * sizeof(Fwd2Stage) + sizeof(ETile) + sizeof(PipeTail);
constexpr int RING_PAIRS = 2 * HALO * (E / 2) + 2 * TZ * (HALO / 2);  // 544 column pairs
static_assert(RING_PAIRS == 544, "ring size");

// Ring pair p -> extended coordinates (ez, ex) of its left cell (ex even).
__device__ __forceinline__ void ring_pair(int p, int &ez, int &ex) {
    constexpr int strip = HALO * (E / 2);  // 144 pairs in the top (bottom) strip
    if (p < 2 * strip) {
        const int q = p < strip ? p : p - strip;
        ez = (p < strip ? 0 : TZ + HALO) + q / (E / 2);
        ex = 2 * (q % (E / 2));
    } else {
        const int q = p - 2 * strip;
        const int side = q / (TZ * (HALO / 2));  // 0 left, 1 right
        const int r = q - side * TZ * (HALO / 2);
        ez = HALO + r / (HALO / 2);
        ex = (side ? TX + HALO : 0) + 2 * (r % (HALO / 2));
    }
}

template <int R, bool STORE_A, bool FULL>
__device__ __forceinline__ void pair_tile(const FwdArgs &A, const Fwd2Stage &S, ETile &V, const TileInfo &T, int lxp,
                                          int lz0, int tid, bool two) {
    constexpr int NT = 32 * (TZ / R);
    const int NZ = A.c.NZ, nb = A.c.nb, nxw = T.nxw, pitch = T.pitch, n = A.n;
    const int j = T.x0 + lxp;
    const int i0 = T.z0 + lz0;
    const long long cbase = T.foff + (long long)i0 * pitch + j;
    const int nrow = FULL ? R : min(R, NZ - i0);
    const bool ok = FULL || j < nxw, hi = FULL || j + 1 < nxw;
    float q0 = 0.f, q1 = 0.f, wx0 = 1.f, wx1 = 1.f;
    if constexpr (!FULL) {
        q0 = A.c.wav[T.wav_off + n];
        q1 = two ? A.c.wav[T.wav_off + n + 1] : 0.f;
        wx0 = sponge1(j, nxw, nb);
        wx1 = sponge1(j + 1, nxw, nb);
    }

    // ---- step n on the core -------------------------------------------
    float2 zc[R + 2 * HALO];
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++)
        zc[r] = *reinterpret_cast<const float2 *>(&S.u[lz0 + HALO + r][lxp + HALO2]);
    f2 dn1[R];
#pragma unroll
    for (int rr = 0; rr < R; rr++) {
        const bool valid = ok && rr < nrow;
        f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&S.u[lz0 + rr + HALO2][lxp + HALO]), zc + rr);
        if constexpr (!FULL) a = inject(a, i0 + rr, j, T.sz, T.sx, q0);
        const f2 u = pk(zc[rr + HALO]);
        const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[lz0 + rr + HALO][lxp + HALO]));
        const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr + HALO][lxp + HALO]));
        f2 dn, un;
        if constexpr (FULL) {
            dn = fma2(kv, a, dv);
            un = add2(u, dn);
        } else {
            const float wz = sponge1(i0 + rr, NZ, nb);
            const f2 w = pk2(wz * wx0, wz * wx1);
            dn = keep_lo(mul2(w, fma2(kv, a, dv)), hi);
            un = keep_lo(fma2(w, u, dn), hi);
            if (!valid) dn = un = 0ull;
        }
        dn1[rr] = dn;
        *reinterpret_cast<f2 *>(&V[lz0 + rr + HALO][lxp + HALO]) = un;
        if (valid) {
            const long long c = cbase + (long long)rr * pitch;
            if (!STORE_A && A.ck_u) {
                *reinterpret_cast<f2 *>(A.ck_u + c) = keep_lo(u, hi);
                *reinterpret_cast<f2 *>(A.ck_d + c) = keep_lo(dv, hi);
            }
            if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out + c) = keep_lo(a, hi);
        }
    }

    // ---- step n on the ring ----------------------------------------------
    for (int p = tid; p < RING_PAIRS; p += NT) {
        int ez, ex;
        ring_pair(p, ez, ex);
        float2 zr[2 * HALO + 1];
#pragma unroll
        for (int r = 0; r <= 2 * HALO; r++) zr[r] = *reinterpret_cast<const float2 *>(&S.u[ez + r][ex + HALO]);
        f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&S.u[ez + HALO][ex]), zr);
        const f2 u = pk(zr[HALO]);
        const f2 dv = pk(*reinterpret_cast<const float2 *>(&S.d[ez][ex]));
        const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[ez][ex]));
        f2 un;
        if constexpr (FULL) {
            un = add2(u, fma2(kv, a, dv));
        } else {
            const int i = T.z0 - HALO + ez, jj = T.x0 - HALO + ex;
            const bool rok = i >= 0 && i < NZ;
            const bool v0 = rok && jj >= 0 && jj < nxw, v1 = rok && jj + 1 >= 0 && jj + 1 < nxw;
            a = inject(a, i, jj, T.sz, T.sx, q0);
            const float wz = sponge1(i, NZ, nb);
            const f2 w = pk2(wz * sponge1(jj, nxw, nb), wz * sponge1(jj + 1, nxw, nb));
            const f2 dn = mul2(w, fma2(kv, a, dv));
            un = fma2(w, u, dn);
            if (!v0) un &= 0xffffffff00000000ull;
            if (!v1) un &= 0x00000000ffffffffull;
        }
        *reinterpret_cast<f2 *>(&V[ez][ex]) = un;
    }
    __syncthreads();  // u^{n+1} complete on the grown tile

    // Receivers: sample n is u^{n+1}.
    if (!STORE_A && A.d) {
        for (int e = T.rec_begin + tid; e < T.rec_end; e += NT) {
            const TileRec tr = A.c.recs[e];
            A.d[T.doff + (long long)n * T.nrec + tr.r] = V[tr.cell / TX + HALO][tr.cell % TX + HALO];
        }
    }
    if (!two) {  // the record ends at n+1: store u^{n+1}, D^{n+1}
#pragma unroll
        for (int rr = 0; rr < R; rr++) {
            if (ok && rr < nrow) {
                const long long c = cbase + (long long)rr * pitch;
                *reinterpret_cast<f2 *>(A.un + c) = *reinterpret_cast<const f2 *>(&V[lz0 + rr + HALO][lxp + HALO]);
                *reinterpret_cast<f2 *>(A.dd_out + c) = dn1[rr];
            }
        }
        return;
    }

    // ---- step n+1 on the core ---------------------------------------------
#pragma unroll
    for (int r = 0; r < R + 2 * HALO; r++) zc[r] = *reinterpret_cast<const float2 *>(&V[lz0 + r][lxp + HALO]);
#pragma unroll
    for (int rr = 0; rr < R; rr++) {
        if (!(ok && rr < nrow)) continue;
        f2 a = lap8x2_seg(reinterpret_cast<const float2 *>(&V[lz0 + rr + HALO][lxp]), zc + rr);
        if constexpr (!FULL) a = inject(a, i0 + rr, j, T.sz, T.sx, q1);
        const f2 u = pk(zc[rr + HALO]);
        const f2 kv = pk(*reinterpret_cast<const float2 *>(&S.k[lz0 + rr + HALO][lxp + HALO]));
        f2 dn, un;
        if constexpr (FULL) {
            dn = fma2(kv, a, dn1[rr]);
            un = add2(u, dn);
        } else {
            const float wz = sponge1(i0 + rr, NZ, nb);
            const f2 w = pk2(wz * wx0, wz * wx1);
            dn = keep_lo(mul2(w, fma2(kv, a, dn1[rr])), hi);
            un = keep_lo(fma2(w, u, dn), hi);
        }
        const long long c = cbase + (long long)rr * pitch;
        *reinterpret_cast<f2 *>(A.dd_out + c) = dn;
        *reinterpret_cast<f2 *>(A.un + c) = un;
        if constexpr (STORE_A) *reinterpret_cast<f2 *>(A.a_out2 + c) = keep_lo(a, hi);
    }
    // Receivers: sample n+1 is u^{n+2}, read back from the pool.
    if (!STORE_A && A.d && T.rec_end > T.rec_begin) sample_from_pool<NT>(A.c, T, A.un, A.d, n + 1);
}

template <bool STORE_A>
__global__ void __launch_bounds__(256, 1) fwd_pair_kernel(FwdArgs A, const __grid_constant__ TileMaps M, int ntiles) {
    constexpr int R = 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Fwd2Stage *st = reinterpret_cast<Fwd2Stage *>(smem_raw);
    ETile &V = *reinterpret_cast<ETile *>(smem_raw + NS2 * sizeof(Fwd2Stage));
    PipeTail *tail = reinterpret_cast<PipeTail *>(smem_raw + NS2 * sizeof(Fwd2Stage) + sizeof(ETile));
    const int tid = threadIdx.x + threadIdx.y * 32;
    const int lxp = 2 * threadIdx.x;
    const int lz0 = threadIdx.y * R;
    run_tiles<NS2>(
        A.c, kFwd2StageBytes, ntiles, st, tail,
        [&](Fwd2Stage &S, unsigned bar, int4 co, int mc) {
            tma_load_3d(smem_u32(&S.u), &M.m[0], co.z - HALO2, co.y - HALO2, co.x, bar);
            tma_load_3d(smem_u32(&S.d), &M.m[1], co.z - HALO, co.y - HALO, co.x, bar);
            tma_load_3d(smem_u32(&S.k), &M.m[2], co.w - HALO, co.y - HALO, mc, bar);
        },
        [&](const Fwd2Stage &S, const TileInfo &T) {
            const bool two = T.nt > A.n + 1;
            if ((T.flags & TI_FULL2) && two) pair_tile<R, STORE_A, true>(A, S, V, T, lxp, lz0, tid, true);
            else pair_tile<R, STORE_A, false>(A, S, V, T, lxp, lz0, tid, two);
        });
}

template <typename K>
void launch_pdl2(K kernel, int grid, const FwdArgs &a, const TileMaps &maps, int ntiles, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32, TZ / 8);
    cfg.dynamicSmemBytes = kFwd2Smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, a, maps, ntiles);
}

int occupancy_of(const void *fn) {
    int n = 0;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwd2Smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 256, kFwd2Smem);
    return n < 1 ? 1 : n;
}

}  // namespace

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
