// Finite-difference kernels for sm_103a: forward step (with source injection,
// receiver sampling, checkpoint and segment stores fused), adjoint step (with
// receiver injection and imaging condition fused), Born joint step, model
// preparation, residual/misfit and the shot-ordered image reduction.
//
// Discretisation (Section 2.1 Eq. 1 of arXiv 2403.17518, constant-density
// acoustic): with kappa = v^2 dt^2/h^2, D the unscaled 8th-order Laplacian,
// q^n the source sample at the source node and w the Cerjan sponge factor,
//     a^n = D u^n + q^n,  u^{n+1} = w (2u^n + kappa a^n) - w^2 u^{n-1}.
//
// Adjoint: the exact transpose of that recurrence, written for the scaled
// field nu = kappa w lambda, obeys the same recurrence with the data injected
// where the source is, and gives the velocity gradient (Eq. 13 with the sign
// of dJ/dv) as sum_k (2/v) a^{k-1} nu^k.
//
// Born (Section 2.2 Eqs. 9-11, solved jointly): the tangent of the recurrence
// in v, secondary source w dkappa a0^n with dkappa = 2 kappa dv / v.
#include <cuda_runtime.h>
#include <math.h>

#include "fd_internal.h"

namespace dhfwi {

// 8th-order central second-difference weights for unit spacing.
#define FD_C0 (-205.0f / 72.0f)
#define FD_C1 (8.0f / 5.0f)
#define FD_C2 (-1.0f / 5.0f)
#define FD_C3 (8.0f / 315.0f)
#define FD_C4 (-1.0f / 560.0f)

constexpr int NTHREADS = NTHR_X * NTHR_Z;

typedef float STile[SROWS][SROW];

__device__ __forceinline__ void load_tile(STile &s, const float *__restrict__ f, const ShotDesc &sd,
                                          int NZ, int z0, int x0) {
    const float *base = f + sd.foff;
    const int tid = threadIdx.x + threadIdx.y * NTHR_X;
    for (int idx = tid; idx < SROWS * SROW; idx += NTHREADS) {
        const int r = idx / SROW;
        const int cc = idx - r * SROW;
        const int gz = z0 - HALO + r;
        const int gx = x0 - HALO + cc;
        float val = 0.f;
        if (gz >= 0 && gz < NZ && gx >= 0 && gx < sd.nxw) val = base[(long long)gz * sd.pitch + gx];
        s[r][cc] = val;
    }
}

// D u at tile-local (lz, lx).
__device__ __forceinline__ float lap8(const STile &s, int lz, int lx) {
    const int z = lz + HALO, x = lx + HALO;
    float acc = (2.0f * FD_C0) * s[z][x];
    acc = fmaf(FD_C1, (s[z][x - 1] + s[z][x + 1]) + (s[z - 1][x] + s[z + 1][x]), acc);
    acc = fmaf(FD_C2, (s[z][x - 2] + s[z][x + 2]) + (s[z - 2][x] + s[z + 2][x]), acc);
    acc = fmaf(FD_C3, (s[z][x - 3] + s[z][x + 3]) + (s[z - 3][x] + s[z + 3][x]), acc);
    acc = fmaf(FD_C4, (s[z][x - 4] + s[z][x + 4]) + (s[z - 4][x] + s[z + 4][x]), acc);
    return acc;
}

// Cerjan sponge: exp(-(0.015 (nb - d))^2) per axis, d = cells from the outer edge.
__device__ __forceinline__ float sponge(int i, int NZ, int j, int NXW, int nb) {
    const int dz = min(i, NZ - 1 - i), dx = min(j, NXW - 1 - j);
    const int pz = max(nb - dz, 0), px = max(nb - dx, 0);
    if ((pz | px) == 0) return 1.0f;
    return expf(-2.25e-4f * (float)(pz * pz + px * px));
}

__global__ void __launch_bounds__(NTHREADS) fwd_step_kernel(FwdArgs A) {
    __shared__ STile s;
    __shared__ float so[TZ][TX];
    const Tile t = A.c.tiles[blockIdx.x];
    const ShotDesc sd = A.c.shots[t.slot];
    const int NZ = A.c.NZ;
    load_tile(s, A.u, sd, NZ, t.z0, t.x0);
    __syncthreads();
    const int lx = threadIdx.x;
    const int j = t.x0 + lx;
    const float q = A.c.wav[sd.wav_off + A.n];
#pragma unroll 4
    for (int rr = 0; rr < ROWS_PER_THR; rr++) {
        const int lz = threadIdx.y + rr * NTHR_Z;
        const int i = t.z0 + lz;
        if (i < NZ && j < sd.nxw) {
            const long long c = sd.foff + (long long)i * sd.pitch + j;
            float a = lap8(s, lz, lx);
            if (i == sd.sz && j == sd.sx) a += q;
            const float kap = __ldg(A.c.kap + (long long)i * A.c.pf + sd.x0 + j);
            const float w = sponge(i, NZ, j, sd.nxw, A.c.nb);
            const float uc = s[lz + HALO][lx + HALO];
            const float uold = A.uo[c];
            const float un = w * (2.0f * uc + kap * a) - (w * w) * uold;
            A.uo[c] = un;
            if (A.ck_old) {
                A.ck_old[c] = uold;
                A.ck_cur[c] = uc;
            }
            if (A.a_out) A.a_out[c] = a;
            so[lz][lx] = un;
        }
    }
    if (A.d) {
        const int rb = t.rec_begin, re = A.c.tiles[blockIdx.x + 1].rec_begin;
        if (re > rb) {
            __syncthreads();
            const int tid = threadIdx.x + threadIdx.y * NTHR_X;
            for (int e = rb + tid; e < re; e += NTHREADS) {
                const TileRec tr = A.c.recs[e];
                A.d[sd.doff + (long long)A.n * sd.nrec + tr.r] = so[tr.cell / TX][tr.cell % TX];
            }
        }
    }
}

__global__ void __launch_bounds__(NTHREADS) adj_step_kernel(AdjArgs A) {
    __shared__ STile s;
    __shared__ float inj[TZ][TX];
    const Tile t = A.c.tiles[blockIdx.x];
    const ShotDesc sd = A.c.shots[t.slot];
    const int NZ = A.c.NZ;
    const int tid = threadIdx.x + threadIdx.y * NTHR_X;
    const int rb = t.rec_begin, re = A.c.tiles[blockIdx.x + 1].rec_begin;
    const bool has_rec = re > rb;
    load_tile(s, A.nu, sd, NZ, t.z0, t.x0);
    if (has_rec) {
        for (int e = tid; e < TZ * TX; e += NTHREADS) (&inj[0][0])[e] = 0.f;
        __syncthreads();
        const float *rk = A.r + sd.doff + (long long)(A.k - 1) * sd.nrec;
        for (int e = rb + tid; e < re; e += NTHREADS) {
            const TileRec tr = A.c.recs[e];
            atomicAdd(&inj[tr.cell / TX][tr.cell % TX], rk[tr.r]);
        }
    }
    __syncthreads();
    const int lx = threadIdx.x;
    const int j = t.x0 + lx;
#pragma unroll 4
    for (int rr = 0; rr < ROWS_PER_THR; rr++) {
        const int lz = threadIdx.y + rr * NTHR_Z;
        const int i = t.z0 + lz;
        if (i < NZ && j < sd.nxw) {
            const long long c = sd.foff + (long long)i * sd.pitch + j;
            float a = lap8(s, lz, lx);
            if (has_rec) a += inj[lz][lx];
            const long long mc = (long long)i * A.c.pf + sd.x0 + j;
            const float kap = __ldg(A.c.kap + mc);
            const float v = __ldg(A.c.vpad + mc);
            const float w = sponge(i, NZ, j, sd.nxw, A.c.nb);
            const float nc = s[lz + HALO][lx + HALO];
            const float nold = A.nuo[c];
            const float nn = w * (2.0f * nc + kap * a) - (w * w) * nold;
            A.nuo[c] = nn;
            A.g[c] += (2.0f / v) * A.a[c] * nn;
        }
    }
}

__global__ void __launch_bounds__(NTHREADS) born_step_kernel(BornArgs A) {
    __shared__ STile su;
    __shared__ STile sp;
    __shared__ float so[TZ][TX];
    const Tile t = A.c.tiles[blockIdx.x];
    const ShotDesc sd = A.c.shots[t.slot];
    const int NZ = A.c.NZ;
    load_tile(su, A.u, sd, NZ, t.z0, t.x0);
    load_tile(sp, A.p, sd, NZ, t.z0, t.x0);
    __syncthreads();
    const int lx = threadIdx.x;
    const int j = t.x0 + lx;
    const float q = A.c.wav[sd.wav_off + A.n];
#pragma unroll 4
    for (int rr = 0; rr < ROWS_PER_THR; rr++) {
        const int lz = threadIdx.y + rr * NTHR_Z;
        const int i = t.z0 + lz;
        if (i < NZ && j < sd.nxw) {
            const long long c = sd.foff + (long long)i * sd.pitch + j;
            const long long mc = (long long)i * A.c.pf + sd.x0 + j;
            float a0 = lap8(su, lz, lx);
            if (i == sd.sz && j == sd.sx) a0 += q;
            const float kap = __ldg(A.c.kap + mc);
            const float dk = __ldg(A.dkap + mc);
            const float w = sponge(i, NZ, j, sd.nxw, A.c.nb);
            const float ww = w * w;
            const float un = w * (2.0f * su[lz + HALO][lx + HALO] + kap * a0) - ww * A.uo[c];
            const float pn =
                w * (2.0f * sp[lz + HALO][lx + HALO] + kap * lap8(sp, lz, lx) + dk * a0) - ww * A.po[c];
            A.uo[c] = un;
            A.po[c] = pn;
            so[lz][lx] = pn;
        }
    }
    const int rb = t.rec_begin, re = A.c.tiles[blockIdx.x + 1].rec_begin;
    if (re > rb) {
        __syncthreads();
        const int tid = threadIdx.x + threadIdx.y * NTHR_X;
        for (int e = rb + tid; e < re; e += NTHREADS) {
            const TileRec tr = A.c.recs[e];
            A.d[sd.doff + (long long)A.n * sd.nrec + tr.r] = so[tr.cell / TX][tr.cell % TX];
        }
    }
}

void launch_fwd_step(const FwdArgs &a, int ntiles, cudaStream_t s) {
    if (ntiles > 0) fwd_step_kernel<<<ntiles, dim3(NTHR_X, NTHR_Z), 0, s>>>(a);
}
void launch_adj_step(const AdjArgs &a, int ntiles, cudaStream_t s) {
    if (ntiles > 0) adj_step_kernel<<<ntiles, dim3(NTHR_X, NTHR_Z), 0, s>>>(a);
}
void launch_born_step(const BornArgs &a, int ntiles, cudaStream_t s) {
    if (ntiles > 0) born_step_kernel<<<ntiles, dim3(NTHR_X, NTHR_Z), 0, s>>>(a);
}

// ---------------------------------------------------------------------------
// Model preparation
// ---------------------------------------------------------------------------
__global__ void prep_model_kernel(const float *__restrict__ v, const float *__restrict__ dv, int rel,
                                  int nz, int nx, int nb, float c, float *kap, float *vpad,
                                  float *dkap, int pf, unsigned *status) {
    const int NZ = nz + 2 * nb, NXF = nx + 2 * nb;
    const int pc = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    float kmax = 0.f;
    bool bad = false;
    if (pc < NXF && i < NZ) {
        const int iz = min(max(i - nb, 0), nz - 1);
        const int ix = min(max(pc - nb, 0), nx - 1);
        const float vv = v[(long long)iz * nx + ix];
        bad = !(vv > 0.f) || !isfinite(vv);
        const float k = vv * vv * c;
        const long long o = (long long)i * pf + pc;
        kap[o] = k;
        vpad[o] = vv;
        if (dkap) {
            const float dd = dv[(long long)iz * nx + ix];
            bad = bad || !isfinite(dd);
            dkap[o] = rel ? 2.0f * k * dd : (2.0f * k / vv) * dd;
        }
        kmax = bad ? 0.f : k;
    }
    // Warp reduction of the max and of the bad flag, one atomic per warp.
    for (int off = 16; off > 0; off >>= 1) {
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
        bad = __any_sync(0xffffffffu, bad);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(status, 1u);
        atomicMax(status + 1, __float_as_uint(kmax));
    }
}

void launch_prep_model(const float *v, const float *dv, int rel, int nz, int nx, int nb, float c,
                       float *kap, float *vpad, float *dkap, int pf, unsigned *status,
                       cudaStream_t s) {
    const int NZ = nz + 2 * nb, NXF = nx + 2 * nb;
    dim3 grid((NXF + 127) / 128, NZ);
    prep_model_kernel<<<grid, 128, 0, s>>>(v, dv, rel, nz, nx, nb, c, kap, vpad, dkap, pf, status);
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
    if (rel) acc *= v[(long long)iz * nx + ix];
    out[(long long)iz * nx + ix] = acc;
}

void launch_reduce_image(const ShotDesc *shots, const int *slot_of_shot, int n_shots,
                         const float *gpool, int nz, int nx, int nb, const float *v, int rel,
                         float *out, cudaStream_t s) {
    dim3 grid((nx + 127) / 128, nz);
    reduce_image_kernel<<<grid, 128, 0, s>>>(shots, slot_of_shot, n_shots, gpool, nz, nx, nb, v, rel,
                                             out);
}

}  // namespace dhfwi
