// Device helpers shared by the finite-difference step kernels (fd_kernels.cu,
// fd_tma.cu): stencil weights, tile types, packed two-lane FP32 arithmetic,
// the difference-form Laplacian, source injection, the sponge factor and
// receiver sampling.  Formulas: Section 2.1, Eq. 1 (see fd_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "fd_internal.h"

namespace dhfwi {

// 8th-order central second-difference weights for unit spacing (c0 is
// implied by c0 = -2 (c1 + c2 + c3 + c4)).
#define FD_C1 (8.0f / 5.0f)
#define FD_C2 (-1.0f / 5.0f)
#define FD_C3 (8.0f / 315.0f)
#define FD_C4 (-1.0f / 560.0f)

typedef float STile[SROWS][SROW];
typedef float CTile[TZ][TX];

// ---------------------------------------------------------------------------
// Packed two-lane FP32 arithmetic (sm_100+ add/sub/mul/fma .f32x2): lane 0 is
// the low word (float2.x).  Each lane is rounded exactly like the scalar op.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float2 a) { return *reinterpret_cast<f2 *>(&a); }
__device__ __forceinline__ float2 upk(f2 a) { return *reinterpret_cast<float2 *>(&a); }
__device__ __forceinline__ f2 pk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Difference-form D u for the two cells (row lzr, columns lxp, lxp+1) of a
// thread, both lanes at once.  zc holds the two columns for rows lzr-4 ..
// lzr+4 (index 4 = the cells).
// rp: the row segment of the two cells, columns x-4 .. x+5 as five float2
// (the cells are x, x+1); zc: the two columns for rows -4 .. +4.
__device__ __forceinline__ f2 lap8x2_seg(const float2 *rp, const float2 *zc) {
    const float2 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3], r4 = rp[4];
    // r0=(x-4,x-3) r1=(x-2,x-1) r2=(x,x+1) r3=(x+2,x+3) r4=(x+4,x+5)
    const f2 u = pk(r2);
    const f2 m4 = pk(r0), p4 = pk(r4);
    const f2 m3 = pk2(r0.y, r1.x), p3 = pk2(r3.y, r4.x);
    const f2 m2 = pk(r1), p2 = pk(r3);
    const f2 m1 = pk2(r1.y, r2.x), p1 = pk2(r2.y, r3.x);
    const f2 c1 = pk2(FD_C1, FD_C1), c2 = pk2(FD_C2, FD_C2), c3 = pk2(FD_C3, FD_C3), c4 = pk2(FD_C4, FD_C4);
    f2 a = mul2(c4, add2(add2(sub2(p4, u), sub2(m4, u)), add2(sub2(pk(zc[8]), u), sub2(pk(zc[0]), u))));
    a = fma2(c3, add2(add2(sub2(p3, u), sub2(m3, u)), add2(sub2(pk(zc[7]), u), sub2(pk(zc[1]), u))), a);
    a = fma2(c2, add2(add2(sub2(p2, u), sub2(m2, u)), add2(sub2(pk(zc[6]), u), sub2(pk(zc[2]), u))), a);
    a = fma2(c1, add2(add2(sub2(p1, u), sub2(m1, u)), add2(sub2(pk(zc[5]), u), sub2(pk(zc[3]), u))), a);
    return a;
}
__device__ __forceinline__ f2 lap8x2(const STile &s, const float2 *zc, int lzr, int lxp) {
    // Row segment: columns lxp .. lxp+9 (the cells sit at lxp+4, lxp+5).
    return lap8x2_seg(reinterpret_cast<const float2 *>(&s[lzr + HALO][lxp]), zc);
}

// Source injection into lane 0 / 1 of a when the cell is the source node.
__device__ __forceinline__ f2 inject(f2 a, int i, int j, int sz, int sx, float q) {
    if (i == sz && (j == sx || j + 1 == sx)) {
        float2 v = upk(a);
        if (j == sx) v.x += q;
        else v.y += q;
        a = pk(v);
    }
    return a;
}

// Cerjan sponge factor along one axis: exp(-(0.015 (nb - d))^2), d = cells
// from the outer edge; 1 inside.
__device__ __forceinline__ float sponge1(int i, int N, int nb) {
    const int d = min(i, N - 1 - i);
    const int p = nb - d;
    return p > 0 ? expf(-2.25e-4f * (float)(p * p)) : 1.0f;
}

template <int NT>
__device__ __forceinline__ void sample_receivers(const STile &so, const Tile &t, const Tile &tn,
                                                 const TileRec *__restrict__ recs, const ShotDesc &sd,
                                                 float *__restrict__ d, int n) {
    const int tid = threadIdx.x + threadIdx.y * 32;
    for (int e = t.rec_begin + tid; e < tn.rec_begin; e += NT) {
        const TileRec tr = recs[e];
        d[sd.doff + (long long)n * sd.nrec + tr.r] = so[tr.cell / TX + HALO][tr.cell % TX + HALO];
    }
}

// Model arrays are stored as 4 copies, copy r shifted left by r columns, so
// the model row of a window starting at model column x0 is 16-byte aligned in
// copy (x0 & 3) at column (x0 & ~3).
__device__ __forceinline__ const float *model_base(const float *arr, const StepCommon &c, int x0) {
    return arr + (long long)(x0 & 3) * c.mstride + (x0 & ~3);
}

template <typename T>
__device__ __forceinline__ T &sm2(float *p) { return *reinterpret_cast<T *>(p); }

// Receiver injection of one adjoint step into a TZ x TX tile: inj[cell] =
// the sum of the data sample rk[r] over the tile's receivers at that cell,
// zero elsewhere.  A tile's receiver entries are sorted by cell, then by
// receiver, so duplicates are summed in a fixed order by the thread that
// owns the first entry of their cell (deterministic, no atomics).  Ends
// with a barrier.
__device__ __forceinline__ float receiver_sum(const TileRec *__restrict__ recs, int e, int re,
                                              const float *__restrict__ rk) {
    const int cell = recs[e].cell;
    float s = rk[recs[e].r];
    for (int f = e + 1; f < re && recs[f].cell == cell; f++) s += rk[recs[f].r];
    return s;
}
template <int NT>
__device__ __forceinline__ void build_injection(CTile &inj, const TileRec *__restrict__ recs, int rb, int re,
                                                const float *__restrict__ rk, int tid) {
    for (int e = tid; e < TZ * TX; e += NT) (&inj[0][0])[e] = 0.f;
    __syncthreads();
    for (int e = rb + tid; e < re; e += NT)
        if (e == rb || recs[e - 1].cell != recs[e].cell) {
            const int cell = recs[e].cell;
            inj[cell / TX][cell % TX] = receiver_sum(recs, e, re, rk);
        }
    __syncthreads();
}

// Lane 1 (column j+1) cleared when it lies past the window (odd widths), so
// the padding columns of a field pool stay zero: tiles staged straight from
// a pool read them as the zero boundary.
__device__ __forceinline__ f2 keep_lo(f2 v, bool hi) { return hi ? v : (v & 0xffffffffull); }

}  // namespace dhfwi
