// TMA tile pipeline shared by the TMA-staged step kernels (fd_tma.cu,
// fd_tma2.cu): mbarrier and bulk-tensor PTX wrappers, programmatic-launch
// control, the per-CTA tile loop and receiver sampling from a pool.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "fd_device.cuh"
#include "fd_internal.h"

namespace dhfwi {
namespace {


__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity to complete; false after ~1 s.
__device__ __noinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}
// Programmatic dependent launch: wait until the previous kernel in the
// stream has completed and its writes are visible; let the next one start
// its prologue.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// 3-D tiled tensor load into shared memory, completing on bar.  x (the
// column) is always a multiple of 4 floats (16 bytes).
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// 3-D tile of a tensor map prefetched into L2 (no shared memory, nothing to
// wait for); coordinates as for tma_load_3d.
__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap *map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Tile pipeline of the TMA kernels.  Shared memory holds the stages, then
// PipeTail (two mbarriers and the two stages' tile descriptors).  With two
// stages, at tile i every thread waits for stage i mod 2; a barrier then
// certifies that all threads are done with tile i-1, and the leader (thread
// 0) issues tile i+1 into the freed stage: the tensor loads (coordinates
// prefetched into registers one tile earlier) and a cp.async copy of its
// TileInfo into the stage's descriptor slot, awaited before the next barrier.
// With one stage the leader refills it after a barrier that ends the tile.
// The tile's arithmetic then reads the descriptor from shared memory, so no
// dependent global load sits on its critical path.
//
// Launched as programmatic dependents: the prologue (barrier init, first
// descriptors: data no kernel writes) overlaps the previous step kernel, and
// griddepcontrol.wait precedes every access to the fields.
// ---------------------------------------------------------------------------
struct PipeTail {
    unsigned long long bar[2];
    TileInfo desc[2];
};
static_assert(sizeof(TileInfo) == 80 && alignof(TileInfo) == 16, "TileInfo is five 16-byte chunks");
static_assert(sizeof(PipeTail) % 16 == 0, "tail layout");

__device__ __forceinline__ void fetch_coords(const TileInfo *infos, int tix, int4 &co, int &mc) {
    co = __ldg(reinterpret_cast<const int4 *>(&infos[tix].slot));  // slot, z0, x0, mx
    mc = __ldg(&infos[tix].mc);
}
__device__ __forceinline__ void copy_desc(TileInfo *dst, const TileInfo *src) {
#pragma unroll
    for (int q = 0; q < 5; q++) cp_async16(reinterpret_cast<int4 *>(dst) + q, reinterpret_cast<const int4 *>(src) + q);
}

// Runs the CTA's tiles blockIdx.x, blockIdx.x + gridDim.x, ... < ntiles.
// issue_loads(stage, bar, co, mc): the leader's tensor loads of one tile;
// body(stage, desc): the tile's arithmetic (called by every thread).
// NS = 2: double-buffered stages (the next tile loads during this one);
// NS = 1: one stage, refilled after the tile (the latency is covered by the
// other CTAs on the SM).
template <int NS, class Stage, class IssueFn, class BodyFn>
__device__ __forceinline__ void run_tiles(const StepCommon &c, unsigned stage_bytes, int ntiles, Stage *st,
                                          PipeTail *tail, IssueFn issue_loads, BodyFn body) {
    static_assert(NS == 1 || NS == 2, "one or two stages");
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    const unsigned bar0 = smem_u32(&tail->bar[0]);
    const int b = blockIdx.x, g = gridDim.x;
    int4 co = make_int4(0, 0, 0, 0);
    int mc = 0;
    // TMA destinations must be 128-byte aligned; the stage sizes keep them
    // so, only the base is checked (uniform: the whole CTA leaves together).
    if (smem_u32(st) & 127u) {
        if (leader) atomicExch(c.tflag, 2u);
        return;
    }
    if (leader) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_mbar_init();
        fetch_coords(c.infos, b, co, mc);
        copy_desc(&tail->desc[0], &c.infos[b]);
    }
    griddep_wait();
    griddep_launch_dependents();
    unsigned pending = 0;  // leader: stages whose copies have not been seen to land
    auto issue = [&](int s) {
        fence_proxy_async();
        mbar_expect_tx(bar0 + 8 * s, stage_bytes);
        issue_loads(st[s], bar0 + 8 * s, co, mc);
        pending |= 1u << s;
    };
    if (leader) {
        issue(0);
        if (b + g < ntiles) fetch_coords(c.infos, b + g, co, mc);
    }
    __syncthreads();  // barrier init visible before anyone waits
    unsigned phase = 0;
    int k = 0;
    for (int tix = b; tix < ntiles; tix += g, k = NS == 2 ? k ^ 1 : 0) {
        const unsigned par = (phase >> k) & 1u;
        const bool landed = mbar_wait(bar0 + 8 * k, par);
        phase ^= 1u << k;
        if (leader) cp_async_wait_all();  // this stage's descriptor
        if (__syncthreads_or(!landed)) {
            if (leader) {
                // Before the CTA leaves, give its copies still in flight a
                // second bounded wait, so that none lands in shared memory
                // the next CTA on this SM owns.
                for (int s = 0; s < NS; s++)
                    if (pending & (1u << s)) mbar_wait(bar0 + 8 * s, s == k ? par : (phase >> s) & 1u);
                atomicExch(c.tflag, 1u);
            }
            return;
        }
        if (leader) pending &= ~(1u << k);
        if (NS == 2 && leader && tix + g < ntiles) {
            copy_desc(&tail->desc[k ^ 1], &c.infos[tix + g]);
            issue(k ^ 1);
            if (tix + 2 * g < ntiles) fetch_coords(c.infos, tix + 2 * g, co, mc);
        }
        body(st[k], tail->desc[k]);
        if (NS == 1) {
            __syncthreads();  // the stage and its descriptor are free
            if (leader && tix + g < ntiles) {
                copy_desc(&tail->desc[0], &c.infos[tix + g]);
                issue(0);
                if (tix + 2 * g < ntiles) fetch_coords(c.infos, tix + 2 * g, co, mc);
            }
        }
    }
}

// Receivers of a tile, sampled from the pool the tile has just written
// (this CTA's stores are visible to it after the barrier).
template <int NT>
__device__ __forceinline__ void sample_from_pool(const StepCommon &c, const TileInfo &T, const float *__restrict__ f,
                                                 float *__restrict__ d, int n) {
    __syncthreads();
    const int tid = threadIdx.x + threadIdx.y * 32;
    for (int e = T.rec_begin + tid; e < T.rec_end; e += NT) {
        const TileRec tr = c.recs[e];
        const long long cell = T.foff + (long long)(T.z0 + tr.cell / TX) * T.pitch + T.x0 + tr.cell % TX;
        d[T.doff + (long long)n * T.nrec + tr.r] = f[cell];
    }
}

}  // namespace
}  // namespace dhfwi
