// hjlo_persist.cuh -- the persistent batched pass: all passes of one time
// step of every instance of a batch in one launch (see pass_kernel_persist).
#pragma once

#include "hjlo_device.cuh"

namespace hjlo {

// The dynamic shared memory of the pass kernels.
__device__ __forceinline__ unsigned char *pass_smem()
{
    extern __shared__ __align__(128) unsigned char smem[];
    return smem;
}


// One work item of the persistent batched pass: tiles [tile0, tile0 + ntile)
// of instance `inst` on axis `axis`, launch shape `shape` (a (group, axis)
// entry of PersistParams::shapes).
struct PersistItem {
    int shape, inst, axis, tile0, ntile, pad;
};

struct PersistParams {
    const PersistItem *work;   // every axis-a item comes before any axis-(a+1) item
    long long nwork;
    const PassParams *shapes;  // shared launch fields per (group, axis)
    const BatchItem *items;    // per (axis, instance): [axis * count + inst]
    const int *tiles;          // per (instance, axis): tiles of that pass
    unsigned long long *queue; // next work item (0 before the launch)
    unsigned *done;            // per (instance, axis): tiles finished (0 before the launch)
    int *flags;
    int count, ndim;
    long long wait_ns;         // bound on a dependency wait
    int test_extra_dep;        // test knob: tiles a dependency wait expects beyond the real count (0 in use)
    int pad;
};

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// All passes of one time step of every instance in one launch: CTAs take
// work items in queue order; an item of axis a >= 1 first waits (thread 0,
// bounded by the global timer) until every tile of the instance's axis a - 1
// pass is finished, since that pass writes the grid this one reads.  The
// waits only ever point at items taken earlier, by CTAs that are running,
// so the launch cannot deadlock whatever the grid size.  A wait that runs
// out raises FLAG_TIMEOUT and the item (and every later wait) is skipped.
// Every instance runs the monotone search.  The launch's thread count and
// shared memory are the largest over the shapes; a shape with fewer threads
// leaves the extra ones idle in its tiles.
template <typename T>
__global__ void __launch_bounds__(1024) pass_kernel_persist(const __grid_constant__ PersistParams pp)
{
    __shared__ PassParams s_p;
    __shared__ PersistItem s_it;
    __shared__ long long s_w;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const long long w = (long long)atomicAdd(pp.queue, 1ull);
            int ok = 0;
            if (w < pp.nwork) {
                const PersistItem it = pp.work[w];
                s_it = it;
                ok = 1;
                if (it.axis > 0) {
                    const volatile unsigned *d = pp.done + (size_t)it.inst * pp.ndim + it.axis - 1;
                    const unsigned need =
                        (unsigned)(pp.tiles[(size_t)it.inst * pp.ndim + it.axis - 1] + pp.test_extra_dep);
                    const unsigned long long t0 = global_ns();
                    while (*d < need) {
                        if (*(const volatile int *)pp.flags & FLAG_TIMEOUT) { ok = 0; break; }
                        if ((long long)(global_ns() - t0) > pp.wait_ns) {
                            atomicOr(pp.flags, FLAG_TIMEOUT);
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                    // the previous pass's stores (generic proxy) before this
                    // pass's bulk copies (async proxy) read them
                    __threadfence();
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
            }
            s_w = w;
            s_ok = ok;
        }
        __syncthreads();
        const long long w = s_w;
        if (w >= pp.nwork) break;
        const PersistItem it = s_it;
        if (s_ok) {
            // the item's launch fields, then its instance's
            const unsigned *sw = reinterpret_cast<const unsigned *>(pp.shapes + it.shape);
            unsigned *dw = reinterpret_cast<unsigned *>(&s_p);
            for (int k = tid; k < (int)(sizeof(PassParams) / 4); k += blockDim.x) dw[k] = sw[k];
            __syncthreads();
            const BatchItem *bi = pp.items + (size_t)it.axis * pp.count + it.inst;
            if (tid == 0) {
                s_p.src = bi->src;
                s_p.dst = bi->dst;
                s_p.hv = bi->hv;
                s_p.kr64 = bi->kr64;
                s_p.kmax = bi->kmax;
                s_p.curv = bi->curv;
                s_p.hoff = bi->hoff;
                s_p.dhi = bi->dhi;
                s_p.use_tma = bi->use_tma;
                if (bi->use_tma && s_p.inner != 1)
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&bi->tmap)
                                 : "memory");
            }
            __syncthreads();
            const bool contig = (s_p.inner == 1);
            for (int t = 0; t < it.ntile; ++t) {
                if (contig)
                    pass_tile<T, LAYOUT_CONTIG, KALGO_MONGE>(&bi->tmap, s_p, it.tile0 + t);
                else
                    pass_tile<T, LAYOUT_STRIDED, KALGO_MONGE>(&bi->tmap, s_p, it.tile0 + t);
                __syncthreads();
                if (tid == 0) mbar_inval(reinterpret_cast<uint64_t *>(pass_smem() + s_p.off_misc));
                __syncthreads();
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(pp.done + (size_t)it.inst * pp.ndim + it.axis, (unsigned)it.ntile);
        }
    }
}

}  // namespace hjlo
