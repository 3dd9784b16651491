// hjlo_noalloc.cu -- hjlo_step_noalloc: one time step without a plan and
// without any allocation, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a framework whose
// caching allocator must own every device byte, code that runs while another
// thread captures a CUDA graph (cudaMalloc may synchronise the device), and
// latency-bound loops where an allocation's implicit synchronisation is not
// acceptable.  For them this entry point keeps the only scratch memory the
// axis-pass kernel needs -- the kernel tables of each axis and the device
// counters -- in one file-scope static device array, sized for windows of up
// to HJLO_NOALLOC_MAX_WINDOW displacements per axis (about 200 KB, held by
// every GPU that loads the library until the process exits).  The caller
// passes the inputs and the output; the potential term is formed inside the
// kernel from V, so no grid-sized scratch is needed.
//
// The array is shared by every call: a call overwrites the previous call's
// tables and clears the counters before its kernels run.  Calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on the array.  The device error word (a bounded wait that
// ran out, a failed precondition) is not cleared by a step: it collects the
// flags of every step until hjlo_noalloc_status reads and clears it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "hjlo_internal.h"

using namespace hjlo;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kCounterWords = CNT_N + 1;   // counters, then the flags word

// Tables of up to three axes, then the counters and the flags word.
struct NoAllocScratch {
    double kr64[HJLO_MAX_DIM][HJLO_NOALLOC_MAX_WINDOW];
    unsigned long long counters[kCounterWords];
};

static __device__ __align__(256) NoAllocScratch g_scratch;

// Device address of g_scratch per device (host code sees only a stand-in for
// the symbol; the address comes from cudaGetSymbolAddress).
struct ScratchAddr {
    bool ready = false;
    NoAllocScratch *ptr = nullptr;
};
ScratchAddr g_addr[kMaxDevices];
std::mutex g_addr_mu;

hjlo_status scratch_for_current_device(NoAllocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(HJLO_EUNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[dev].ready) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)");
        hjlo_status s = prepare_kernels();
        if (s != HJLO_OK) return s;
        g_addr[dev].ptr = static_cast<NoAllocScratch *>(ptr);
        g_addr[dev].ready = true;
    }
    *out = g_addr[dev].ptr;
    return HJLO_OK;
}

// Window and reversed kernel table of one axis into a caller-provided buffer
// of `cap` doubles (the plans' resolver; no allocation).
hjlo_status table_into(long long N, double dx, double h, double P, long long W, AxisPlan &ax, double *kr64,
                       int cap)
{
    AxisWindow win;
    hjlo_status s = resolve_window(N, dx, h, P, W, win);
    if (s != HJLO_OK) return s;
    if (win.weff > cap)
        return set_error(HJLO_EUNSUPPORTED, "window of %lld displacements exceeds the no-allocation limit %d",
                         win.weff, cap);
    fill_axis_table(N, dx, h, P, win, ax, kr64);
    return HJLO_OK;
}

}  // namespace

extern "C" hjlo_status hjlo_step_noalloc(const hjlo_desc *d, void *cuda_stream, const void *u_in, void *u_out,
                                         const double *V)
{
    if (!d) return set_error(HJLO_EINVAL, "descriptor is NULL");
    if (!u_in || !u_out) return set_error(HJLO_EINVAL, "u_in/u_out is NULL");
    if (d->ndim < 1 || d->ndim > HJLO_MAX_DIM) return set_error(HJLO_EINVAL, "ndim must be 1..3");
    if (d->dtype != HJLO_F64 && d->dtype != HJLO_F32_STORAGE) return set_error(HJLO_EINVAL, "unknown dtype");
    if (d->algo == HJLO_ALGO_DECOMP) return set_error(HJLO_EUNSUPPORTED, "the no-allocation step runs the brute or monotone pass");
    if (d->algo < HJLO_ALGO_AUTO || d->algo > HJLO_ALGO_MONGE) return set_error(HJLO_EINVAL, "unknown algo");
    if (d->reserved != 0) return set_error(HJLO_EINVAL, "reserved field must be 0");
    if (!(d->h > 0) || !std::isfinite(d->h)) return set_error(HJLO_EINVAL, "h must be finite and > 0");
    long long npts = 1;
    for (int a = 0; a < d->ndim; ++a) {
        if (d->shape[a] < 1) return set_error(HJLO_EINVAL, "shape[%d] must be >= 1", a);
        if (d->shape[a] > (1LL << 24)) return set_error(HJLO_EUNSUPPORTED, "shape[%d] too large", a);
        if (!(d->dx[a] > 0) || !std::isfinite(d->dx[a])) return set_error(HJLO_EINVAL, "dx[%d] must be > 0", a);
        if (!std::isfinite(d->P[a])) return set_error(HJLO_EINVAL, "P[%d] must be finite", a);
        npts *= d->shape[a];
        if (npts > (1LL << 40)) return set_error(HJLO_EUNSUPPORTED, "grid too large");
    }
    const int esize = (d->dtype == HJLO_F64) ? 8 : 4;
    if (u_in != u_out) {
        uintptr_t x = (uintptr_t)u_in, y = (uintptr_t)u_out, n = (uintptr_t)npts * esize;
        if (x < y + n && y < x + n) return set_error(HJLO_EINVAL, "u_in and u_out overlap without being equal");
    }

    // host tables on the stack, one axis at a time, copied into the scratch;
    // every window is checked against the limit before any device call
    AxisPlan ax[HJLO_MAX_DIM];
    double host_tab[HJLO_NOALLOC_MAX_WINDOW];
    hjlo_status s;
    for (int a = 0; a < d->ndim; ++a)
        if ((s = table_into(d->shape[a], d->dx[a], d->h, d->P[a], d->window[a], ax[a], host_tab,
                            HJLO_NOALLOC_MAX_WINDOW)) != HJLO_OK)
            return s;
    NoAllocScratch *scr = nullptr;
    if ((s = scratch_for_current_device(&scr)) != HJLO_OK) return s;
    DeviceFacts df;
    if ((s = device_facts(df)) != HJLO_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    for (int a = 0; a < d->ndim; ++a) {
        long long inner = 1, outer = 1;
        for (int b = 0; b < a; ++b) outer *= d->shape[b];
        for (int b = a + 1; b < d->ndim; ++b) inner *= d->shape[b];
        ax[a].inner = inner;
        ax[a].outer = outer;
        if ((s = table_into(d->shape[a], d->dx[a], d->h, d->P[a], d->window[a], ax[a], host_tab,
                            HJLO_NOALLOC_MAX_WINDOW)) != HJLO_OK)
            return s;
        int algo = KALGO_MONGE;
        if (d->algo == HJLO_ALGO_BRUTE) algo = KALGO_BRUTE;
        if (d->algo == HJLO_ALGO_AUTO && (ax[a].weff < 8 || !(ax[a].curv > 0))) algo = KALGO_BRUTE;
        // whole lines only: row blocks cannot run in place and this step owns no scratch
        if ((s = shape_launch(ax[a], esize, algo, df.num_sms, df.smem_optin, 1, nullptr, false)) != HJLO_OK)
            return s;
        apply_test_knobs(ax[a]);
        ax[a].d_kr64 = scr->kr64[a];
        // synchronous with respect to this host buffer for pageable memory
        cudaError_t e = cudaMemcpyAsync(ax[a].d_kr64, host_tab, sizeof(double) * ax[a].weff,
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(no-allocation tables)");
    }
    unsigned long long *counters = scr->counters;
    int *flags = reinterpret_cast<int *>(scr->counters + CNT_N);
    // counters start at zero for this step; the error word keeps earlier
    // steps' flags until hjlo_noalloc_status reads it
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * CNT_N, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(no-allocation counters)");
    for (int a = 0; a < d->ndim; ++a) {
        const bool last = (a == d->ndim - 1);
        s = launch_pass(ax[a], d->dtype, a == 0 ? u_in : u_out, u_out, last ? V : nullptr, last && V ? d->h : 0.0,
                        nullptr, counters, flags, st);
        if (s != HJLO_OK) return s;
    }
    return HJLO_OK;
}

extern "C" hjlo_status hjlo_noalloc_status(void *cuda_stream, hjlo_counters *out)
{
    NoAllocScratch *scr = nullptr;
    hjlo_status s = scratch_for_current_device(&scr);
    if (s != HJLO_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long c[kCounterWords];
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, scr->counters, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "no-allocation status copy");
    int flags = 0;
    memcpy(&flags, &c[CNT_N], sizeof(int));
    if (out) {
        memset(out, 0, sizeof(*out));
        out->exact_rescans = (int64_t)c[CNT_RESCAN];
        out->brute_fallback_lines = (int64_t)c[CNT_FALLBACK];
        out->window_edge_hits = (int64_t)c[CNT_EDGE];
        out->error_flags = flags;
    }
    if (flags) {
        e = cudaMemsetAsync(&scr->counters[CNT_N], 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_error(e, "no-allocation status clear");
        if (flags & FLAG_TIMEOUT) return set_error(HJLO_ETIMEOUT, "a bounded device wait of a no-allocation step gave up");
        return set_error(HJLO_EPRECOND, "a numerical precondition of a no-allocation step failed");
    }
    return HJLO_OK;
}
