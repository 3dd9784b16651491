// hjlo_api.cu -- the C ABI declared in include/hjlo.h: plans, one step, the
// time loop of eq. uN (replayed from a CUDA graph), the end-to-end host
// variant, the effective-Hamiltonian readout of Prop. prop:klm and status.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hjlo_internal.h"

using namespace hjlo;

namespace {

constexpr int kGraphSteps = 16;  // steps per captured graph

}  // namespace

namespace {

__global__ void scale_kernel(const double *__restrict__ V, double h, double *__restrict__ hv, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        hv[i] = __dmul_rn(h, V[i]);
}

constexpr int kReduceBlocks = 512;
constexpr int kReduceThreads = 256;

template <typename T>
__device__ __forceinline__ double as_f64(T x) { return (double)x; }

// Per-block partial (sum, min, max) of un - u0 in a fixed order; the second
// kernel folds the partials in block order, so the readout is deterministic.
template <typename T>
__global__ void diff_partials(const T *__restrict__ u0, const T *__restrict__ un, long long n,
                              double *__restrict__ part)
{
    __shared__ double ss[kReduceThreads], smn[kReduceThreads], smx[kReduceThreads];
    double s = 0.0, mn = INFINITY, mx = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double d = __dsub_rn(as_f64(un[i]), as_f64(u0[i]));
        s = __dadd_rn(s, d);
        mn = fmin(mn, d);
        mx = fmax(mx, d);
    }
    ss[threadIdx.x] = s;
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int o = kReduceThreads / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] = __dadd_rn(ss[threadIdx.x], ss[threadIdx.x + o]);
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = ss[0];
        part[3 * blockIdx.x + 1] = smn[0];
        part[3 * blockIdx.x + 2] = smx[0];
    }
}

__global__ void fold_partials(double *part, int nblocks)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, mn = INFINITY, mx = -INFINITY;
    for (int b = 0; b < nblocks; ++b) {
        s = __dadd_rn(s, part[3 * b]);
        mn = fmin(mn, part[3 * b + 1]);
        mx = fmax(mx, part[3 * b + 2]);
    }
    part[3 * nblocks + 0] = s;
    part[3 * nblocks + 1] = mn;
    part[3 * nblocks + 2] = mx;
}

hjlo_status check_plan(const hjlo_plan *p)
{
    if (!p) return set_error(HJLO_EINVAL, "plan is NULL");
    return HJLO_OK;
}

hjlo_status set_device(const hjlo_plan *p)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) {
        cudaError_t e = cudaSetDevice(p->device);
        if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    }
    return HJLO_OK;
}

bool ranges_overlap(const void *a, const void *b, size_t n)
{
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
}

// All passes of one step.  src -> dst for axis 0, then in place on dst.  An
// axis in row blocks cannot run in place: a block stages its rows' window
// span, which holds rows of other blocks, and a block that starts late would
// read rows another block has already written (the same holds for the
// write-back blocks of a decomposition cut across CTAs).  Such a pass writes
// to the plan's scratch and is copied back (stream-ordered, so graphs
// capture it).
hjlo_status enqueue_step(hjlo_plan *p, const void *src, void *dst, const double *hv, double hv_scale,
                         int32_t *amin, cudaStream_t st)
{
    const size_t bytes = (size_t)p->npts * p->esize;
    for (int a = 0; a < p->ndim; ++a) {
        const bool last = (a == p->ndim - 1);
        const void *from = (a == 0) ? src : dst;
        const bool via_scratch = (p->ax[a].vblocks > 1 || p->ax[a].dsplit) && ranges_overlap(from, dst, bytes);
        if (via_scratch && !p->d_scratch) return set_error(HJLO_ECUDA, "row-block scratch missing");
        hjlo_status s = launch_pass(p->ax[a], p->dtype, from, via_scratch ? p->d_scratch : dst, last ? hv : nullptr,
                                    last ? hv_scale : 0.0, amin ? amin + (long long)a * p->npts : nullptr,
                                    p->d_counters, p->d_flags, st);
        if (s != HJLO_OK) return s;
        if (via_scratch) {
            cudaError_t e = cudaMemcpyAsync(dst, p->d_scratch, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_error(e, "row-block copy");
        }
    }
    return HJLO_OK;
}

// nsteps steps in place on u (V: nsteps rows, one per step, when tv; else
// hv for every step).  Passes in row blocks alternate between u and the
// plan's scratch instead of copying back after each one; the state is copied
// to u at the end only when an odd number of them ran.
hjlo_status enqueue_steps(hjlo_plan *p, void *u, const double *V, bool tv, long long nsteps, cudaStream_t st)
{
    void *cur = u;
    for (long long n = 0; n < nsteps; ++n) {
        const double *v = tv ? (V ? V + n * p->npts : nullptr) : V;
        for (int a = 0; a < p->ndim; ++a) {
            const bool last = (a == p->ndim - 1);
            void *next = cur;
            if (p->ax[a].vblocks > 1 || p->ax[a].dsplit) {
                if (!p->d_scratch) return set_error(HJLO_ECUDA, "row-block scratch missing");
                next = (cur == u) ? p->d_scratch : u;
            }
            hjlo_status s = launch_pass(p->ax[a], p->dtype, cur, next, last ? v : nullptr,
                                        (last && tv) ? p->desc.h : 0.0, nullptr, p->d_counters, p->d_flags, st);
            if (s != HJLO_OK) return s;
            cur = next;
        }
    }
    if (cur != u) {
        cudaError_t e = cudaMemcpyAsync(u, cur, (size_t)p->npts * p->esize, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "row-block copy");
    }
    return HJLO_OK;
}

hjlo_status ensure_hv(hjlo_plan *p)
{
    if (p->d_hv) return HJLO_OK;
    cudaError_t e = cudaMalloc(&p->d_hv, sizeof(double) * p->npts);
    if (e != cudaSuccess) { p->d_hv = nullptr; return cuda_error(e, "cudaMalloc(h*V)"); }
    return HJLO_OK;
}

hjlo_status form_hv(hjlo_plan *p, const double *V)
{
    hjlo_status s = ensure_hv(p);
    if (s != HJLO_OK) return s;
    long long blocks = std::min<long long>((p->npts + 255) / 256, 4096);
    scale_kernel<<<(unsigned)blocks, 256, 0, p->stream>>>(V, p->desc.h, p->d_hv, p->npts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "h*V kernel launch");
    return HJLO_OK;
}

void destroy_graph(hjlo_plan *p)
{
    if (p->graph.exec) cudaGraphExecDestroy(p->graph.exec);
    p->graph = GraphCache();
}

hjlo_status capture_graph(hjlo_plan *p, void *u, const double *hv)
{
    destroy_graph(p);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
    hjlo_status s = enqueue_steps(p, u, hv, false, kGraphSteps, p->cap_stream);
    e = cudaStreamEndCapture(p->cap_stream, &g);
    if (s != HJLO_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->graph.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { p->graph.exec = nullptr; return cuda_error(e, "cudaGraphInstantiate"); }
    p->graph.u = u;
    p->graph.hv = hv;
    return HJLO_OK;
}

hjlo_status run_impl(hjlo_plan *p, void *u, const double *V, long long nsteps, bool tv)
{
    const double *hv = nullptr;
    if (V && !tv) {
        hjlo_status s = form_hv(p, V);
        if (s != HJLO_OK) return s;
        hv = p->d_hv;
    }
    long long n = 0;
    if (!tv && nsteps >= 2 * kGraphSteps) {
        if (!p->graph.exec || p->graph.u != u || p->graph.hv != hv) {
            hjlo_status s = capture_graph(p, u, hv);
            if (s != HJLO_OK) return s;
        }
        for (; n + kGraphSteps <= nsteps; n += kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(p->graph.exec, p->stream);
            if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
        }
    }
    if (n < nsteps) {
        hjlo_status s = tv ? enqueue_steps(p, u, V ? V + n * p->npts : nullptr, true, nsteps - n, p->stream)
                           : enqueue_steps(p, u, hv, false, nsteps - n, p->stream);
        if (s != HJLO_OK) return s;
    }
    p->steps += nsteps;
    return HJLO_OK;
}

}  // namespace

namespace hjlo {
hjlo_status plan_enqueue_step(hjlo_plan *p, const void *src, void *dst, const double *hv, double hv_scale,
                              int32_t *amin, cudaStream_t st)
{
    return enqueue_step(p, src, dst, hv, hv_scale, amin, st);
}
hjlo_status plan_form_hv(hjlo_plan *p, const double *V) { return form_hv(p, V); }
hjlo_status plan_run(hjlo_plan *p, void *u, const double *V, long long nsteps)
{
    return run_impl(p, u, V, nsteps, false);
}
hjlo_status plan_set_device(const hjlo_plan *p) { return set_device(p); }
}  // namespace hjlo

extern "C" {

int32_t hjlo_version(void) { return HJLO_VERSION; }

hjlo_status hjlo_shape_query(int64_t N, int64_t lines, int64_t weff, int32_t esize, int32_t algo, int32_t num_sms,
                             int64_t smem_optin, hjlo_shape_info *out)
{
    clear_error();
    if (!out || N < 1 || N > (1LL << 30) || lines < 1 || weff < 1 || weff > N ||
        (esize != 8 && esize != 4) ||
        (algo != HJLO_ALGO_BRUTE && algo != HJLO_ALGO_MONGE && algo != HJLO_ALGO_DECOMP) ||
        (algo == HJLO_ALGO_DECOMP && esize != 8) || num_sms < 1 || smem_optin < 1024)
        return set_error(HJLO_EINVAL, "invalid shape query");
    if (weff > 65535) return set_error(HJLO_EUNSUPPORTED, "window of %lld displacements exceeds 65535", (long long)weff);
    AxisPlan ax;
    ax.N = N;
    ax.inner = 1;
    ax.outer = lines;
    ax.weff = (int)weff;
    ax.hoff = 0;
    ax.curv = 1.0;                               // a strictly convex table (the decomposition pass needs one)
    memset(out, 0, sizeof(*out));
    if (algo == HJLO_ALGO_DECOMP) {
        hjlo_status s = shape_decomp(ax, (size_t)smem_optin, num_sms);
        if (s != HJLO_OK) return s;
        const bool blocks = ax.vblocks > 1;
        out->lanes_per_line = ax.threads;        // one CTA per line or row block
        out->segment_rows = 0;
        out->lines_per_tile = 1;
        out->threads = ax.threads;
        out->smem_bytes = (int64_t)ax.smem;
        out->tiles = ax.ntiles;
        out->row_blocks = ax.vblocks;
        out->block_rows = blocks ? ax.vR : 0;
        out->line_points = blocks ? ax.vR + weff - 1 : N;
        out->split_chunks = ax.dsplit ? ax.dB : 0;
        out->split_rows = ax.dsplit ? ax.dvR : 0;
        return HJLO_OK;
    }
    hjlo_status s = shape_launch(ax, esize, algo == HJLO_ALGO_BRUTE ? KALGO_BRUTE : KALGO_MONGE, num_sms,
                                 (size_t)smem_optin);
    if (s != HJLO_OK) return s;
    out->lanes_per_line = ax.lpl;
    out->segment_rows = ax.seg;
    out->lines_per_tile = ax.C;
    out->threads = ax.threads;
    out->smem_bytes = (int64_t)ax.smem;
    out->tiles = ax.ntiles;
    out->row_blocks = ax.vblocks;
    out->block_rows = (ax.vblocks > 1) ? ax.vR : 0;
    out->line_points = (ax.vblocks > 1) ? ax.vNp : N;
    return HJLO_OK;
}

const char *hjlo_last_error(void) { return last_error_cstr(); }

hjlo_status hjlo_plan_create(const hjlo_desc *d, void *cuda_stream, hjlo_plan **out)
{
    if (!out) return set_error(HJLO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d) return set_error(HJLO_EINVAL, "descriptor is NULL");
    if (d->ndim < 1 || d->ndim > HJLO_MAX_DIM) return set_error(HJLO_EINVAL, "ndim must be 1..3");
    if (d->dtype != HJLO_F64 && d->dtype != HJLO_F32_STORAGE) return set_error(HJLO_EINVAL, "unknown dtype");
    if (d->algo < HJLO_ALGO_AUTO || d->algo > HJLO_ALGO_DECOMP) return set_error(HJLO_EINVAL, "unknown algo");
    if (d->algo == HJLO_ALGO_DECOMP && d->dtype != HJLO_F64)
        return set_error(HJLO_EUNSUPPORTED, "the decomposition method runs in binary64 storage only");
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
    DeviceFacts df;
    hjlo_status s = device_facts(df);
    if (s != HJLO_OK) return s;
    if ((s = prepare_kernels()) != HJLO_OK) return s;

    hjlo_plan *p = new (std::nothrow) hjlo_plan();
    if (!p) return set_error(HJLO_ENOMEM, "host allocation");
    p->desc = *d;
    p->ndim = d->ndim;
    p->dtype = d->dtype;
    p->npts = npts;
    p->esize = (d->dtype == HJLO_F64) ? 8 : 4;
    p->stream = (cudaStream_t)cuda_stream;
    p->device = df.device;
    bool all_monge = true;
    for (int a = 0; a < p->ndim; ++a) {
        AxisPlan &ax = p->ax[a];
        long long inner = 1, outer = 1;
        for (int b = 0; b < a; ++b) outer *= d->shape[b];
        for (int b = a + 1; b < p->ndim; ++b) inner *= d->shape[b];
        ax.inner = inner;
        ax.outer = outer;
        double *k64 = nullptr;
        s = resolve_axis(d->shape[a], d->dx[a], d->h, d->P[a], d->window[a], ax, &k64);
        if (s != HJLO_OK) { hjlo_plan_destroy(p); return s; }
        int algo = KALGO_MONGE;
        if (d->algo == HJLO_ALGO_BRUTE) algo = KALGO_BRUTE;
        if (d->algo == HJLO_ALGO_AUTO && (ax.weff < 8 || !(ax.curv > 0))) algo = KALGO_BRUTE;
        if (d->algo == HJLO_ALGO_DECOMP) algo = KALGO_DECOMP;
        s = (algo == KALGO_DECOMP) ? shape_decomp(ax, df.smem_optin, df.num_sms)
                                   : shape_launch(ax, p->esize, algo, df.num_sms, df.smem_optin);
        if (s == HJLO_EUNSUPPORTED && algo == KALGO_MONGE && d->algo == HJLO_ALGO_AUTO) {
            // a line too long for the monotone search's shared-memory layout:
            // brute force needs only the line and its argmins on chip
            algo = KALGO_BRUTE;
            s = shape_launch(ax, p->esize, algo, df.num_sms, df.smem_optin);
        }
        if (algo != KALGO_MONGE) all_monge = false;
        apply_test_knobs(ax);
        if (s == HJLO_OK) s = dmalloc((void **)&ax.d_kr64, sizeof(double) * ax.weff, "cudaMalloc(kernel table)");
        if (s == HJLO_OK && ax.dsplit) {
            ax.split_bytes = split_scratch_bytes(ax);
            s = dmalloc(&ax.d_split, ax.split_bytes, "cudaMalloc(decomposition scratch)");
        }
        if (s == HJLO_OK) {
            cudaError_t e = cudaMemcpy(ax.d_kr64, k64, sizeof(double) * ax.weff, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) s = cuda_error(e, "kernel table upload");
        }
        if (s == HJLO_OK) s = split_prepare(ax, p->stream);
        free(k64);
        if (s != HJLO_OK) { hjlo_plan_destroy(p); return s; }
    }
    p->algo = (d->algo == HJLO_ALGO_DECOMP) ? HJLO_ALGO_DECOMP : (all_monge ? HJLO_ALGO_MONGE : HJLO_ALGO_BRUTE);
    bool blocks = false;
    for (int a = 0; a < p->ndim; ++a) blocks = blocks || p->ax[a].vblocks > 1 || p->ax[a].dsplit;
    s = blocks ? dmalloc(&p->d_scratch, (size_t)p->npts * p->esize, "cudaMalloc(row-block scratch)") : HJLO_OK;
    if (s != HJLO_OK) { hjlo_plan_destroy(p); return s; }
    s = dmalloc((void **)&p->d_counters, sizeof(unsigned long long) * CNT_N, "cudaMalloc(counters)");
    if (s == HJLO_OK) s = dmalloc((void **)&p->d_flags, sizeof(int), "cudaMalloc(flags)");
    if (s != HJLO_OK) { hjlo_plan_destroy(p); return s; }
    cudaError_t e = cudaMemset(p->d_counters, 0, sizeof(unsigned long long) * CNT_N);
    if (e == cudaSuccess) e = cudaMemset(p->d_flags, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { s = cuda_error(e, "plan allocation"); hjlo_plan_destroy(p); return s; }
    *out = p;
    return HJLO_OK;
}

hjlo_status hjlo_plan_destroy(hjlo_plan *p)
{
    if (!p) return HJLO_OK;
    set_device(p);
    if (p->stream || p->cap_stream) cudaStreamSynchronize(p->stream);
    destroy_graph(p);
    for (int a = 0; a < HJLO_MAX_DIM; ++a) {
        cudaFree(p->ax[a].d_kr64);
        cudaFree(p->ax[a].d_split);
    }
    cudaFree(p->d_counters);
    cudaFree(p->d_flags);
    cudaFree(p->d_hv);
    cudaFree(p->d_part);
    cudaFree(p->d_u_host_run);
    cudaFree(p->d_scratch);
    cudaFree(p->d_V_host_run);
    cudaFree(p->d_ckpt);
    cudaFree(p->d_amin);
    cudaFree(p->d_work);
    cudaFree(p->d_pbar_part);
    cudaFree(p->d_proj);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
    return HJLO_OK;
}

hjlo_status hjlo_plan_info(const hjlo_plan *p, hjlo_plan_facts *info)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!info) return set_error(HJLO_EINVAL, "info is NULL");
    memset(info, 0, sizeof(*info));
    info->ndim = p->ndim;
    info->algo = p->algo;
    info->npts = p->npts;
    for (int a = 0; a < p->ndim; ++a) {
        info->dlo[a] = p->ax[a].dlo;
        info->dhi[a] = p->ax[a].dhi;
        info->centre[a] = p->ax[a].centre;
        info->kmin[a] = p->ax[a].kmin;
        info->curvature[a] = p->ax[a].curv;
        info->row_blocks[a] = p->ax[a].vblocks;
        info->block_rows[a] = (p->ax[a].vblocks > 1) ? p->ax[a].vR : 0;
        info->split_chunks[a] = p->ax[a].dsplit ? p->ax[a].dB : 0;
    }
    return HJLO_OK;
}

hjlo_status hjlo_step(hjlo_plan *p, const void *u_in, void *u_out, const double *V, int32_t *argmin_out)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u_in || !u_out) return set_error(HJLO_EINVAL, "u_in/u_out is NULL");
    const size_t bytes = (size_t)p->npts * p->esize;
    if (u_in != u_out && ranges_overlap(u_in, u_out, bytes))
        return set_error(HJLO_EINVAL, "u_in and u_out overlap without being equal");
    if ((s = set_device(p)) != HJLO_OK) return s;
    const double *hv = nullptr;
    if (V) {
        if ((s = form_hv(p, V)) != HJLO_OK) return s;
        hv = p->d_hv;
    }
    s = enqueue_step(p, u_in, u_out, hv, 0.0, argmin_out, p->stream);
    if (s == HJLO_OK) p->steps += 1;
    return s;
}

hjlo_status hjlo_run(hjlo_plan *p, void *u, const double *V, int64_t nsteps)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    if ((s = set_device(p)) != HJLO_OK) return s;
    return run_impl(p, u, V, nsteps, false);
}

hjlo_status hjlo_run_tv(hjlo_plan *p, void *u, const double *V, int64_t nsteps)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    if ((s = set_device(p)) != HJLO_OK) return s;
    return run_impl(p, u, V, nsteps, true);
}

hjlo_status hjlo_run_host(hjlo_plan *p, void *u_host, const double *V_host, int64_t nsteps)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u_host) return set_error(HJLO_EINVAL, "u_host is NULL");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    if ((s = set_device(p)) != HJLO_OK) return s;
    const size_t ub = (size_t)p->npts * p->esize, vb = (size_t)p->npts * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (!p->d_u_host_run) e = cudaMalloc(&p->d_u_host_run, ub);
    if (e == cudaSuccess && V_host && !p->d_V_host_run) e = cudaMalloc(&p->d_V_host_run, vb);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(host-run buffers)");
    e = cudaMemcpyAsync(p->d_u_host_run, u_host, ub, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && V_host) e = cudaMemcpyAsync(p->d_V_host_run, V_host, vb, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(H2D)");
    s = run_impl(p, p->d_u_host_run, V_host ? p->d_V_host_run : nullptr, nsteps, false);
    if (s != HJLO_OK) return s;
    e = cudaMemcpyAsync(u_host, p->d_u_host_run, ub, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(D2H)");
    return HJLO_OK;
}

hjlo_status hjlo_hbar(hjlo_plan *p, const void *u0, const void *un, int64_t nsteps, double *out3)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u0 || !un || !out3) return set_error(HJLO_EINVAL, "NULL argument");
    if (nsteps < 1) return set_error(HJLO_EINVAL, "nsteps must be >= 1");
    if ((s = set_device(p)) != HJLO_OK) return s;
    cudaError_t e = cudaSuccess;
    if (!p->d_part) e = cudaMalloc(&p->d_part, sizeof(double) * 3 * (kReduceBlocks + 1));
    if (e != cudaSuccess) { p->d_part = nullptr; return cuda_error(e, "cudaMalloc(readout)"); }
    if (p->dtype == HJLO_F64)
        diff_partials<double><<<kReduceBlocks, kReduceThreads, 0, p->stream>>>(
            (const double *)u0, (const double *)un, p->npts, p->d_part);
    else
        diff_partials<float><<<kReduceBlocks, kReduceThreads, 0, p->stream>>>(
            (const float *)u0, (const float *)un, p->npts, p->d_part);
    fold_partials<<<1, 32, 0, p->stream>>>(p->d_part, kReduceBlocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "readout kernels");
    double r[3];
    e = cudaMemcpyAsync(r, p->d_part + 3 * kReduceBlocks, sizeof(r), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_error(e, "readout copy");
    const double T = (double)nsteps * p->desc.h;
    out3[0] = -(r[0] / (double)p->npts) / T;
    out3[1] = -r[2] / T;
    out3[2] = -r[1] / T;
    return HJLO_OK;
}

hjlo_status hjlo_plan_autotune(hjlo_plan *p, const void *u, const double *V, int64_t nsteps, hjlo_tune_report *report)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 1) return set_error(HJLO_EINVAL, "nsteps must be >= 1");
    if ((s = set_device(p)) != HJLO_OK) return s;
    DeviceFacts df;
    if ((s = device_facts(df)) != HJLO_OK) return s;
    // trial launches do not count: the device counters are put back afterwards
    unsigned long long saved[CNT_N];
    cudaError_t se = cudaStreamSynchronize(p->stream);
    if (se == cudaSuccess) se = cudaMemcpy(saved, p->d_counters, sizeof(saved), cudaMemcpyDeviceToHost);
    if (se != cudaSuccess) return cuda_error(se, "autotune counter save");
    const size_t bytes = (size_t)p->npts * p->esize;
    void *scratch = nullptr;
    if ((s = dmalloc(&scratch, bytes, "cudaMalloc(autotune scratch)")) != HJLO_OK) return s;
    const double *hv = nullptr;
    if (V) {
        if ((s = form_hv(p, V)) != HJLO_OK) { cudaFree(scratch); return s; }
        hv = p->d_hv;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // best of two timed runs of nsteps from a fresh copy of u
    auto trial = [&](float *ms) -> hjlo_status {
        float best = 1e30f;
        for (int r = 0; r < 2; ++r) {
            cudaError_t ce = cudaMemcpyAsync(scratch, u, bytes, cudaMemcpyDeviceToDevice, p->stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, p->stream);
            if (ce != cudaSuccess) return cuda_error(ce, "autotune trial");
            for (long long n = 0; n < nsteps; ++n) {
                hjlo_status ts = enqueue_step(p, scratch, scratch, hv, 0.0, nullptr, p->stream);
                if (ts != HJLO_OK) return ts;
            }
            ce = cudaEventRecord(e1, p->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) return cuda_error(ce, "autotune timing");
            best = std::min(best, t);
        }
        *ms = best;
        return HJLO_OK;
    };
    hjlo_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    float ms0 = 0.0f;
    if (e != cudaSuccess) s = cuda_error(e, "cudaEventCreate");
    if (s == HJLO_OK) s = trial(&ms0);
    float cur = ms0;
    for (int a = 0; a < p->ndim && s == HJLO_OK; ++a) {
        if (p->ax[a].algo != KALGO_MONGE) continue;
        AxisPlan best = p->ax[a];
        for (const ShapeHints &h : tune_candidates(p->ax[a])) {
            AxisPlan t = p->ax[a];
            if (shape_launch(t, p->esize, KALGO_MONGE, df.num_sms, df.smem_optin, 1, &h) != HJLO_OK) continue;
            if (t.lpl == best.lpl && t.C == best.C && t.wide_mul == best.wide_mul && t.wide_add == best.wide_add &&
                t.vR == best.vR)
                continue;
            AxisPlan keep = p->ax[a];
            p->ax[a] = t;
            float ms = 0.0f;
            s = trial(&ms);
            p->ax[a] = keep;
            if (s != HJLO_OK) break;
            ++rep.trials;
            if (ms < 0.98f * cur) {
                cur = ms;
                best = t;
            }
        }
        p->ax[a] = best;
    }
    float ms1 = cur;
    if (s == HJLO_OK) s = trial(&ms1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(scratch);
    destroy_graph(p);
    se = cudaStreamSynchronize(p->stream);
    if (se == cudaSuccess) se = cudaMemcpy(p->d_counters, saved, sizeof(saved), cudaMemcpyHostToDevice);
    if (s == HJLO_OK && se != cudaSuccess) s = cuda_error(se, "autotune counter restore");
    if (s != HJLO_OK) return s;
    for (int a = 0; a < p->ndim; ++a) {
        if (p->ax[a].algo != KALGO_MONGE) continue;
        rep.lanes_per_line[a] = p->ax[a].lpl;
        rep.lines_per_tile[a] = p->ax[a].C;
        rep.offload[a] = (p->ax[a].wide_add < (1 << 20)) ? 1 : 0;
    }
    rep.ms_initial = ms0;
    rep.ms_tuned = ms1;
    if (report) *report = rep;
    return HJLO_OK;
}

hjlo_status hjlo_plan_set_decomp(hjlo_plan *p, double eta, int32_t restart_blocks)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if (p->algo != HJLO_ALGO_DECOMP) return set_error(HJLO_EINVAL, "the tolerance applies to HJLO_ALGO_DECOMP plans");
    if (!(eta >= 0.0) || !std::isfinite(eta)) return set_error(HJLO_EINVAL, "eta must be finite and >= 0");
    if (restart_blocks != 0 && restart_blocks != 1) return set_error(HJLO_EINVAL, "restart_blocks must be 0 or 1");
    if ((s = set_device(p)) != HJLO_OK) return s;
    DeviceFacts df;
    if ((s = device_facts(df)) != HJLO_OK) return s;
    // launch shapes first (nothing changes if one does not fit): at eta = 0
    // the result does not depend on where a line's cut starts, so long or
    // lonely lines keep their row blocks; at eta > 0 a period is decomposed
    // whole unless the caller asked for restarts at each block
    const bool blocks_ok = (eta == 0.0) || restart_blocks;
    AxisPlan shaped[HJLO_MAX_DIM];
    bool need_scratch = false;
    for (int a = 0; a < p->ndim; ++a) {
        shaped[a] = p->ax[a];
        if ((s = shape_decomp(shaped[a], df.smem_optin, df.num_sms, blocks_ok)) != HJLO_OK) return s;
        need_scratch = need_scratch || shaped[a].vblocks > 1 || shaped[a].dsplit;
    }
    // device memory the new shapes need, also before anything changes
    void *fresh[HJLO_MAX_DIM] = {};
    void *fresh_scratch = nullptr;
    for (int a = 0; a < p->ndim && s == HJLO_OK; ++a)
        if (split_scratch_bytes(shaped[a]) > p->ax[a].split_bytes)
            s = dmalloc(&fresh[a], split_scratch_bytes(shaped[a]), "cudaMalloc(decomposition scratch)");
    if (s == HJLO_OK && need_scratch && !p->d_scratch)
        s = dmalloc(&fresh_scratch, (size_t)p->npts * p->esize, "cudaMalloc(row-block scratch)");
    // launches already enqueued keep their own copy of the parameters; the
    // cached graph holds the old value and is rebuilt on next use
    cudaError_t e = (s == HJLO_OK) ? cudaStreamSynchronize(p->stream) : cudaSuccess;
    if (s != HJLO_OK || e != cudaSuccess) {
        for (int a = 0; a < HJLO_MAX_DIM; ++a) cudaFree(fresh[a]);
        cudaFree(fresh_scratch);
        return (s != HJLO_OK) ? s : cuda_error(e, "cudaStreamSynchronize");
    }
    // slopes per unit length (Sec. 4.1): the second differences along axis a
    // are compared with -eta * dx_a
    for (int a = 0; a < p->ndim; ++a) {
        p->ax[a] = shaped[a];             // keeps the axis's scratch pointer
        if (fresh[a]) {
            cudaFree(p->ax[a].d_split);
            p->ax[a].d_split = fresh[a];
            p->ax[a].split_bytes = split_scratch_bytes(shaped[a]);
        }
        p->ax[a].eta = eta * p->desc.dx[a];
    }
    if (fresh_scratch) p->d_scratch = fresh_scratch;
    for (int a = 0; a < p->ndim; ++a)
        if ((s = split_prepare(p->ax[a], p->stream)) != HJLO_OK) return s;
    p->decomp_restart = restart_blocks;
    destroy_graph(p);
    return HJLO_OK;
}

hjlo_status hjlo_plan_set_tolerance(hjlo_plan *p, double eta) { return hjlo_plan_set_decomp(p, eta, 0); }

hjlo_status hjlo_sync(hjlo_plan *p, hjlo_counters *out)
{
    hjlo_status s = check_plan(p);
    if (s != HJLO_OK) return s;
    if ((s = set_device(p)) != HJLO_OK) return s;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    unsigned long long c[CNT_N];
    int flags = 0;
    e = cudaMemcpy(c, p->d_counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&flags, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "counter copy");
    if (out) {
        memset(out, 0, sizeof(*out));
        out->exact_rescans = (int64_t)c[CNT_RESCAN];
        out->brute_fallback_lines = (int64_t)c[CNT_FALLBACK];
        out->components = (int64_t)c[CNT_COMPONENTS];
        out->window_edge_hits = (int64_t)c[CNT_EDGE];
        out->steps = p->steps;
        out->error_flags = flags;
    }
    if (flags) {
        cudaMemset(p->d_flags, 0, sizeof(int));
        if (flags & FLAG_TIMEOUT) return set_error(HJLO_ETIMEOUT, "a bounded device wait gave up");
        return set_error(HJLO_EPRECOND, "a device precondition failed");
    }
    return HJLO_OK;
}

}  // extern "C"
