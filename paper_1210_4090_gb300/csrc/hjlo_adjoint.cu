// hjlo_adjoint.cu -- reverse mode of the scheme (hjlo_adjoint, hjlo_project).
//
// The value of every pass output comes from exactly one source (the
// discrete optimal path of eq. raslebol, Appendix B): m_i = u[src(i)] + k[d_i]
// with src(i) = (i - d_i) mod N.  So, for J = <ubar_n, u^n>:
//   ubar_src += ubar_i        (the pass's transpose, per line)
//   Pbar_a   += ubar_i * (-d_i * dx_a)    (dk/dP = -d*dx for k = h(v^2/2 - P v))
//   Vbar     += -h * ubar^{n+1}          (the potential term of eq. eqconvol)
// taken in reverse over steps and, within a step, over passes.
//
// The transpose is a gather, not a scatter: the recorded argmins of a line
// are non-decreasing (Monge, hypothesis (i)), so the targets of each source
// form one contiguous range of i (two at the periodic seam).  A CTA inverts
// the argmin sequence in shared memory (first target of every lifted source)
// and each thread sums its source's targets in ascending i -- the same order
// as the definition's sequential scatter, so ubar_0 and Vbar are reproduced
// bit for bit and no atomics are needed.  A line whose argmins are not
// monotone (possible only where the Monge rounding margin failed) is done by
// one thread scattering sequentially.  Pbar is summed per line by a warp
// (strided partial sums, then a fixed butterfly), accumulated per line over
// the steps, and the lines are folded once in a fixed order (deterministic;
// its rounding order differs from a single running sum).  The potential
// term's derivative Vbar -= h * ubar^{n+1} is taken by the step's first
// reverse pass as it loads ubar.
//
// Memory: forward states are checkpointed every S steps; each segment is
// recomputed once with argmin recording (S x ndim x npts int32) and then
// reversed.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hjlo_internal.h"

using namespace hjlo;

namespace {

struct AdjParams {
    double *ub;               // cotangent, updated in place
    const int32_t *amin;      // argmin displacement per point of this pass
    double *pline;            // per-line P partials of this axis, accumulated over steps
    double *vbar;             // Vbar -= h * ub at load (the step's first reverse pass), or null
    double h;
    long long N, inner, outer, ntiles, tiles_per_outer;
    int C, log2C;
    double dx;
};

template <int LAYOUT>
__device__ __forceinline__ void adj_tile(const AdjParams &p, long long tile, long long &base, long long &lstride,
                                         long long &pstride, int &valid, long long &line0, long long &linestep)
{
    if (LAYOUT == LAYOUT_CONTIG) {
        long long l0 = tile << p.log2C;
        base = l0 * p.N;
        lstride = p.N;
        pstride = 1;
        long long rem = p.outer - l0;
        valid = (int)(rem < p.C ? rem : p.C);
        line0 = l0;
        linestep = 1;
    } else {
        long long o = tile / p.tiles_per_outer;
        long long in0 = (tile - o * p.tiles_per_outer) << p.log2C;
        base = o * p.N * p.inner + in0;
        lstride = 1;
        pstride = p.inner;
        long long rem = p.inner - in0;
        valid = (int)(rem < p.C ? rem : p.C);
        line0 = o * p.inner + in0;
        linestep = 1;
    }
}

// Transpose of one axis pass over a tile of C lines.
template <int LAYOUT>
__global__ void __launch_bounds__(256) adjoint_pass_kernel(AdjParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = (int)p.N, C = p.C;
    double *mb = reinterpret_cast<double *>(smem);               // [C][N]
    int *a = reinterpret_cast<int *>(mb + (size_t)C * N);          // [C][N] lifted sources i - d
    int *first = a + (size_t)C * N;                                // [C][N+2]
    int *mono = first + (size_t)C * (N + 2);                       // [C]
    const int tid = threadIdx.x, nthr = blockDim.x;
    long long base, lstride, pstride, line0, linestep;
    int valid;
    adj_tile<LAYOUT>(p, blockIdx.x, base, lstride, pstride, valid, line0, linestep);

    if (tid < C) mono[tid] = 1;
    for (int idx = tid; idx < C * N; idx += nthr) {
        int l, i;
        if (LAYOUT == LAYOUT_CONTIG) { l = idx / N; i = idx - l * N; }
        else { i = idx >> p.log2C; l = idx & (C - 1); }
        if (l >= valid) continue;
        long long x = base + l * lstride + (long long)i * pstride;
        const double u = p.ub[x];
        mb[l * N + i] = u;
        a[l * N + i] = i - p.amin[x];
        if (p.vbar) p.vbar[x] = __dsub_rn(p.vbar[x], __dmul_rn(p.h, u));
    }
    __syncthreads();
    // monotone argmins (lifted), and within one period of the first
    for (int idx = tid; idx < C * N; idx += nthr) {
        int l = idx / N, i = idx - l * N;
        if (l >= valid) continue;
        const int *la = a + l * N;
        bool bad = (i + 1 < N) ? (la[i] > la[i + 1]) : (la[N - 1] > la[0] + N);
        if (bad) mono[l] = 0;
    }
    __syncthreads();
    // first target of every lifted source a0 + k, k in [0, N+1]
    for (int idx = tid; idx < C * N; idx += nthr) {
        int l = idx / N, i = idx - l * N;
        if (l >= valid || !mono[l]) continue;
        const int *la = a + l * N;
        int *lf = first + l * (N + 2);
        const int a0 = la[0];
        const int prev = (i == 0) ? a0 - 1 : la[i - 1];
        for (int L = prev + 1; L <= la[i]; ++L) lf[L - a0] = i;
        if (i == N - 1)
            for (int L = la[N - 1] + 1; L <= a0 + N + 1; ++L) lf[L - a0] = N;
    }
    __syncthreads();
    // gather, ascending target order
    for (int idx = tid; idx < C * N; idx += nthr) {
        int l, r;
        if (LAYOUT == LAYOUT_CONTIG) { l = idx / N; r = idx - l * N; }
        else { r = idx >> p.log2C; l = idx & (C - 1); }
        if (l >= valid || !mono[l]) continue;
        const int *lf = first + l * (N + 2);
        const double *lm = mb + l * N;
        const int a0 = a[l * N];
        int k1 = (r - a0) % N;
        if (k1 < 0) k1 += N;
        double s = 0.0;
        for (int i = lf[k1]; i < lf[k1 + 1]; ++i) s = __dadd_rn(s, lm[i]);
        if (k1 == 0)
            for (int i = lf[N]; i < lf[N + 1]; ++i) s = __dadd_rn(s, lm[i]);
        p.ub[base + l * lstride + (long long)r * pstride] = s;
    }
    // lines with non-monotone argmins: one thread scatters in ascending i
    if (tid < valid && !mono[tid]) {
        const int l = tid;
        const double *lm = mb + l * N;
        const int *la = a + l * N;
        for (int r = 0; r < N; ++r) p.ub[base + l * lstride + (long long)r * pstride] = 0.0;
        for (int i = 0; i < N; ++i) {
            int r = la[i] % N;
            if (r < 0) r += N;
            double *dst = p.ub + base + l * lstride + (long long)r * pstride;
            *dst = __dadd_rn(*dst, lm[i]);
        }
    }
    // P partial of every line: a warp per line, each lane sums its terms in
    // ascending i, then a fixed butterfly (the same order on every run; every
    // lane ends with the same sum since a + b == b + a)
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    for (int l = warp; l < valid; l += nwarps) {
        const double *lm = mb + l * N;
        const int *la = a + l * N;
        double s = 0.0;
        for (int i = lane; i < N; i += 32) {
            const double g = __dmul_rn(-(double)(i - la[i]), p.dx);
            s = __dadd_rn(s, __dmul_rn(lm[i], g));
        }
        for (int o = 16; o; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) {
            double *acc = p.pline + line0 + l * linestep;
            *acc = __dadd_rn(*acc, s);
        }
    }
}

// Pbar[axis] += sum of the per-line partials (each accumulated over all steps
// by the adjoint passes), in a fixed order: 256 threads sum contiguous
// chunks, then a fixed pairwise tree.
__global__ void pbar_fold_kernel(const double *__restrict__ pline, long long nlines, double *__restrict__ pbar)
{
    __shared__ double sh[256];
    const int t = threadIdx.x;
    long long chunk = (nlines + 255) / 256;
    long long lo = t * chunk, hi = lo + chunk < nlines ? lo + chunk : nlines;
    double s = 0.0;
    for (long long i = lo; i < hi; ++i) s = __dadd_rn(s, pline[i]);
    sh[t] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o) sh[t] = __dadd_rn(sh[t], sh[t + o]);
        __syncthreads();
    }
    if (t == 0) *pbar = __dadd_rn(*pbar, sh[0]);
}

// out[k] = sum_x f(x) B_k(x): per-block partials (fixed order), then a fold.
__global__ void project_partials(const double *__restrict__ f, const double *__restrict__ B, long long n,
                                 double *__restrict__ part)
{
    __shared__ double sh[256];
    const double *Bk = B + (long long)blockIdx.y * n;
    double s = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        s = __dadd_rn(s, __dmul_rn(f[i], Bk[i]));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void project_fold(const double *__restrict__ part, int nblocks, int nbasis, double *__restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbasis) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s = __dadd_rn(s, part[(long long)k * nblocks + b]);
    out[k] = s;
}

struct AdjShape {
    int layout, C, log2C, threads;
    long long ntiles, tiles_per_outer, nlines;
    size_t smem;
};

AdjShape adj_shape(const AxisPlan &ax, int num_sms)
{
    AdjShape s;
    s.layout = (ax.inner == 1) ? LAYOUT_CONTIG : LAYOUT_STRIDED;
    const long long N = ax.N;
    auto smem_for = [&](int C) { return (size_t)C * (N * 12 + (N + 2) * 4 + 4) + 16; };
    int C = 1;
    const int cmax = (s.layout == LAYOUT_STRIDED) ? (int)std::min<long long>(32, ax.inner) : 32;
    while (2 * C <= cmax && smem_for(2 * C) <= 96 * 1024) {
        long long tiles = (s.layout == LAYOUT_CONTIG) ? (ax.outer + 2 * C - 1) / (2 * C)
                                                      : ax.outer * ((ax.inner + 2 * C - 1) / (2 * C));
        if (tiles < 2LL * num_sms) break;
        C *= 2;
    }
    s.C = C;
    s.log2C = 0;
    while ((1 << s.log2C) < C) ++s.log2C;
    s.threads = 256;
    s.tiles_per_outer = (s.layout == LAYOUT_STRIDED) ? (ax.inner + C - 1) / C : 1;
    s.ntiles = (s.layout == LAYOUT_CONTIG) ? (ax.outer + C - 1) / C : ax.outer * s.tiles_per_outer;
    s.nlines = ax.inner * ax.outer;
    s.smem = smem_for(C);
    return s;
}

hjlo_status adjoint_prepare(const hjlo_plan *p, const DeviceFacts &df)
{
    static bool done[64] = {false};
    for (int a = 0; a < p->ndim; ++a)
        if (adj_shape(p->ax[a], df.num_sms).smem > df.smem_optin)
            return set_error(HJLO_EUNSUPPORTED, "a line of %lld points is too long for the adjoint", p->ax[a].N);
    if (df.device < 64 && done[df.device]) return HJLO_OK;
    cudaError_t e = cudaFuncSetAttribute(adjoint_pass_kernel<LAYOUT_CONTIG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df.smem_optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(adjoint_pass_kernel<LAYOUT_STRIDED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)df.smem_optin);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(adjoint)");
    if (df.device < 64) done[df.device] = true;
    return HJLO_OK;
}

hjlo_status launch_adjoint_pass(const AxisPlan &ax, double dx, double *ub, const int32_t *amin, double *pline,
                                double *vbar, double h, int num_sms, cudaStream_t st)
{
    AdjShape sh = adj_shape(ax, num_sms);
    AdjParams p;
    p.ub = ub;
    p.amin = amin;
    p.pline = pline;
    p.vbar = vbar;
    p.h = h;
    p.N = ax.N;
    p.inner = ax.inner;
    p.outer = ax.outer;
    p.ntiles = sh.ntiles;
    p.tiles_per_outer = sh.tiles_per_outer;
    p.C = sh.C;
    p.log2C = sh.log2C;
    p.dx = dx;
    if (sh.layout == LAYOUT_CONTIG)
        adjoint_pass_kernel<LAYOUT_CONTIG><<<(unsigned)sh.ntiles, sh.threads, sh.smem, st>>>(p);
    else
        adjoint_pass_kernel<LAYOUT_STRIDED><<<(unsigned)sh.ntiles, sh.threads, sh.smem, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "adjoint pass launch");
    return HJLO_OK;
}

hjlo_status ensure(void **ptr, long long *cap, long long want, size_t elem, const char *what)
{
    if (*ptr && *cap >= want) return HJLO_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(ptr, (size_t)want * elem);
    if (e != cudaSuccess) { *ptr = nullptr; return cuda_error(e, what); }
    *cap = want;
    return HJLO_OK;
}

}  // namespace

extern "C" {

hjlo_status hjlo_adjoint(hjlo_plan *p, const double *u0, const double *V, int64_t nsteps, const double *ubar_n,
                         double *ubar_0, double *Pbar, double *Vbar, int64_t checkpoint_every, double *u_n)
{
    if (!p) return set_error(HJLO_EINVAL, "plan is NULL");
    if (p->dtype != HJLO_F64) return set_error(HJLO_EUNSUPPORTED, "the adjoint needs a binary64 plan");
    if (p->algo == HJLO_ALGO_DECOMP)
        return set_error(HJLO_EUNSUPPORTED, "the adjoint follows argmins, which the decomposition method does not record");
    if (!u0 || !ubar_n || !ubar_0) return set_error(HJLO_EINVAL, "u0, ubar_n and ubar_0 are required");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    hjlo_status s = plan_set_device(p);
    if (s != HJLO_OK) return s;
    DeviceFacts df;
    if ((s = device_facts(df)) != HJLO_OK) return s;
    if ((s = adjoint_prepare(p, df)) != HJLO_OK) return s;
    const long long npts = p->npts, nd = p->ndim;
    const long long S = (checkpoint_every <= 0 || checkpoint_every > nsteps) ? std::max<long long>(nsteps, 1)
                                                                            : checkpoint_every;
    const long long nseg = (nsteps + S - 1) / S;
    long long maxlines = 1;
    for (int a = 0; a < nd; ++a) maxlines = std::max(maxlines, p->ax[a].inner * p->ax[a].outer);
    if ((s = ensure((void **)&p->d_ckpt, &p->ckpt_cap, std::max<long long>(nseg, 1) * npts, sizeof(double),
                    "cudaMalloc(checkpoints)")) != HJLO_OK)
        return s;
    if ((s = ensure((void **)&p->d_amin, &p->amin_cap, S * nd * npts, sizeof(int32_t), "cudaMalloc(argmins)")) !=
        HJLO_OK)
        return s;
    if ((s = ensure((void **)&p->d_work, &p->work_cap, npts, sizeof(double), "cudaMalloc(work)")) != HJLO_OK)
        return s;
    if ((s = ensure((void **)&p->d_pbar_part, &p->pbar_cap, nd * maxlines + 1, sizeof(double),
                    "cudaMalloc(P partials)")) != HJLO_OK)
        return s;
    cudaStream_t st = p->stream;
    const size_t ub = sizeof(double) * npts;

    // forward with checkpoints
    cudaError_t e = cudaMemcpyAsync(p->d_work, u0, ub, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "copy u0");
    for (long long k = 0; k < nseg; ++k) {
        const long long steps = std::min(S, nsteps - k * S);
        e = cudaMemcpyAsync(p->d_ckpt + k * npts, p->d_work, ub, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "checkpoint");
        if ((s = plan_run(p, p->d_work, V, steps)) != HJLO_OK) return s;
    }
    if (u_n) {
        e = cudaMemcpyAsync(u_n, p->d_work, ub, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "copy u_n");
    }
    // reverse
    const double *hv = nullptr;
    if (V) {
        if ((s = plan_form_hv(p, V)) != HJLO_OK) return s;
        hv = p->d_hv;
    }
    e = cudaMemcpyAsync(ubar_0, ubar_n, ub, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && Vbar) e = cudaMemsetAsync(Vbar, 0, ub, st);
    if (e != cudaSuccess) return cuda_error(e, "adjoint init");
    // per-line P partials of every axis, accumulated over all steps (each
    // line by one warp per launch, launches in order), folded once at the end
    e = cudaMemsetAsync(p->d_pbar_part, 0, sizeof(double) * (nd * maxlines + 1), st);
    if (e != cudaSuccess) return cuda_error(e, "P partials init");
    if (Pbar) {
        e = cudaMemsetAsync(Pbar, 0, sizeof(double) * nd, st);
        if (e != cudaSuccess) return cuda_error(e, "Pbar init");
    }
    for (long long k = nseg - 1; k >= 0; --k) {
        const long long steps = std::min(S, nsteps - k * S);
        e = cudaMemcpyAsync(p->d_work, p->d_ckpt + k * npts, ub, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "restore checkpoint");
        for (long long n = 0; n < steps; ++n)
            if ((s = plan_enqueue_step(p, p->d_work, p->d_work, hv, 0.0, p->d_amin + n * nd * npts, st)) != HJLO_OK)
                return s;
        for (long long n = steps - 1; n >= 0; --n) {
            // the step's first reverse pass (last axis) also takes the
            // potential term's derivative, Vbar -= h * ubar^{n+1}, at load
            for (int a = (int)nd - 1; a >= 0; --a) {
                s = launch_adjoint_pass(p->ax[a], p->desc.dx[a], ubar_0, p->d_amin + (n * nd + a) * npts,
                                        p->d_pbar_part + a * maxlines, (a == nd - 1) ? Vbar : nullptr,
                                        p->desc.h, df.num_sms, st);
                if (s != HJLO_OK) return s;
            }
        }
    }
    if (Pbar)
        for (int a = 0; a < (int)nd; ++a)
            pbar_fold_kernel<<<1, 256, 0, st>>>(p->d_pbar_part + a * maxlines, p->ax[a].inner * p->ax[a].outer,
                                                Pbar + a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "adjoint");
    return HJLO_OK;
}

hjlo_status hjlo_project(hjlo_plan *p, const double *field, const double *basis, int32_t nbasis, double *out)
{
    if (!p) return set_error(HJLO_EINVAL, "plan is NULL");
    if (!field || !basis || !out || nbasis < 1) return set_error(HJLO_EINVAL, "bad arguments");
    hjlo_status s = plan_set_device(p);
    if (s != HJLO_OK) return s;
    const int nblk = 64;
    if ((s = ensure((void **)&p->d_proj, &p->proj_cap, (long long)nbasis * nblk, sizeof(double),
                    "cudaMalloc(projection partials)")) != HJLO_OK)
        return s;
    double *part = p->d_proj;
    dim3 grid(nblk, (unsigned)nbasis);
    project_partials<<<grid, 256, 0, p->stream>>>(field, basis, p->npts, part);
    project_fold<<<(nbasis + 127) / 128, 128, 0, p->stream>>>(part, nblk, nbasis, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "projection kernels");
    return HJLO_OK;
}

}  // extern "C"
