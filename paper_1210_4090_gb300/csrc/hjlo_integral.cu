// hjlo_integral.cu -- the first discrete semigroup (Sec. 2.2, eq. cost1).
//
// One step: u'(x) = min over the window box of
//     fl(fl(u(y) + K(d)) - fl(h * S(y, d))),   y = x - d (periodic),
// where K(d) = k_0[d_0] + k_1[d_1] + ... is the kinetic action tau K*(v) of
// eq. cost2's tables (left to right) and h * S(y, d) is the exact integral of
// the Fourier-series potential along the straight path from y to x:
//     S = sum_m Re(A_m(y) phi_m(d)) = sum_m (Are_m Pre_m - Aim_m Pim_m)
// with A_m(y) = c_m exp(i alpha_m(y)) and (Pre, Pim) = phi(theta_m(d)),
// phi(theta) = (sin theta / theta, (1 - cos theta) / theta), phi(0) = (1, 0).
// S is accumulated with fused multiply-adds in two chains (even and odd
// modes, added at the end): two binary64 operations per mode instead of
// four, and two independent dependency chains.  The potential term does not
// separate by axis, so the minimum runs over the whole box; there is no
// monotone structure to use and every candidate is evaluated.
//
// Tables are formed once per plan on the host (libm sin / cos): A per point
// and mode (mode-major, so the threads of a warp read consecutive sources),
// K and phi per displacement.  Four threads per output point (consecutive
// lanes) share its displacements and merge their minima by shuffles;
// ping-pong buffers (a step reads its whole source before any output is
// final).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hjlo_internal.h"

using namespace hjlo;

struct hjlo_integral {
    int ndim = 1, device = 0;
    long long shape[HJLO_MAX_DIM] = {1, 1, 1};
    long long npts = 1;
    int nmodes = 0;
    long long ndisp = 1;
    double h = 0.0;
    cudaStream_t stream = nullptr;
    double *d_A = nullptr;        // [2][nmodes][npts]: real parts, then imaginary parts
    double *d_K = nullptr;        // [ndisp]
    double *d_phi = nullptr;      // [ndisp][nmodes][2]
    int *d_disp = nullptr;        // [ndisp][3] displacement per axis, mod N
    double *d_tmp = nullptr;      // ping-pong buffer, npts
    long long steps = 0;
};

namespace {

constexpr int kIntegralSplit = 4;      // threads per output point

__global__ void integral_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                const double *__restrict__ A, const double *__restrict__ K,
                                const double *__restrict__ phi, const int *__restrict__ disp, long long ndisp,
                                int nmodes, long long n0, long long n1, long long n2, long long npts, double h)
{
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long x = gt / kIntegralSplit;
    const int part = (int)(gt % kIntegralSplit);
    const bool live = x < npts;
    double best = INFINITY;
    if (live) {
        const int m0 = (int)n0, m1 = (int)n1, m2 = (int)n2;
        const int i2 = (int)(x % n2);
        const long long r = x / n2;
        const int i1 = (int)(r % n1), i0 = (int)(r / n1);
        for (long long di = part; di < ndisp; di += kIntegralSplit) {
            // periodic source coordinates: displacements are stored mod N, so
            // one conditional add wraps them (32-bit arithmetic)
            int y0 = i0 - disp[3 * di], y1 = i1 - disp[3 * di + 1], y2 = i2 - disp[3 * di + 2];
            y0 += (y0 < 0) ? m0 : 0;
            y1 += (y1 < 0) ? m1 : 0;
            y2 += (y2 < 0) ? m2 : 0;
            const long long y = ((long long)y0 * m1 + y1) * m2 + y2;
            const double *ph = phi + 2 * (long long)nmodes * di;
            double se = 0.0, so = 0.0;
            int m = 0;
            for (; m + 1 < nmodes; m += 2) {
                se = __fma_rn(A[(long long)m * npts + y], ph[2 * m], se);
                se = __fma_rn(-A[((long long)nmodes + m) * npts + y], ph[2 * m + 1], se);
                so = __fma_rn(A[(long long)(m + 1) * npts + y], ph[2 * m + 2], so);
                so = __fma_rn(-A[((long long)nmodes + m + 1) * npts + y], ph[2 * m + 3], so);
            }
            if (m < nmodes) {
                se = __fma_rn(A[(long long)m * npts + y], ph[2 * m], se);
                se = __fma_rn(-A[((long long)nmodes + m) * npts + y], ph[2 * m + 1], se);
            }
            const double S = __dadd_rn(se, so);
            const double c = __dsub_rn(__dadd_rn(src[y], K[di]), __dmul_rn(h, S));
            best = (c < best) ? c : best;
        }
    }
    // the point's minimum over its kIntegralSplit consecutive lanes
    for (int o = 1; o < kIntegralSplit; o <<= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        best = (ob < best) ? ob : best;
    }
    if (live && part == 0) dst[x] = best;
}

void release(hjlo_integral *s)
{
    cudaFree(s->d_A);
    cudaFree(s->d_K);
    cudaFree(s->d_phi);
    cudaFree(s->d_disp);
    cudaFree(s->d_tmp);
}

}  // namespace

extern "C" {

hjlo_status hjlo_integral_create(const hjlo_desc *d, int32_t nmodes, const int32_t *modes, const double *coef,
                                 void *cuda_stream, hjlo_integral **out)
{
    if (!out) return set_error(HJLO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d) return set_error(HJLO_EINVAL, "descriptor is NULL");
    if (d->ndim < 1 || d->ndim > HJLO_MAX_DIM) return set_error(HJLO_EINVAL, "ndim must be 1..3");
    if (d->dtype != HJLO_F64) return set_error(HJLO_EUNSUPPORTED, "the integral semigroup runs in binary64");
    if (d->algo != HJLO_ALGO_AUTO && d->algo != HJLO_ALGO_BRUTE)
        return set_error(HJLO_EUNSUPPORTED, "the integral semigroup evaluates every candidate (brute force)");
    if (d->reserved != 0) return set_error(HJLO_EINVAL, "reserved field must be 0");
    if (!(d->h > 0) || !std::isfinite(d->h)) return set_error(HJLO_EINVAL, "h must be finite and > 0");
    if (nmodes < 0 || (nmodes > 0 && (!modes || !coef))) return set_error(HJLO_EINVAL, "bad Fourier modes");
    hjlo_integral *s = new (std::nothrow) hjlo_integral();
    if (!s) return set_error(HJLO_ENOMEM, "host allocation");
    s->ndim = d->ndim;
    s->h = d->h;
    s->nmodes = nmodes;
    s->stream = (cudaStream_t)cuda_stream;
    std::vector<long long> dlo(3, 0), weff(3, 1);
    std::vector<std::vector<double>> ktab(3, std::vector<double>(1, 0.0));
    hjlo_status st = HJLO_OK;
    for (int a = 0; a < d->ndim && st == HJLO_OK; ++a) {
        if (d->shape[a] < 1 || !(d->dx[a] > 0) || !std::isfinite(d->P[a])) {
            st = set_error(HJLO_EINVAL, "bad shape, dx or P on axis %d", a);
            break;
        }
        s->shape[a] = d->shape[a];
        AxisPlan ax;
        double *kr = nullptr;
        st = resolve_axis(d->shape[a], d->dx[a], d->h, d->P[a], d->window[a], ax, &kr);
        if (st != HJLO_OK) break;
        dlo[a] = ax.dlo;
        weff[a] = ax.weff;
        ktab[a].assign(ax.weff, 0.0);
        for (long long t = 0; t < ax.weff; ++t) ktab[a][t] = kr[ax.weff - 1 - t];     // k[dlo + t]
        free(kr);
    }
    // the trailing axes of a 1D/2D grid are length-1 axes with the zero displacement
    for (int a = d->ndim; a < 3; ++a) s->shape[a] = 1;
    s->npts = s->shape[0] * s->shape[1] * s->shape[2];
    s->ndisp = weff[0] * weff[1] * weff[2];
    if (st == HJLO_OK && (s->npts > (1LL << 31) || s->ndisp > (1LL << 24) ||
                          (double)s->npts * (double)s->ndisp * (nmodes + 1) > 1e15))
        st = set_error(HJLO_EUNSUPPORTED, "grid or window box too large for the integral semigroup");
    std::vector<double> K, phi, A;
    std::vector<int> disp;
    if (st == HJLO_OK) {
        const double twopi = 2.0 * M_PI;
        K.resize(s->ndisp);
        phi.resize(2 * (size_t)s->ndisp * nmodes);
        disp.resize(3 * (size_t)s->ndisp);
        long long di = 0;
        for (long long t0 = 0; t0 < weff[0]; ++t0)
            for (long long t1 = 0; t1 < weff[1]; ++t1)
                for (long long t2 = 0; t2 < weff[2]; ++t2, ++di) {
                    const long long dd[3] = {dlo[0] + t0, dlo[1] + t1, dlo[2] + t2};
                    const long long tt[3] = {t0, t1, t2};
                    double k = 0.0;
                    for (int a = 0; a < d->ndim; ++a) k = k + ktab[a][tt[a]];
                    K[di] = k;
                    // the source only depends on d mod N (K and phi keep the lift)
                    for (int a = 0; a < 3; ++a) {
                        long long dm = dd[a] % s->shape[a];
                        disp[3 * di + a] = (int)(dm < 0 ? dm + s->shape[a] : dm);
                    }
                    for (int m = 0; m < nmodes; ++m) {
                        double sarg = 0.0;
                        for (int a = 0; a < d->ndim; ++a)
                            sarg = sarg + ((double)modes[m * d->ndim + a] * (double)dd[a]) / (double)s->shape[a];
                        const double th = twopi * sarg;
                        double pre = 1.0, pim = 0.0;
                        if (th != 0.0) {
                            pre = std::sin(th) / th;
                            pim = (1.0 - std::cos(th)) / th;
                        }
                        phi[2 * ((size_t)di * nmodes + m)] = pre;
                        phi[2 * ((size_t)di * nmodes + m) + 1] = pim;
                    }
                }
        A.resize(2 * (size_t)nmodes * s->npts);
        for (int m = 0; m < nmodes; ++m) {
            const double cre = coef[2 * m], cim = coef[2 * m + 1];
            for (long long x = 0; x < s->npts; ++x) {
                const long long ii[3] = {x / (s->shape[1] * s->shape[2]), (x / s->shape[2]) % s->shape[1],
                                         x % s->shape[2]};
                double sarg = 0.0;
                for (int a = 0; a < d->ndim; ++a)
                    sarg = sarg + (double)modes[m * d->ndim + a] * ((double)ii[a] / (double)s->shape[a]);
                const double al = twopi * sarg;
                const double ca = std::cos(al), sa = std::sin(al);
                A[(size_t)m * s->npts + x] = cre * ca - cim * sa;
                A[((size_t)nmodes + m) * s->npts + x] = cre * sa + cim * ca;
            }
        }
    }
    if (st == HJLO_OK) {
        cudaError_t e = cudaGetDevice(&s->device);
        if (e == cudaSuccess && !A.empty()) e = cudaMalloc(&s->d_A, sizeof(double) * A.size());
        if (e == cudaSuccess) e = cudaMalloc(&s->d_K, sizeof(double) * K.size());
        if (e == cudaSuccess && !phi.empty()) e = cudaMalloc(&s->d_phi, sizeof(double) * phi.size());
        if (e == cudaSuccess) e = cudaMalloc(&s->d_disp, sizeof(int) * disp.size());
        if (e == cudaSuccess) e = cudaMalloc(&s->d_tmp, sizeof(double) * s->npts);
        if (e == cudaSuccess && !A.empty())
            e = cudaMemcpy(s->d_A, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->d_K, K.data(), sizeof(double) * K.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !phi.empty())
            e = cudaMemcpy(s->d_phi, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(s->d_disp, disp.data(), sizeof(int) * disp.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_error(e, "integral semigroup tables");
    }
    if (st != HJLO_OK) {
        release(s);
        delete s;
        return st;
    }
    *out = s;
    return HJLO_OK;
}

hjlo_status hjlo_integral_run(hjlo_integral *s, double *u, int64_t nsteps)
{
    if (!s) return set_error(HJLO_EINVAL, "plan is NULL");
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    double *a = u, *b = s->d_tmp;
    const unsigned blocks = (unsigned)((s->npts * kIntegralSplit + 255) / 256);
    for (long long n = 0; n < nsteps; ++n) {
        integral_kernel<<<blocks, 256, 0, s->stream>>>(a, b, s->d_A, s->d_K, s->d_phi, s->d_disp, s->ndisp, s->nmodes,
                                                       s->shape[0], s->shape[1], s->shape[2], s->npts, s->h);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "integral kernel launch");
        std::swap(a, b);
    }
    if (a != u) {
        e = cudaMemcpyAsync(u, a, sizeof(double) * s->npts, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync");
    }
    s->steps += nsteps;
    return HJLO_OK;
}

hjlo_status hjlo_integral_sync(hjlo_integral *s)
{
    if (!s) return set_error(HJLO_EINVAL, "plan is NULL");
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? HJLO_OK : cuda_error(e, "cudaStreamSynchronize");
}

hjlo_status hjlo_integral_destroy(hjlo_integral *s)
{
    if (!s) return HJLO_OK;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    release(s);
    delete s;
    return HJLO_OK;
}

}  // extern "C"
