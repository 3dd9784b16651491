/*
 * hjlo_oracle.c -- plain, slow, obviously-correct CPU oracle for the fully
 * discrete Lax--Oleinik scheme of Bouillard, Faou & Zavidovique,
 * "Fast weak-KAM integrators for separable Hamiltonian systems".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library; it is written from the paper alone.
 *
 * What it computes (notation: dx = space step, h = time step, the paper's tau):
 *
 *   Kernel table, per axis a (eq. cost2 with the mechanical Lagrangian of
 *   Sec. 2.1, L(v) = 1/2 v^2 - P_a v, restricted to one axis by Remark rk28):
 *       k_a[d] = h * L(d*dx_a/h),  evaluated in the fixed order
 *       v = (d*dx)/h;  t1 = 0.5*v;  t1 = t1*v;  t2 = P*v;  L = t1 - t2;  k = h*L
 *   (all IEEE binary64 round-to-nearest, no fused multiply-add).
 *
 *   Window of displacements d (torus grid, Sec. 3.3 eq. los, and Sec. 4.2,
 *   where the kernel is restricted to a support centred on its minimum):
 *     c = the largest d attaining min_d k[d];
 *     windowed (W > 0 and 2W+1 < N):   d in [c-W, c+W];
 *     full     (otherwise):            the N consecutive displacements that
 *       realise the lift-minimised cost kappa~ (one lift per residue mod N,
 *       the cheaper one; equal costs keep the larger d).
 *
 *   One axis pass (Remark rk28), for every line along axis a and every i:
 *       m_i = min over d in the window of  fl(u[(i-d) mod N] + k_a[d]),
 *   scanning the source j = i-d in ascending lifted order (descending d) and
 *   keeping a candidate only if it is strictly smaller, so equal values keep
 *   the smallest lifted source j (the largest d).  The recorded argmin is d.
 *
 *   One time step (eq. eqconvol and eq. uN): passes along axis 0 (slowest
 *   varying) first, ..., axis ndim-1 (contiguous) last, then the potential
 *   term of eq. eqconvol:  u^{n+1}_x = fl(m_x - hV_x),  hV_x = fl(h*V(t_n,x)).
 *
 *   FP32 storage: u is held in binary32; each pass loads exactly to binary64,
 *   computes as above and rounds (to nearest) to binary32 at its store; the
 *   last pass rounds fl(m - hV) to binary32.
 *
 *   Adjoint (the discrete optimal path of eq. raslebol routes every value to
 *   exactly one source): reverse steps, and within a step reverse passes;
 *       Vbar_x  <- fl(Vbar_x - fl(h*ubar_x))          (per step, before passes)
 *       ubar'_src(i) += ubar_i  for i ascending        (per line)
 *       Pbar_a  += ubar_i * (-d_i*dx_a)                 (d k/d P = -d*dx)
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared hjlo_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HJO_MAXDIM 3

/* ---------------------------------------------------------------- tables */

/* One kernel entry: eq. cost2 with L(v) = v^2/2 - P v, v = d*dx/h. */
double hjo_kernel(int64_t d, double dx, double h, double P)
{
    double v = ((double)d * dx) / h;
    double t1 = 0.5 * v;
    t1 = t1 * v;
    double t2 = P * v;
    double L = t1 - t2;
    return h * L;
}

/* Largest d attaining the minimum of the kernel.  The continuous minimiser
 * of h*L(d*dx/h) is d = P*h/dx; the discrete minimiser is within one cell of
 * it, so a scan of a few integers on each side finds it.  Returns 0 on
 * success, -1 if the minimiser is not representable. */
static int hjo_centre(double dx, double h, double P, int64_t *c_out)
{
    double ds = P * h / dx;
    if (!(fabs(ds) < 4.0e18)) return -1;
    int64_t base = (int64_t)floor(ds);
    int64_t best = base - 4;
    double kb = hjo_kernel(best, dx, h, P);
    for (int64_t d = base - 3; d <= base + 5; ++d) {
        double kd = hjo_kernel(d, dx, h, P);
        if (kd <= kb) { kb = kd; best = d; }   /* '<=' keeps the largest d */
    }
    *c_out = best;
    return 0;
}

/* Window [dlo, dhi] of displacements (see header).  Returns 0 or -1. */
int hjo_window(int64_t N, double dx, double h, double P, int64_t W,
               int64_t *dlo, int64_t *dhi)
{
    int64_t c;
    if (N < 1 || !(dx > 0) || !(h > 0)) return -1;
    if (hjo_centre(dx, h, P, &c)) return -1;
    if (W > 0 && 2 * W + 1 < N) {
        *dlo = c - W;
        *dhi = c + W;
        return 0;
    }
    /* Full periodic window: for each residue keep the cheaper lift.  Growing
     * the block one displacement at a time towards the cheaper neighbour
     * gives the N cheapest consecutive displacements of the convex kernel. */
    int64_t lo = c, hi = c;
    while (hi - lo + 1 < N) {
        double kl = hjo_kernel(lo - 1, dx, h, P);
        double kh = hjo_kernel(hi + 1, dx, h, P);
        if (kl < kh) --lo; else ++hi;
    }
    *dlo = lo;
    *dhi = hi;
    return 0;
}

/* Fill k[0 .. dhi-dlo] with k[d] for d = dlo .. dhi. */
void hjo_table(int64_t dlo, int64_t dhi, double dx, double h, double P, double *k)
{
    for (int64_t d = dlo; d <= dhi; ++d) k[d - dlo] = hjo_kernel(d, dx, h, P);
}

/* ---------------------------------------------------------------- passes */

typedef struct {
    int ndim;
    int64_t shape[HJO_MAXDIM];
    int64_t npts;
    int64_t dlo[HJO_MAXDIM], dhi[HJO_MAXDIM];
    double *k[HJO_MAXDIM];
} hjo_geom;

static int hjo_geom_init(hjo_geom *g, int ndim, const int64_t *shape, const double *dx,
                         double h, const double *P, const int64_t *W)
{
    memset(g, 0, sizeof(*g));
    if (ndim < 1 || ndim > HJO_MAXDIM) return -1;
    g->ndim = ndim;
    g->npts = 1;
    for (int a = 0; a < ndim; ++a) {
        if (shape[a] < 1) return -1;
        g->shape[a] = shape[a];
        g->npts *= shape[a];
        if (hjo_window(shape[a], dx[a], h, P[a], W[a], &g->dlo[a], &g->dhi[a])) return -1;
        g->k[a] = (double *)malloc(sizeof(double) * (size_t)(g->dhi[a] - g->dlo[a] + 1));
        if (!g->k[a]) return -1;
        hjo_table(g->dlo[a], g->dhi[a], dx[a], h, P[a], g->k[a]);
    }
    return 0;
}

static void hjo_geom_free(hjo_geom *g)
{
    for (int a = 0; a < HJO_MAXDIM; ++a) free(g->k[a]);
}

static void hjo_axis_split(const hjo_geom *g, int a, int64_t *outer, int64_t *inner)
{
    int64_t o = 1, in = 1;
    for (int b = 0; b < a; ++b) o *= g->shape[b];
    for (int b = a + 1; b < g->ndim; ++b) in *= g->shape[b];
    *outer = o;
    *inner = in;
}

/* Minimum over the window for one output point; scans ascending lifted
 * source (descending d) with a strict comparison. */
static inline double hjo_min_f64(const double *s, int64_t inner, int64_t N, int64_t i,
                                 const double *k, int64_t dlo, int64_t dhi, int64_t *dbest)
{
    double best = 0.0;
    int64_t bd = dhi;
    int first = 1;
    for (int64_t d = dhi; d >= dlo; --d) {
        int64_t r = (i - d) % N;
        if (r < 0) r += N;
        double cand = s[r * inner] + k[d - dlo];
        if (first || cand < best) { best = cand; bd = d; first = 0; }
    }
    *dbest = bd;
    return best;
}

static inline double hjo_min_f32src(const float *s, int64_t inner, int64_t N, int64_t i,
                                    const double *k, int64_t dlo, int64_t dhi, int64_t *dbest)
{
    double best = 0.0;
    int64_t bd = dhi;
    int first = 1;
    for (int64_t d = dhi; d >= dlo; --d) {
        int64_t r = (i - d) % N;
        if (r < 0) r += N;
        double cand = (double)s[r * inner] + k[d - dlo];
        if (first || cand < best) { best = cand; bd = d; first = 0; }
    }
    *dbest = bd;
    return best;
}

/* One pass of axis a: dst = min-plus(src, k_a).  If hv != NULL the potential
 * term is applied (dst = m - hv).  amin (NULL allowed) receives d per point. */
static void hjo_pass_f64(const hjo_geom *g, int a, const double *src, double *dst,
                         const double *hv, int32_t *amin)
{
    int64_t outer, inner, N = g->shape[a];
    hjo_axis_split(g, a, &outer, &inner);
    const double *k = g->k[a];
    int64_t dlo = g->dlo[a], dhi = g->dhi[a];
    int64_t nlines = outer * inner;
#pragma omp parallel for schedule(static)
    for (int64_t line = 0; line < nlines; ++line) {
        int64_t o = line / inner, in = line % inner;
        int64_t base = o * N * inner + in;
        for (int64_t i = 0; i < N; ++i) {
            int64_t d;
            double m = hjo_min_f64(src + base, inner, N, i, k, dlo, dhi, &d);
            int64_t x = base + i * inner;
            if (hv) m = m - hv[x];
            dst[x] = m;
            if (amin) amin[x] = (int32_t)d;
        }
    }
}

static void hjo_pass_f32(const hjo_geom *g, int a, const float *src, float *dst,
                         const double *hv, int32_t *amin)
{
    int64_t outer, inner, N = g->shape[a];
    hjo_axis_split(g, a, &outer, &inner);
    const double *k = g->k[a];
    int64_t dlo = g->dlo[a], dhi = g->dhi[a];
    int64_t nlines = outer * inner;
#pragma omp parallel for schedule(static)
    for (int64_t line = 0; line < nlines; ++line) {
        int64_t o = line / inner, in = line % inner;
        int64_t base = o * N * inner + in;
        for (int64_t i = 0; i < N; ++i) {
            int64_t d;
            double m = hjo_min_f32src(src + base, inner, N, i, k, dlo, dhi, &d);
            int64_t x = base + i * inner;
            if (hv) m = m - hv[x];
            dst[x] = (float)m;
            if (amin) amin[x] = (int32_t)d;
        }
    }
}

static void hjo_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int hjo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* hV = fl(h*V) for the V of one step (V == NULL means V = 0). */
static void hjo_hv(int64_t npts, double h, const double *V, double *hv)
{
    for (int64_t x = 0; x < npts; ++x) hv[x] = h * V[x];
}

/*
 * Run nsteps of the scheme in place on u (binary64).
 *   V: NULL (V = 0) or the potential; step n uses V + n*V_step_stride
 *      (V_step_stride = 0: time-independent V).
 *   amin: NULL, or nsteps*ndim*npts int32 receiving the argmin d of every
 *      pass, laid out [step][axis][point].
 * Returns 0, or -1 on invalid arguments / allocation failure.
 */
int hjo_run_f64(int ndim, const int64_t *shape, const double *dx, double h, const double *P,
                const int64_t *W, double *u, const double *V, int64_t V_step_stride,
                int64_t nsteps, int32_t *amin, int nthreads)
{
    hjo_geom g;
    if (hjo_geom_init(&g, ndim, shape, dx, h, P, W)) { hjo_geom_free(&g); return -1; }
    hjo_set_threads(nthreads);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)g.npts);
    double *hv = (double *)malloc(sizeof(double) * (size_t)g.npts);
    if (!tmp || !hv) { free(tmp); free(hv); hjo_geom_free(&g); return -1; }
    for (int64_t n = 0; n < nsteps; ++n) {
        const double *hvp = NULL;
        if (V) { hjo_hv(g.npts, h, V + n * V_step_stride, hv); hvp = hv; }
        for (int a = 0; a < ndim; ++a) {
            double *src = (a % 2 == 0) ? u : tmp;
            double *dst = (a % 2 == 0) ? tmp : u;
            int last = (a == ndim - 1);
            int32_t *am = amin ? amin + ((size_t)n * ndim + a) * g.npts : NULL;
            hjo_pass_f64(&g, a, src, dst, last ? hvp : NULL, am);
        }
        if (ndim % 2 == 1) memcpy(u, tmp, sizeof(double) * (size_t)g.npts);
    }
    free(tmp);
    free(hv);
    hjo_geom_free(&g);
    return 0;
}

/* Same scheme with binary32 storage (see header). */
int hjo_run_f32(int ndim, const int64_t *shape, const double *dx, double h, const double *P,
                const int64_t *W, float *u, const double *V, int64_t V_step_stride,
                int64_t nsteps, int32_t *amin, int nthreads)
{
    hjo_geom g;
    if (hjo_geom_init(&g, ndim, shape, dx, h, P, W)) { hjo_geom_free(&g); return -1; }
    hjo_set_threads(nthreads);
    float *tmp = (float *)malloc(sizeof(float) * (size_t)g.npts);
    double *hv = (double *)malloc(sizeof(double) * (size_t)g.npts);
    if (!tmp || !hv) { free(tmp); free(hv); hjo_geom_free(&g); return -1; }
    for (int64_t n = 0; n < nsteps; ++n) {
        const double *hvp = NULL;
        if (V) { hjo_hv(g.npts, h, V + n * V_step_stride, hv); hvp = hv; }
        for (int a = 0; a < ndim; ++a) {
            float *src = (a % 2 == 0) ? u : tmp;
            float *dst = (a % 2 == 0) ? tmp : u;
            int last = (a == ndim - 1);
            int32_t *am = amin ? amin + ((size_t)n * ndim + a) * g.npts : NULL;
            hjo_pass_f32(&g, a, src, dst, last ? hvp : NULL, am);
        }
        if (ndim % 2 == 1) memcpy(u, tmp, sizeof(float) * (size_t)g.npts);
    }
    free(tmp);
    free(hv);
    hjo_geom_free(&g);
    return 0;
}

/*
 * Reverse-mode derivative of  J = sum_x ubar_n[x] * u^nsteps[x]  (binary64
 * scheme, static or per-step V as in hjo_run_f64) with respect to u^0, P and
 * V.  Forward argmins are recomputed here and held for the whole run, so this
 * is for small grids.
 *   ubar0: npts, receives dJ/du^0.
 *   Pbar:  ndim, receives dJ/dP_a.
 *   Vbar:  npts (static V) or nsteps*npts (V_step_stride != 0), dJ/dV.
 */
int hjo_adjoint_f64(int ndim, const int64_t *shape, const double *dx, double h, const double *P,
                    const int64_t *W, const double *u0, const double *V, int64_t V_step_stride,
                    int64_t nsteps, const double *ubar_n, double *ubar0, double *Pbar,
                    double *Vbar, int nthreads)
{
    hjo_geom g;
    if (hjo_geom_init(&g, ndim, shape, dx, h, P, W)) { hjo_geom_free(&g); return -1; }
    int64_t npts = g.npts;
    int32_t *amin = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsteps * ndim * npts + 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)npts);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)npts);
    if (!amin || !u || !nxt ||
        (memcpy(u, u0, sizeof(double) * (size_t)npts),
         hjo_run_f64(ndim, shape, dx, h, P, W, u, V, V_step_stride, nsteps, amin, nthreads))) {
        free(amin); free(u); free(nxt); hjo_geom_free(&g);
        return -1;
    }

    double *ub = u; /* reuse: current cotangent */
    memcpy(ub, ubar_n, sizeof(double) * (size_t)npts);
    for (int a = 0; a < ndim; ++a) Pbar[a] = 0.0;
    int64_t nv = (V_step_stride != 0) ? nsteps * npts : npts;
    for (int64_t x = 0; x < nv; ++x) Vbar[x] = 0.0;

    for (int64_t n = nsteps - 1; n >= 0; --n) {
        double *vb = Vbar + ((V_step_stride != 0) ? n * npts : 0);
        for (int64_t x = 0; x < npts; ++x) vb[x] = vb[x] - h * ub[x];
        for (int a = ndim - 1; a >= 0; --a) {
            int64_t outer, inner, N = g.shape[a];
            hjo_axis_split(&g, a, &outer, &inner);
            const int32_t *am = amin + ((size_t)n * ndim + a) * npts;
            for (int64_t x = 0; x < npts; ++x) nxt[x] = 0.0;
            double pb = 0.0;
            for (int64_t line = 0; line < outer * inner; ++line) {
                int64_t o = line / inner, in = line % inner;
                int64_t base = o * N * inner + in;
                for (int64_t i = 0; i < N; ++i) {
                    int64_t x = base + i * inner;
                    int64_t d = am[x];
                    int64_t r = (i - d) % N;
                    if (r < 0) r += N;
                    nxt[base + r * inner] += ub[x];
                    pb += ub[x] * (-(double)d * dx[a]);
                }
            }
            Pbar[a] += pb;
            memcpy(ub, nxt, sizeof(double) * (size_t)npts);
        }
    }
    memcpy(ubar0, ub, sizeof(double) * (size_t)npts);
    free(amin);
    free(u);
    free(nxt);
    hjo_geom_free(&g);
    return 0;
}

/* ------------------------------------------------------------- sampled step */

/* Value after passes 0..a at the point y (coordinates), by the definition of
 * the passes: min over the window of axis a of (value after passes 0..a-1 at
 * y with y_a moved to the source) + k_a[d].  Pass -1 is u itself. */
static double hjo_point_value(const hjo_geom *g, const double *u, int a, int64_t *y)
{
    if (a < 0) {
        int64_t x = 0;
        for (int b = 0; b < g->ndim; ++b) x = x * g->shape[b] + y[b];
        return u[x];
    }
    int64_t N = g->shape[a], keep = y[a];
    double best = 0.0;
    int first = 1;
    for (int64_t d = g->dhi[a]; d >= g->dlo[a]; --d) {
        int64_t r = (keep - d) % N;
        if (r < 0) r += N;
        y[a] = r;
        double cand = hjo_point_value(g, u, a - 1, y) + g->k[a][d - g->dlo[a]];
        if (first || cand < best) { best = cand; first = 0; }
    }
    y[a] = keep;
    return best;
}

/*
 * One step of the binary64 scheme evaluated only at the listed points
 * (flat row-major indices), for checking large grids by sampling.  V: NULL or
 * npts values of the potential for this step.  Returns 0 or -1.
 */
int hjo_step_points_f64(int ndim, const int64_t *shape, const double *dx, double h, const double *P,
                        const int64_t *W, const double *u, const double *V, int64_t npoints,
                        const int64_t *points, double *out, int nthreads)
{
    hjo_geom g;
    if (hjo_geom_init(&g, ndim, shape, dx, h, P, W)) { hjo_geom_free(&g); return -1; }
    hjo_set_threads(nthreads);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < npoints; ++q) {
        int64_t x = points[q];
        if (x < 0 || x >= g.npts) { bad = 1; continue; }
        int64_t y[HJO_MAXDIM];
        int64_t rem = x;
        for (int b = ndim - 1; b >= 0; --b) { y[b] = rem % g.shape[b]; rem /= g.shape[b]; }
        double m = hjo_point_value(&g, u, ndim - 1, y);
        if (V) m = m - h * V[x];
        out[q] = m;
    }
    hjo_geom_free(&g);
    return bad ? -1 : 0;
}
