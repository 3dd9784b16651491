/*
 * hjlo.h -- C ABI of the GB300 (sm_103a) solver for the fully discrete
 * Lax--Oleinik scheme of Bouillard, Faou & Zavidovique, "Fast weak-KAM
 * integrators for separable Hamiltonian systems".
 *
 * The scheme (Sec. 2.3, eq. eqconvol; Sec. 3.3, eq. los): on a periodic grid
 * with space step dx_a along axis a and time step h (the paper's tau),
 *
 *     u^{n+1}(x) = min_y [ u^n(y) + sum_a k_a(x_a - y_a) ] - h V(t_n, x),
 *     k_a[d]     = h * L_a(d dx_a / h),   L_a(v) = v^2/2 - P_a v
 *
 * (the mechanical Hamiltonian H = |p+P|^2/2 + V of eq. HPV; its Legendre
 * dual of Sec. 2.1).  Because the kinetic part is separable the minimum is
 * taken axis by axis (Remark rk28).  Conventions fixed by this library (the
 * paper leaves them open):
 *   - one step = a pass along axis 0 (slowest varying), then axis 1, ...,
 *     then axis ndim-1 (contiguous), then the potential term;
 *   - candidate = one binary64 round-to-nearest add fl(u[j] + k[d]); the
 *     potential term is fl(m - fl(h V)); binary32 storage rounds each pass's
 *     result to nearest binary32 (the last one after the potential term);
 *   - window: displacements d in [c-W, c+W] where c is the largest minimiser
 *     of k_a, or, when W <= 0 or 2W+1 >= N, the N displacements realising the
 *     lift-minimised torus cost of eq. los (equal lift costs keep the larger d);
 *   - argmin = the displacement d of the candidate kept; among equal values
 *     the smallest lifted source j = i - d (the largest d) is kept.
 * Results are identical, bit for bit, between the two algorithms below.
 *
 * Memory: every array argument is a device pointer unless its description
 * says "host".  Arrays are C-contiguous (row-major, last axis contiguous) and
 * owned by the caller; the library never frees them.  A plan owns its kernel
 * tables, its copy of h*V, its status words and any captured CUDA graph.
 * All work is enqueued on the plan's stream and returns without waiting,
 * unless the description says it synchronises.
 *
 * Errors: every call returns an hjlo_status; none aborts, traps or exits.
 * Argument errors are detected before any work is enqueued (HJLO_EINVAL,
 * HJLO_EUNSUPPORTED).  CUDA errors map to HJLO_ECUDA.  hjlo_last_error()
 * returns a description of the last failure on the calling thread.
 */
#ifndef HJLO_H
#define HJLO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HJLO_VERSION 1
#define HJLO_MAX_DIM 3

typedef enum {
    HJLO_OK = 0,
    HJLO_EINVAL = 1,        /* invalid argument (bad sizes, NULL, non-positive steps) */
    HJLO_ENOMEM = 2,        /* device allocation failed */
    HJLO_ECUDA = 3,         /* a CUDA runtime or driver call failed */
    HJLO_EPRECOND = 4,      /* a numerical precondition failed (see hjlo_counters) */
    HJLO_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    HJLO_EUNSUPPORTED = 6   /* valid request the library cannot serve (e.g. line too long) */
} hjlo_status;

typedef enum {
    HJLO_F64 = 0,           /* u stored and computed in binary64 */
    HJLO_F32_STORAGE = 1    /* u stored in binary32, every candidate computed in binary64 */
} hjlo_dtype;

typedef enum {
    HJLO_ALGO_AUTO = 0,     /* library's choice (results do not depend on it) */
    HJLO_ALGO_BRUTE = 1,    /* every window candidate evaluated in binary64 */
    HJLO_ALGO_MONGE = 2,    /* monotone-argmin search (see hjlo_plan_create) */
    HJLO_ALGO_DECOMP = 3    /* the paper's own fast convolution (Sec. 4): convex/concave
                               decomposition of every line; see hjlo_plan_set_decomp */
} hjlo_algo;

/* Problem descriptor (one grid).  Sec. 2.3 eq. cost2 / eqconvol, Sec. 3.3. */
typedef struct {
    int32_t ndim;                 /* 1..3 */
    int32_t dtype;                /* hjlo_dtype */
    int32_t algo;                 /* hjlo_algo */
    int32_t reserved;             /* must be 0 */
    int64_t shape[HJLO_MAX_DIM];  /* N_a >= 1 per axis (entries >= ndim ignored) */
    double dx[HJLO_MAX_DIM];      /* space step per axis, > 0 */
    double h;                     /* time step (the paper's tau), > 0 */
    double P[HJLO_MAX_DIM];       /* the vector P of eq. HPV */
    int64_t window[HJLO_MAX_DIM]; /* W per axis; <= 0 or 2W+1 >= N: full torus window */
} hjlo_desc;

typedef struct hjlo_plan hjlo_plan;

/* What a plan resolved (host struct filled by hjlo_plan_info). */
typedef struct {
    int32_t ndim;
    int32_t algo;                 /* resolved algorithm: BRUTE or MONGE */
    int64_t dlo[HJLO_MAX_DIM];    /* window [dlo, dhi] of displacements per axis */
    int64_t dhi[HJLO_MAX_DIM];
    int64_t centre[HJLO_MAX_DIM]; /* largest minimiser of k_a */
    double kmin[HJLO_MAX_DIM];    /* min_d k_a[d] */
    double curvature[HJLO_MAX_DIM]; /* min second difference of the k_a table */
    int64_t npts;                 /* prod(shape) */
    int64_t row_blocks[HJLO_MAX_DIM]; /* 1: each CTA stages whole lines of axis a; k > 1: every
                                     line of the contiguous axis is cut into k blocks of rows,
                                     each staged with the window span it needs (lines longer
                                     than one CTA's shared memory, or too few lines to fill
                                     the GPU; windows up to a quarter of the line) */
    int64_t block_rows[HJLO_MAX_DIM]; /* rows per block when row_blocks[a] > 1 (the last block
                                     holds the rest), else 0 */
    int64_t split_chunks[HJLO_MAX_DIM]; /* HJLO_ALGO_DECOMP: 0, or the number of chunks each
                                     line's period is cut into when its decomposition runs
                                     whole across CTAs (see hjlo_plan_set_decomp) */
} hjlo_plan_facts;

/* Device-side counters of a plan (host struct filled by hjlo_sync). */
typedef struct {
    int64_t exact_rescans;        /* outputs whose fixed-point screen left >1 survivor (binary64 re-scan) */
    int64_t brute_fallback_lines; /* lines the monotone search handed to brute force */
    int64_t steps;                /* time steps enqueued on this plan so far */
    int32_t error_flags;          /* bit 0: precondition, bit 1: wait timeout */
    int32_t reserved;
    int64_t components;           /* HJLO_ALGO_DECOMP: convex/concave components convolved */
    int64_t window_edge_hits;     /* outputs of brute or monotone passes with a partial window
                                     (2W+1 < N) whose argmin is its first or last displacement
                                     (d = c - W or c + W).  Zero means no output of those passes
                                     sat on the window's edge; a nonzero count says the window
                                     may have cut off a smaller candidate of the full torus
                                     window (eq. los).  Autotuner trials are not counted. */
} hjlo_counters;

/*
 * Create a plan for one grid on a CUDA stream (cudaStream_t, may be NULL for
 * the default stream).  Builds the kernel tables k_a[d] of eq. cost2 on the
 * host in the fixed binary64 order, resolves the window (eq. los, Sec. 4.2)
 * and uploads them.  HJLO_ALGO_MONGE relies on the candidate matrix
 * u[j] + k[i-j] being Monge, which holds because k_a is convex (hypothesis
 * (i), Sec. 2.1): its row minima move monotonically, so each output is
 * searched in a narrow range bracketed by its neighbours' argmins.  The plan
 * checks that the table's second differences are positive; each launch
 * re-checks the rounding margin per line and falls back to brute force for a
 * line that fails it (counted in hjlo_counters).  A contiguous axis whose
 * lines are longer than one CTA's shared memory holds, or too few to fill the
 * GPU, is launched in blocks of rows when its window is at most a quarter of
 * the line: each block is staged with the window span its rows need, so the
 * results are those of whole lines (hjlo_plan_facts.row_blocks).  Other lines
 * too long for the monotone search (full or wide windows, strided axes) take
 * brute force under HJLO_ALGO_AUTO where that fits.
 * HJLO_ALGO_DECOMP runs every pass by the paper's own method (Sec. 4): each
 * line is cut into convex and concave components (tolerance eta, Sec. 4.4,
 * default 0), each is convolved with the convex kernel in linear time
 * (Theorem th:convex, Algorithm 1; Lemmas lm:seg, lm:simplif, Theorem th:ccc,
 * Algorithm 2) and the minimum over components is taken.  Its outputs are
 * candidates of the scheme (never below it; equal to it in exact arithmetic
 * at eta = 0).  It needs binary64 storage, a strictly convex table
 * (HJLO_EPRECOND otherwise) and records no argmins (hjlo_step with
 * argmin_out and hjlo_adjoint return HJLO_EUNSUPPORTED).
 * Errors: HJLO_EINVAL (bad descriptor), HJLO_EUNSUPPORTED (a line of the grid
 * does not fit in one CTA's shared memory and cannot run in row blocks or,
 * for HJLO_ALGO_DECOMP, with its period spread across CTAs),
 * HJLO_EPRECOND, HJLO_ENOMEM, HJLO_ECUDA.
 */
hjlo_status hjlo_plan_create(const hjlo_desc *desc, void *cuda_stream, hjlo_plan **out);

/* What an autotuning call chose (host struct; see hjlo_plan_autotune). */
typedef struct {
    int32_t lanes_per_line[HJLO_MAX_DIM]; /* monotone search: lanes per line (0: axis not tuned) */
    int32_t lines_per_tile[HJLO_MAX_DIM]; /* lines per CTA */
    int32_t offload[HJLO_MAX_DIM];        /* 1: wide brackets searched by warp groups */
    int32_t trials;                       /* launch shapes timed */
    double ms_initial;                    /* trial run with the starting shapes (ms) */
    double ms_tuned;                      /* trial run with the chosen shapes (ms) */
} hjlo_tune_report;

/* Release a plan and everything it owns.  NULL is accepted.  Synchronises
 * the plan's stream first. */
hjlo_status hjlo_plan_destroy(hjlo_plan *plan);

/* Copy the resolved windows and table facts into *info (host). */
hjlo_status hjlo_plan_info(const hjlo_plan *plan, hjlo_plan_facts *info);

/*
 * Convexity tolerance eta >= 0 of an HJLO_ALGO_DECOMP plan (Sec. 4.4): a
 * component stays "convex" while the increase of its slopes, taken per unit
 * length ((u(i+1) - u(i)) / dx_a), is >= -eta (second differences
 * >= -eta * dx_a), so nearly affine stretches join fewer, longer components
 * (fewer components, larger values where the stretch is not convex).
 *
 * Each pass decomposes every line once over one period (its lifted span),
 * as Sec. 4.2-4.3 take the function on the torus.  At eta = 0 the method is
 * exact (every component is convex or concave: Theorems th:convex and
 * th:ccc), so the result does not depend on where the cut starts and long
 * or lonely contiguous lines run in row blocks, each cut on its own span.
 * At eta > 0 the result does depend on the cut: with restart_blocks = 0 each
 * line is decomposed whole.  A line longer than one CTA holds (about 7000
 * points) then has its period's cut and convolutions spread over many CTAs
 * (chunks of the span cut locally and stitched into the one greedy cut of
 * the whole period, then blocks of outputs; hjlo_plan_facts.split_chunks),
 * with the same result as one CTA holding the whole line.  restart_blocks =
 * 1 instead runs such lines in row blocks that restart the decomposition at
 * each block's first source, an approximation of the method with no
 * counterpart in the paper: every output is still one candidate
 * fl(u(y) + k(d)) of the scheme, so never below it, and a component of m
 * pieces treated as convex adds at most eta dx_a m^2 to it (m <= block rows
 * + window - 1).
 *
 * Waits for the plan's stream; later steps use the new settings (the
 * plan's cached graph is rebuilt).  Errors: HJLO_EINVAL (another algorithm,
 * eta negative or not finite, restart_blocks not 0 or 1), HJLO_EUNSUPPORTED
 * (a window too wide for the pass's shared memory), HJLO_ENOMEM; on error
 * the plan keeps its previous settings.
 */
hjlo_status hjlo_plan_set_decomp(hjlo_plan *plan, double eta, int32_t restart_blocks);

/* hjlo_plan_set_decomp(plan, eta, 0). */
hjlo_status hjlo_plan_set_tolerance(hjlo_plan *plan, double eta);

/*
 * Autotune the launch shapes of a plan's monotone passes (no counterpart in
 * the paper: results never depend on the launch shape, only the time does).
 * Axis by axis, shapes around the current one -- lanes per line and lines
 * per tile halved / kept / doubled, wide-bracket offload on / off, and for
 * an axis in row blocks the rows per block halved / kept / doubled -- are
 * timed with CUDA events on nsteps steps from a device copy of u (u itself
 * is not modified; V: npts binary64 or NULL), and each axis keeps the
 * fastest (a candidate must beat the incumbent by 2 %).  Trial launches
 * leave the plan's counters as they were.  Synchronous; the plan's cached
 * graph is rebuilt on next use.  report (host, may be NULL) receives the
 * choice (hjlo_plan_info gives the row blocks).  Brute-force and
 * decomposition axes are left as they are.  Errors: HJLO_EINVAL (NULL
 * plan/u, nsteps < 1), HJLO_ENOMEM, HJLO_ECUDA.
 */
hjlo_status hjlo_plan_autotune(hjlo_plan *plan, const void *u, const double *V, int64_t nsteps,
                               hjlo_tune_report *report);

/*
 * One time step (eq. eqconvol): u_out = T(u_in).  u_in and u_out hold npts
 * values of the plan's dtype and may be the same pointer (in place).  V: npts
 * binary64 values of V(t_n, .) or NULL for V = 0; V must not overlap u_in,
 * u_out or argmin_out (it is read through the read-only cache while the
 * outputs are written).  argmin_out: NULL, or
 * ndim*npts int32 receiving the argmin displacement d of every pass, laid out
 * [axis][point] (the discrete optimal path of eq. raslebol, one step).
 */
hjlo_status hjlo_step(hjlo_plan *plan, const void *u_in, void *u_out, const double *V,
                      int32_t *argmin_out);

/*
 * nsteps time steps in place on u (eq. uN) with a time-independent V (NULL
 * for V = 0).  h*V is formed once per call.  The step loop is replayed from a
 * CUDA graph captured on first use for this (u, V) pair.
 */
hjlo_status hjlo_run(hjlo_plan *plan, void *u, const double *V, int64_t nsteps);

/*
 * Time-dependent potential: step n uses V + n*npts (V holds nsteps*npts
 * binary64 values, V(t_n, .) for n = 0..nsteps-1).  In place on u.
 */
hjlo_status hjlo_run_tv(hjlo_plan *plan, void *u, const double *V, int64_t nsteps);

/*
 * End-to-end variant of hjlo_run for HOST buffers: copies u_host (and
 * V_host, may be NULL) to plan-owned device memory, runs nsteps, copies the
 * result back into u_host and synchronises.  u_host holds npts values of the
 * plan's dtype (host), V_host npts binary64 (host).  Page-locked host memory
 * gives the fastest copies.
 */
hjlo_status hjlo_run_host(hjlo_plan *plan, void *u_host, const double *V_host, int64_t nsteps);

/*
 * Discrete effective Hamiltonian readout (Prop. prop:klm with the sign of
 * u_t + H = 0): r(x) = (u_n(x) - u_0(x)) / (nsteps h); writes to the HOST
 * array out3 = { -mean_x r, -max_x r, -min_x r } (estimate, lower, upper).
 * Synchronises the plan's stream.
 */
hjlo_status hjlo_hbar(hjlo_plan *plan, const void *u0, const void *un, int64_t nsteps,
                      double *out3);

/*
 * Reverse mode of nsteps steps of a binary64 plan with time-independent V:
 * the gradient of J = <ubar_n, u^nsteps> with respect to u^0, P and V.  Every
 * value of a pass comes from one source along the discrete optimal path
 * (eq. raslebol, Appendix B), so the transpose of a pass routes the
 * cotangent back along the recorded argmins; dk/dP_a = -d*dx_a (eq. cost2);
 * the potential term of eq. eqconvol gives dJ/dV = -h * sum_n ubar^{n+1}.
 * Forward states are checkpointed every `checkpoint_every` steps (<= 0: one
 * segment) and each segment is recomputed once with argmin recording.
 *   u0, V (may be NULL), ubar_n: npts binary64 (device).
 *   ubar_0: npts (device), receives dJ/du^0 (may not alias ubar_n).
 *   Pbar: NULL or ndim binary64 (device), receives dJ/dP.
 *   Vbar: NULL or npts binary64 (device), receives dJ/dV.
 *   u_n: NULL or npts binary64 (device), receives u^nsteps.
 * ubar_0 and Vbar are summed in the order of the definition (ascending target
 * per source), Pbar in a fixed but different order.  Plan-owned scratch:
 * checkpoints (ceil(nsteps/S) states), argmins (S*ndim*npts int32), one
 * state, per-line partials.  Errors: HJLO_EUNSUPPORTED for binary32 plans.
 */
hjlo_status hjlo_adjoint(hjlo_plan *plan, const double *u0, const double *V, int64_t nsteps,
                         const double *ubar_n, double *ubar_0, double *Pbar, double *Vbar,
                         int64_t checkpoint_every, double *u_n);

/* out[k] = sum_x field(x) * basis[k*npts + x] for k < nbasis (device arrays,
 * binary64; fixed summation order): gradients of coefficients of a potential
 * V = sum_k c_k basis_k from Vbar. */
hjlo_status hjlo_project(hjlo_plan *plan, const double *field, const double *basis, int32_t nbasis,
                         double *out);

/*
 * Batched grids: `count` independent instances of the scheme (each its own
 * descriptor: P, grid size, window, h) advanced together -- the sweep of the
 * discrete effective Hamiltonian over P of Prop. prop:klm.  Instances with
 * the same shape and window sizes share kernel launches (the convolution
 * blocks are independent, Sec. 4.1), and the groups run as parallel branches
 * of one captured CUDA graph.  Every instance's result is identical, bit for
 * bit, to a single plan's.  All descriptors must share ndim and dtype.
 * Errors as hjlo_plan_create (the message names the instance).
 */
typedef struct hjlo_batch hjlo_batch;
hjlo_status hjlo_batch_create(const hjlo_desc *descs, int32_t count, void *cuda_stream, hjlo_batch **out);

/* Release a batch (synchronises its stream first).  NULL is accepted. */
hjlo_status hjlo_batch_destroy(hjlo_batch *batch);

/*
 * nsteps time steps of every instance, in place.  u: host array of `count`
 * device pointers (instance i: npts_i values of the dtype).  V: NULL, or a
 * host array of `count` device pointers to time-independent binary64
 * potentials (an entry may be NULL for V = 0).
 */
hjlo_status hjlo_batch_run(hjlo_batch *batch, void *const *u, const double *const *V, int64_t nsteps);

/* hjlo_hbar for every instance: out3 (host) receives 3*count doubles,
 * {estimate, lower, upper} per instance.  Synchronises the batch's stream. */
hjlo_status hjlo_batch_hbar(hjlo_batch *batch, const void *const *u0, const void *const *un, int64_t nsteps,
                            double *out3);

/* hjlo_sync for a batch. */
hjlo_status hjlo_batch_sync(hjlo_batch *batch, hjlo_counters *out);

/*
 * hjlo_plan_autotune for a batch: the shape of every launch group's monotone
 * passes is tuned by timing nsteps steps of the whole batch (all groups
 * together, as they run) from device copies of u[i].  report's per-axis
 * fields describe the group with the most points.
 */
hjlo_status hjlo_batch_autotune(hjlo_batch *batch, const void *const *u, const double *const *V, int64_t nsteps,
                                hjlo_tune_report *report);

/* Number of launch groups the batch formed (0 for NULL). */
int32_t hjlo_batch_groups(const hjlo_batch *batch);

/*
 * How a batch's time steps are launched (no counterpart in the paper; the
 * results are the same bit for bit either way).  on = 0: one kernel launch
 * per launch group and axis, the groups as parallel branches of the
 * captured graph.  on = 1: one persistent launch per time step over every
 * instance and axis.  Its CTAs (as many as fit the GPU at once) take work
 * items -- a few tiles of one instance's pass -- from a device queue that
 * lists every axis-a item before any axis-(a+1) item; an item of axis a >= 1
 * first waits until every tile of its instance's axis a - 1 pass is done (a
 * per-instance tile counter), because that pass writes the grid this one
 * reads.  Waits only point at items taken earlier by running CTAs, so the
 * launch cannot deadlock; each wait is bounded (1 s), after which the
 * launch raises the timeout flag that hjlo_batch_sync reports as
 * HJLO_ETIMEOUT and skips the remaining waits.  The launch uses the largest
 * thread count and shared memory of the groups' shapes.  Every instance must
 * run the monotone search.  Waits for the batch's stream; the next
 * hjlo_batch_run rebuilds the graph.  Errors: HJLO_EINVAL (NULL batch, on
 * not 0 or 1), HJLO_EUNSUPPORTED (an instance runs brute force).
 */
hjlo_status hjlo_batch_set_persistent(hjlo_batch *batch, int32_t on);

/* Wait for the plan's stream and copy its device counters into *out (host,
 * may be NULL).  Returns HJLO_EPRECOND / HJLO_ETIMEOUT if a launch since the
 * last call raised the corresponding flag (the flags are then cleared). */
hjlo_status hjlo_sync(hjlo_plan *plan, hjlo_counters *out);

/*
 * The first discrete semigroup (Sec. 2.2, eq. cost1): the cost of a step is
 * the action of the straight path from the source y to the target x in time
 * h, c(y, x) = h K*(v) - int_0^h V(y + s v) ds, v = (x - y)/h, and
 * u'(x) = min_y u(y) + c(y, x) over the box of the per-axis windows of
 * desc (the potential term does not separate by axis: every candidate of
 * the box is evaluated).  V is time-independent and given as a Fourier series
 * on the torus of side L_a = shape[a] * dx[a]:
 *   V(x) = Re sum_m c_m exp(2 pi i sum_a modes[m][a] x_a / L_a),
 * for which the path integral is exact (no quadrature rule):
 *   h Re sum_m c_m exp(i alpha_m(y)) phi(theta_m(x - y)),
 *   phi(theta) = (exp(i theta) - 1)/(i theta).
 * modes: nmodes * ndim int32, coef: nmodes * 2 binary64 (re, im), host,
 * copied.  desc->dtype must be HJLO_F64, desc->algo AUTO or BRUTE.  Tables
 * (per point and mode, per displacement) are formed on the host in binary64
 * with the C library's sin and cos; the sum over modes uses fused
 * multiply-adds.  Errors: HJLO_EINVAL, HJLO_EUNSUPPORTED
 * (grid x box x modes too large), HJLO_ENOMEM, HJLO_ECUDA.
 */
typedef struct hjlo_integral hjlo_integral;
hjlo_status hjlo_integral_create(const hjlo_desc *desc, int32_t nmodes, const int32_t *modes, const double *coef,
                                 void *cuda_stream, hjlo_integral **out);

/* nsteps steps in place on u (npts binary64, device); a ping-pong buffer of
 * the plan holds every other step. */
hjlo_status hjlo_integral_run(hjlo_integral *plan, double *u, int64_t nsteps);

/* Wait for the plan's stream. */
hjlo_status hjlo_integral_sync(hjlo_integral *plan);

/* Release the plan (NULL accepted). */
hjlo_status hjlo_integral_destroy(hjlo_integral *plan);

/* Largest window (displacements per axis, after resolving W) served by
 * hjlo_step_noalloc. */
#define HJLO_NOALLOC_MAX_WINDOW 8192

/*
 * One time step, as hjlo_step with argmin_out = NULL, without a plan and
 * without allocating anything -- for callers that cannot allocate device
 * memory (a framework whose caching allocator must own all device memory,
 * code running while another thread captures a CUDA graph, latency-bound
 * loops that cannot afford an allocation's implicit synchronisation).  The
 * paper has no counterpart: this is a deployment variant of the same step.
 *   desc: the grid (host); every window must resolve to at most
 *         HJLO_NOALLOC_MAX_WINDOW displacements, else HJLO_EUNSUPPORTED.
 *   cuda_stream: cudaStream_t (may be NULL); all work is enqueued on it.
 *   u_in, u_out: npts values of desc->dtype (device), equal or disjoint.
 *   V: npts binary64 (device) or NULL; h*V is formed inside the kernel.
 * Scratch: the kernel tables and device counters live in one static device
 * array of the library (about 200 KB per GPU that loads it, held until the
 * process exits); every call overwrites it and clears the counters, so calls
 * whose GPU work overlaps (other streams, other threads) race.  The first
 * call on a device looks up the array's device address and sets kernel
 * attributes; make that first call before any stream capture.  The kernel
 * tables are copied from host (pageable) memory, which orders the copy after
 * earlier work on the stream.  Results equal hjlo_step's bit for bit.
 * Errors found on the device (a bounded wait that ran out, a failed
 * precondition) cannot be returned by this asynchronous call: they collect
 * in the array's error word, which no step clears; hjlo_noalloc_status
 * reports and clears them.  Argument errors are returned at once.
 */
hjlo_status hjlo_step_noalloc(const hjlo_desc *desc, void *cuda_stream, const void *u_in, void *u_out,
                              const double *V);

/*
 * The device status of hjlo_step_noalloc calls on the current device (no
 * counterpart in the paper).  Waits for cuda_stream, copies the static
 * array's counters of the most recent step and its error word into *out
 * (host, may be NULL; fields a step does not keep are 0), clears the error
 * word and returns HJLO_ETIMEOUT (a bounded device wait gave up: that
 * step's output is incomplete) or HJLO_EPRECOND if any step since the
 * previous status call raised one, else HJLO_OK.  Allocates nothing.
 * Errors: HJLO_ECUDA.
 */
hjlo_status hjlo_noalloc_status(void *cuda_stream, hjlo_counters *out);

/* Launch shape of one axis pass (host struct; see hjlo_shape_query). */
typedef struct {
    int32_t lanes_per_line;       /* threads per launched line (monotone search: lanes, one segment each) */
    int32_t segment_rows;         /* monotone search: rows per lane segment (odd); brute force: 1 */
    int32_t lines_per_tile;       /* launched lines per CTA */
    int32_t threads;              /* threads per CTA */
    int64_t smem_bytes;           /* dynamic shared memory per CTA */
    int64_t tiles;                /* CTAs per pass launch */
    int64_t row_blocks;           /* 1: whole lines; k > 1: every line cut into k blocks of rows */
    int64_t block_rows;           /* rows per block (the last holds the rest); 0 for whole lines */
    int64_t line_points;          /* points staged per launched line: N, or block_rows + weff - 1 */
    int64_t split_chunks;         /* HJLO_ALGO_DECOMP: 0, or the chunks of each line's period when its
                                     decomposition runs across CTAs; tiles then counts the CTAs of the
                                     write-back launch */
    int64_t split_rows;           /* outputs per write-back CTA of that launch (0 otherwise) */
} hjlo_shape_info;

/*
 * The launch shape that hjlo_plan_create chooses for a contiguous axis of
 * `lines` lines of N points with a window of weff displacements (1 <= weff
 * <= N; weff = N is the full torus window), for a GPU with num_sms SMs and
 * smem_optin bytes of opt-in shared memory per CTA.  Host only: no device is
 * touched.  esize: 8 (binary64) or 4 (binary32 storage); algo:
 * HJLO_ALGO_BRUTE, HJLO_ALGO_MONGE or HJLO_ALGO_DECOMP (binary64 only, a
 * strictly convex table assumed; one CTA per line or row block, whose
 * threads are reported as lanes_per_line, segment_rows 0).  The
 * environment's tuning overrides apply as for a plan.  Errors: HJLO_EINVAL (bad arguments, NULL out),
 * HJLO_EUNSUPPORTED (the lines do not fit and cannot run in row blocks).
 */
hjlo_status hjlo_shape_query(int64_t N, int64_t lines, int64_t weff, int32_t esize, int32_t algo, int32_t num_sms,
                             int64_t smem_optin, hjlo_shape_info *out);

/*
 * The binary64 add rate of the current device (a measurement helper, no
 * counterpart in the paper: the brute-force pass is bound by one binary64
 * add per window candidate).  Launches, on cuda_stream, a kernel whose
 * threads run 8 independent add chains of `iters` adds each (grid: 8 CTAs of
 * 256 threads per SM), once to warm up and once timed with CUDA events;
 * *adds_per_s (host) receives adds / elapsed time.  Synchronous.  Errors:
 * HJLO_EINVAL (iters outside 1..2^30, NULL output), HJLO_ECUDA.
 */
hjlo_status hjlo_probe_fp64_add(int64_t iters, void *cuda_stream, double *adds_per_s);

/* Description of the last error on the calling thread ("" if none). */
const char *hjlo_last_error(void);

/* HJLO_VERSION of the loaded library. */
int32_t hjlo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HJLO_H */
