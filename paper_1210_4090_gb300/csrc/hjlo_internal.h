// hjlo_internal.h -- host-side structures shared by the translation units of
// the hjlo library (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hjlo.h"
#include "hjlo_device.cuh"
#include "hjlo_persist.cuh"

namespace hjlo {

// Resolved geometry, tables and launch shape of one axis of a grid.
struct AxisPlan {
    long long N = 1, inner = 1, outer = 1;
    long long dlo = 0, dhi = 0, centre = 0;
    int weff = 1, hoff = 0;
    double kmin = 0, kmax = 0, curv = 0;
    double *d_kr64 = nullptr;   // device, reversed table
    int algo = KALGO_MONGE;
    int layout = LAYOUT_CONTIG;
    int C = 1, log2C = 0, wpl = 1, threads = 32;
    int lpl = 32, log2lpl = 5, seg = 1;   // MONGE: lanes per line, odd segment
    int gs = 1, tp = 2;                    // MONGE pivot group; argmin row pitch
    long long wait_ns = 500000000LL;       // first TMA wait bound (0.5 s)
    int test_extra_tx = 0;                 // test knob, see apply_test_knobs
    int wide_mul = 2, wide_add = 8;        // warp offload of wide brackets (see PassParams)
    int t8_ok = 1;                         // MONGE: argmin offsets may be bytes (single-grid launches)
    int t8 = 0;                            // MONGE: argmin offsets are bytes (weff <= 256 and t8_ok)
    double eta = 0.0;                      // DECOMP: convexity tolerance of the decomposition
    // DECOMP with a period cut across CTAs (dsplit = 1): chunks of dchunk
    // points (dB per line) for the cut, write-back blocks of dvR outputs
    // (dnblk per line), the passes' device scratch (owned by the plan)
    int dsplit = 0, dchunk = 0, dB = 0, dvR = 0;
    long long dnblk = 0;
    void *d_split = nullptr;
    size_t split_bytes = 0;
    // row blocks of a contiguous axis (vblocks > 1): each line is cut into
    // vblocks blocks of vR rows, each launched as a line of vNp = vR + weff - 1
    // points (see PassParams); the launch fields below then describe those
    long long vblocks = 1, vNp = 0;
    int vR = 0;
    long long rows = 0;                    // rows searched per launched line (0: all N)
    int by = 1, nbox = 1, lp = 0;
    long long ntiles = 0, tiles_per_outer = 1;
    size_t smem = 0;
    int off_u = 0, off_fx = 0, off_kfx = 0, off_t = 0, off_k64 = 0, off_misc = 0;
};

// Records an error for hjlo_last_error() and returns it.
hjlo_status set_error(hjlo_status st, const char *fmt, ...);
hjlo_status cuda_error(cudaError_t e, const char *what);

// Host kernel tables of eq. cost2 for one axis (binary64, fixed order).
double kernel_entry(long long d, double dx, double h, double P);

// The window of displacements [lo, hi] of one axis (eq. los, Sec. 4.2: centred
// on the kernel's largest minimiser c, or the N displacements of the full
// torus window) and k[c].
struct AxisWindow {
    long long lo = 0, hi = 0, centre = 0, weff = 1;
    double kmin = 0.0;
};
hjlo_status resolve_window(long long N, double dx, double h, double P, long long W, AxisWindow &win);

// The reversed table k64[t] = k[hi - t], t < weff, into a caller buffer of at
// least win.weff doubles, and the axis facts (window, hoff, kmax, curvature).
void fill_axis_table(long long N, double dx, double h, double P, const AxisWindow &win, AxisPlan &ax, double *k64);

// resolve_window + fill_axis_table into a malloc'ed table (*kr64_host, freed
// by the caller).
hjlo_status resolve_axis(long long N, double dx, double h, double P, long long W, AxisPlan &ax,
                         double **kr64_host);

// Explicit launch-shape choices (0 / negative: the cost model decides).
struct ShapeHints {
    int lpl = 0;                 // MONGE lanes per line (power of two <= N)
    int C = 0;                   // lines per tile (power of two)
    int wide_mul = -1;           // offload rule of wide brackets (wide_mul, wide_add);
    int wide_add = -1;           // wide_mul = 0 with a huge wide_add turns it off
    long long block_rows = 0;    // rows per row block of a contiguous axis (0: cost model)
};

// The tuning overrides of the environment (HJLO_LANES_PER_LINE,
// HJLO_LINES_PER_TILE, HJLO_OFFLOAD, HJLO_BLOCK_ROWS) as hints.
ShapeHints env_hints();

// Chooses lines per tile, lanes per line and shared-memory layout; `replicas`
// grids of this shape run in the same launch (batched passes).  `hints`
// (null: the environment's) override the cost model where they are valid.
// `row_blocks`: a contiguous axis may be launched as row blocks (single
// grids only; the batched kernel launches whole lines).
hjlo_status shape_launch(AxisPlan &ax, int esize, int algo, int num_sms, size_t smem_optin,
                         long long replicas = 1, const ShapeHints *hints = nullptr, bool row_blocks = true);

// Candidate shapes around ax's current one for the autotuner: lanes per line
// and lines per tile halved / kept / doubled, offload on / off.
std::vector<ShapeHints> tune_candidates(const AxisPlan &ax);

// 3D TMA descriptor {inner, N, outer} of `ptr` for lines along a strided
// axis; false if TMA cannot serve this pointer/shape.
bool encode_strided(const AxisPlan &ax, int esize, const void *ptr, CUtensorMap *map);

// The launch fields of one axis pass (the per-grid pointers left null).
void fill_params(const AxisPlan &ax, PassParams &p);

// The persistent batched pass (hjlo_persist_*.cu): shared-memory opt-in,
// resident CTAs per SM for a launch shape, and the launch.
hjlo_status persist_allow_smem_f64();
hjlo_status persist_allow_smem_f32();
hjlo_status persist_occupancy(int dtype, int threads, size_t smem, int *blocks_per_sm);
hjlo_status persist_launch(int dtype, const PersistParams &pp, int grid, int threads, size_t smem, cudaStream_t st);

// Enqueues one batched pass over `count` grids sharing ax's launch shape.
hjlo_status launch_pass_batch(const AxisPlan &ax, int dtype, const BatchItem *d_items, long long count,
                              unsigned long long *counters, int *flags, cudaStream_t st);

// Enqueues one pass. src/dst may alias.  hv may be null.  amin may be null.
// hv_scale != 0: hv holds V and the potential term is fl(m - fl(hv_scale*V)).
hjlo_status launch_pass(const AxisPlan &ax, int dtype, const void *src, void *dst, const double *hv,
                        double hv_scale, int32_t *amin, unsigned long long *counters, int *flags,
                        cudaStream_t st);

// Device allocation through one place, so tests can inject failures
// (HJLO_TEST_FAIL_ALLOC=k makes the k-th allocation of the process fail).
hjlo_status dmalloc(void **ptr, size_t bytes, const char *what);

// Test knobs read when a plan is created (never set in normal use):
// HJLO_TEST_EXTRA_TX=b makes every TMA barrier expect b bytes more than its
// copy delivers, so the bounded wait runs out (HJLO_ETIMEOUT);
// HJLO_TEST_WAIT_NS=n shortens the first wait to n ns.
void apply_test_knobs(AxisPlan &ax);

// Kernel instantiations, one translation unit per storage type and layout
// (hjlo_kern_*.cu): shared-memory opt-in and launchers.
hjlo_status kern_allow_smem_f64_contig();
hjlo_status kern_single_f64_contig(const AxisPlan &ax, const CUtensorMap &map, const PassParams &p, cudaStream_t st);
hjlo_status kern_batch_f64_contig(const AxisPlan &ax, const BatchItem *items, const PassParams &p, long long count,
                             cudaStream_t st);
hjlo_status kern_allow_smem_f64_strided();
hjlo_status kern_single_f64_strided(const AxisPlan &ax, const CUtensorMap &map, const PassParams &p, cudaStream_t st);
hjlo_status kern_batch_f64_strided(const AxisPlan &ax, const BatchItem *items, const PassParams &p, long long count,
                             cudaStream_t st);
hjlo_status kern_allow_smem_f32_contig();
hjlo_status kern_single_f32_contig(const AxisPlan &ax, const CUtensorMap &map, const PassParams &p, cudaStream_t st);
hjlo_status kern_batch_f32_contig(const AxisPlan &ax, const BatchItem *items, const PassParams &p, long long count,
                             cudaStream_t st);
hjlo_status kern_allow_smem_f32_strided();
hjlo_status kern_single_f32_strided(const AxisPlan &ax, const CUtensorMap &map, const PassParams &p, cudaStream_t st);
hjlo_status kern_batch_f32_strided(const AxisPlan &ax, const BatchItem *items, const PassParams &p, long long count,
                             cudaStream_t st);

// The paper's decomposition method as an axis pass (hjlo_decomp.cu).
hjlo_status decomp_allow_smem();
// The decomposition pass over whole periods cut across CTAs (hjlo_split.cu):
// launch shape and scratch size of an axis, its scratch, its launches.
hjlo_status shape_split(AxisPlan &ax, size_t smem_optin, int num_sms);
size_t split_scratch_bytes(const AxisPlan &ax);
hjlo_status split_allow_smem();
// Per-plan set-up of an axis's scratch (the kernel's slope keys), after it is allocated.
hjlo_status split_prepare(const AxisPlan &ax, cudaStream_t st);
hjlo_status launch_split(const AxisPlan &ax, const void *src, void *dst, const double *hv, double hv_scale,
                         unsigned long long *counters, int *flags, cudaStream_t st);
// blocks_ok: a contiguous axis may run in row blocks (each decomposed on its
// own span); false: whole lines only (EUNSUPPORTED when a line does not fit).
hjlo_status shape_decomp(AxisPlan &ax, size_t smem_optin, int num_sms, bool blocks_ok = true);
hjlo_status launch_decomp(const AxisPlan &ax, const void *src, void *dst, const double *hv, double hv_scale,
                          unsigned long long *counters, int *flags, cudaStream_t st);

// One-time per-device kernel attributes; call outside stream capture.
hjlo_status prepare_kernels();

const char *last_error_cstr();
void clear_error();

// Device properties used for launch shaping.
struct DeviceFacts {
    int device = 0, num_sms = 0;
    size_t smem_optin = 0;
};
hjlo_status device_facts(DeviceFacts &f);

// Graph of a plan's time loop, captured for one (u, h*V) pair.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    const void *u = nullptr;
    const double *hv = nullptr;
};

}  // namespace hjlo

// A plan: one grid, its tables, launch shapes and scratch.
struct hjlo_plan {
    hjlo_desc desc;
    int ndim = 1;
    int dtype = HJLO_F64;
    int algo = HJLO_ALGO_MONGE;
    int decomp_restart = 0;                    // DECOMP: row blocks restart the cut at eta > 0 (approximate)
    long long npts = 1;
    int esize = 8;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    hjlo::AxisPlan ax[HJLO_MAX_DIM];
    unsigned long long *d_counters = nullptr;  // CNT_N
    int *d_flags = nullptr;
    double *d_hv = nullptr;                    // npts, h*V of the current run
    double *d_part = nullptr;                  // readout partials
    void *d_u_host_run = nullptr;              // hjlo_run_host staging
    void *d_scratch = nullptr;                 // npts values: output of in-place row-block passes
    double *d_V_host_run = nullptr;
    hjlo::GraphCache graph;
    long long steps = 0;
    int device = 0;
    // adjoint scratch (allocated on first use)
    double *d_ckpt = nullptr;                  // checkpoints, ckpt_cap states
    long long ckpt_cap = 0;
    int32_t *d_amin = nullptr;                 // argmins of one segment
    long long amin_cap = 0;                    // steps of argmins held
    double *d_work = nullptr;                  // recomputed state
    long long work_cap = 0;
    double *d_pbar_part = nullptr;             // per-line P partials, then one spare slot
    long long pbar_cap = 0;
    double *d_proj = nullptr;                  // projection partials
    long long proj_cap = 0;
};

namespace hjlo {
// Steps of the plan (shared with the adjoint): src -> dst for axis 0, then in
// place; h*V precomputed (hv_scale = 0) or formed in the kernel.
hjlo_status plan_enqueue_step(hjlo_plan *p, const void *src, void *dst, const double *hv, double hv_scale,
                              int32_t *amin, cudaStream_t st);
hjlo_status plan_form_hv(hjlo_plan *p, const double *V);
hjlo_status plan_run(hjlo_plan *p, void *u, const double *V, long long nsteps);
hjlo_status plan_set_device(const hjlo_plan *p);
}  // namespace hjlo
