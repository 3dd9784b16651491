// hjlo_batch.cu -- many independent grids advanced together (sweeps of the
// effective Hamiltonian over P, Prop. prop:klm): every instance runs the
// scheme of eq. uN with its own P, V, grid size and window.
//
// Instances are grouped by launch shape (same shape and window size per
// axis, so the same tile geometry); one kernel launch per group and axis
// covers the tiles of all its instances, the fields that differ (pointers,
// kernel tables, window offsets, TMA descriptors) coming from a device array
// of BatchItem.  The groups are independent branches of one captured CUDA
// graph (fork/join on per-group streams), replayed for the time loop.  The
// convolution blocks are independent (distributivity of min-plus convolution
// over min, Sec. 4.1), so grouping changes nothing in the results: each
// instance is bit-identical to a single-grid plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "hjlo_internal.h"

using namespace hjlo;

namespace hjlo {
hjlo_status persist_occupancy_f64(int threads, size_t smem, int *blocks_per_sm);
hjlo_status persist_occupancy_f32(int threads, size_t smem, int *blocks_per_sm);
hjlo_status persist_launch_f64(const PersistParams &pp, int grid, int threads, size_t smem, cudaStream_t st);
hjlo_status persist_launch_f32(const PersistParams &pp, int grid, int threads, size_t smem, cudaStream_t st);

hjlo_status persist_occupancy(int dtype, int threads, size_t smem, int *blocks_per_sm)
{
    return dtype == HJLO_F64 ? persist_occupancy_f64(threads, smem, blocks_per_sm)
                             : persist_occupancy_f32(threads, smem, blocks_per_sm);
}

hjlo_status persist_launch(int dtype, const PersistParams &pp, int grid, int threads, size_t smem, cudaStream_t st)
{
    return dtype == HJLO_F64 ? persist_launch_f64(pp, grid, threads, smem, st)
                             : persist_launch_f32(pp, grid, threads, smem, st);
}
}  // namespace hjlo

namespace {

constexpr int kBatchGraphSteps = 8;
constexpr int kRedBlocks = 32;
constexpr int kRedThreads = 256;

struct Group {
    std::vector<int> members;
    AxisPlan ax[HJLO_MAX_DIM];         // shared launch shape (tables per instance)
    BatchItem *d_items[HJLO_MAX_DIM] = {nullptr, nullptr, nullptr};
    std::vector<BatchItem> h_items[HJLO_MAX_DIM];
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct hjlo_batch {
    int count = 0, ndim = 1, dtype = HJLO_F64, esize = 8, device = 0;
    std::vector<hjlo_desc> descs;
    std::vector<long long> npts, hv_off;
    std::vector<AxisPlan> inst;        // count * ndim, per-instance tables and offsets
    std::vector<Group> groups;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaEvent_t fork = nullptr;
    unsigned long long *d_counters = nullptr;
    int *d_flags = nullptr;
    double *d_hv = nullptr;
    double *d_part = nullptr;
    cudaGraphExec_t graph_many = nullptr, graph_one = nullptr;
    std::vector<const void *> graph_u;
    std::vector<const double *> graph_v;
    long long steps = 0;
    // persistent mode (hjlo_batch_set_persistent): one launch per time step
    int persist = 0;
    bool pbuilt = false;                 // work list and shapes match the groups' current shapes
    PersistItem *d_pwork = nullptr;
    PassParams *d_pshapes = nullptr;
    BatchItem *d_pitems = nullptr;       // [axis * count + instance]
    int *d_ptiles = nullptr;             // [instance * ndim + axis]
    unsigned long long *d_pstate = nullptr;   // the queue word, then done[count * ndim] (32-bit)
    size_t pstate_bytes = 0;
    std::vector<BatchItem> h_pitems;
    long long pnwork = 0;
    int pgrid = 0, pthreads = 0;
    size_t psmem = 0;
    long long pwait_ns = 1000000000LL;   // bound on a dependency wait (1 s)
    int ptest_extra_dep = 0;             // test knob HJLO_TEST_EXTRA_DEP
};

namespace {

__global__ void batch_scale_kernel(const double *__restrict__ V, double h, double *__restrict__ hv, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        hv[i] = __dmul_rn(h, V[i]);
}

struct DiffArgs {
    const void *u0;
    const void *un;
    long long n;
};

// Partial (sum, min, max) of un - u0 per (instance, block), fixed order.
template <typename T>
__global__ void batch_diff_partials(const DiffArgs *__restrict__ args, double *__restrict__ part)
{
    __shared__ double ss[kRedThreads], smn[kRedThreads], smx[kRedThreads];
    const DiffArgs a = args[blockIdx.y];
    const T *u0 = static_cast<const T *>(a.u0);
    const T *un = static_cast<const T *>(a.un);
    double s = 0.0, mn = INFINITY, mx = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
         i += (long long)gridDim.x * blockDim.x) {
        double d = __dsub_rn((double)un[i], (double)u0[i]);
        s = __dadd_rn(s, d);
        mn = fmin(mn, d);
        mx = fmax(mx, d);
    }
    ss[threadIdx.x] = s;
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int o = kRedThreads / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] = __dadd_rn(ss[threadIdx.x], ss[threadIdx.x + o]);
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *q = part + 3 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
        q[0] = ss[0];
        q[1] = smn[0];
        q[2] = smx[0];
    }
}

__global__ void batch_fold(const double *__restrict__ part, int nblocks, long long count, double *__restrict__ out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s = 0.0, mn = INFINITY, mx = -INFINITY;
    for (int b = 0; b < nblocks; ++b) {
        const double *q = part + 3 * (i * nblocks + b);
        s = __dadd_rn(s, q[0]);
        mn = fmin(mn, q[1]);
        mx = fmax(mx, q[2]);
    }
    out[3 * i + 0] = s;
    out[3 * i + 1] = mn;
    out[3 * i + 2] = mx;
}

hjlo_status validate_desc(const hjlo_desc *d, long long *npts)
{
    if (d->ndim < 1 || d->ndim > HJLO_MAX_DIM) return set_error(HJLO_EINVAL, "ndim must be 1..3");
    if (d->dtype != HJLO_F64 && d->dtype != HJLO_F32_STORAGE) return set_error(HJLO_EINVAL, "unknown dtype");
    if (d->algo == HJLO_ALGO_DECOMP) return set_error(HJLO_EUNSUPPORTED, "batches run the brute or monotone pass");
    if (d->algo < HJLO_ALGO_AUTO || d->algo > HJLO_ALGO_MONGE) return set_error(HJLO_EINVAL, "unknown algo");
    if (d->reserved != 0) return set_error(HJLO_EINVAL, "reserved field must be 0");
    if (!(d->h > 0) || !std::isfinite(d->h)) return set_error(HJLO_EINVAL, "h must be finite and > 0");
    long long n = 1;
    for (int a = 0; a < d->ndim; ++a) {
        if (d->shape[a] < 1) return set_error(HJLO_EINVAL, "shape[%d] must be >= 1", a);
        if (d->shape[a] > (1LL << 24)) return set_error(HJLO_EUNSUPPORTED, "shape[%d] too large", a);
        if (!(d->dx[a] > 0) || !std::isfinite(d->dx[a])) return set_error(HJLO_EINVAL, "dx[%d] must be > 0", a);
        if (!std::isfinite(d->P[a])) return set_error(HJLO_EINVAL, "P[%d] must be finite", a);
        n *= d->shape[a];
        if (n > (1LL << 40)) return set_error(HJLO_EUNSUPPORTED, "grid too large");
    }
    *npts = n;
    return HJLO_OK;
}

void release(hjlo_batch *b)
{
    if (b->graph_many) cudaGraphExecDestroy(b->graph_many);
    if (b->graph_one) cudaGraphExecDestroy(b->graph_one);
    for (auto &g : b->groups) {
        for (int a = 0; a < HJLO_MAX_DIM; ++a) cudaFree(g.d_items[a]);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    for (auto &ax : b->inst) cudaFree(ax.d_kr64);
    cudaFree(b->d_pwork);
    cudaFree(b->d_pshapes);
    cudaFree(b->d_pitems);
    cudaFree(b->d_ptiles);
    cudaFree(b->d_pstate);
    cudaFree(b->d_counters);
    cudaFree(b->d_flags);
    cudaFree(b->d_hv);
    cudaFree(b->d_part);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

// Copy a launch shape onto a group and every member of it (their tables and
// window offsets stay their own).
void apply_group_shape(hjlo_batch *b, Group &g, int a, const AxisPlan &ax)
{
    for (int i : g.members) {
        AxisPlan &m = b->inst[(size_t)i * b->ndim + a];
        AxisPlan keep = m;
        m = ax;
        m.d_kr64 = keep.d_kr64;
        m.dlo = keep.dlo;
        m.dhi = keep.dhi;
        m.centre = keep.centre;
        m.hoff = keep.hoff;
        m.kmin = keep.kmin;
        m.kmax = keep.kmax;
        m.curv = keep.curv;
    }
    g.ax[a] = ax;
    g.ax[a].d_kr64 = nullptr;
}

void drop_graphs(hjlo_batch *b)
{
    if (b->graph_many) cudaGraphExecDestroy(b->graph_many);
    if (b->graph_one) cudaGraphExecDestroy(b->graph_one);
    b->graph_many = nullptr;
    b->graph_one = nullptr;
    b->pbuilt = false;                   // shapes may have changed
}

// The persistent launch's work list, launch shapes and state (device), from
// the groups' current shapes.  Items of one axis come in groups of tiles of
// one instance, largest instances first within an axis; an axis's items all
// precede the next axis's, so every dependency wait points at items taken
// earlier.  Chunks are sized for about 32 items per resident CTA.
hjlo_status build_persist(hjlo_batch *b)
{
    const int nd = b->ndim, count = b->count;
    const int ng = (int)b->groups.size();
    std::vector<PassParams> shapes((size_t)ng * nd);
    int threads = 32;
    size_t smem = 0;
    for (int gi = 0; gi < ng; ++gi)
        for (int a = 0; a < nd; ++a) {
            const AxisPlan &ax = b->groups[gi].ax[a];
            if (ax.algo != KALGO_MONGE)
                return set_error(HJLO_EUNSUPPORTED, "the persistent batch runs the monotone search only");
            PassParams &pp = shapes[(size_t)gi * nd + a];
            fill_params(ax, pp);
            pp.counters = b->d_counters;
            pp.flags = b->d_flags;
            threads = std::max(threads, ax.threads);
            smem = std::max(smem, ax.smem);
        }
    int per_sm = 0;
    hjlo_status s = persist_occupancy(b->dtype, threads, smem, &per_sm);
    if (s != HJLO_OK) return s;
    if (per_sm < 1) return set_error(HJLO_EUNSUPPORTED, "the persistent batch's launch shape does not fit an SM");
    DeviceFacts df;
    if ((s = device_facts(df)) != HJLO_OK) return s;
    const int grid = df.num_sms * per_sm;
    std::vector<int> tiles((size_t)count * nd);
    long long total = 0;
    for (int gi = 0; gi < ng; ++gi)
        for (int i : b->groups[gi].members)
            for (int a = 0; a < nd; ++a) {
                tiles[(size_t)i * nd + a] = (int)b->groups[gi].ax[a].ntiles;
                total += b->groups[gi].ax[a].ntiles;
            }
    const long long chunk = std::max(1LL, total / (32LL * grid));
    std::vector<PersistItem> work;
    for (int a = 0; a < nd; ++a) {
        std::vector<int> order(ng);
        for (int gi = 0; gi < ng; ++gi) order[gi] = gi;
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            const long long wx = b->groups[x].ax[a].ntiles * b->groups[x].ax[a].threads;
            const long long wy = b->groups[y].ax[a].ntiles * b->groups[y].ax[a].threads;
            return wx != wy ? wx > wy : x < y;
        });
        for (int gi : order) {
            const Group &g = b->groups[gi];
            const long long nt = g.ax[a].ntiles;
            for (int i : g.members)
                for (long long t = 0; t < nt; t += chunk) {
                    PersistItem it;
                    it.shape = gi * nd + a;
                    it.inst = i;
                    it.axis = a;
                    it.tile0 = (int)t;
                    it.ntile = (int)std::min(chunk, nt - t);
                    it.pad = 0;
                    work.push_back(it);
                }
        }
    }
    cudaFree(b->d_pwork);
    cudaFree(b->d_pshapes);
    cudaFree(b->d_ptiles);
    b->d_pwork = nullptr;
    b->d_pshapes = nullptr;
    b->d_ptiles = nullptr;
    cudaError_t e = cudaMalloc(&b->d_pwork, sizeof(PersistItem) * work.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pshapes, sizeof(PassParams) * shapes.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ptiles, sizeof(int) * tiles.size());
    if (e == cudaSuccess && !b->d_pitems) e = cudaMalloc(&b->d_pitems, sizeof(BatchItem) * (size_t)count * nd);
    if (e == cudaSuccess && !b->d_pstate) {
        b->pstate_bytes = sizeof(unsigned long long) + sizeof(unsigned) * (size_t)count * nd;
        e = cudaMalloc(&b->d_pstate, b->pstate_bytes);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pwork, work.data(), sizeof(PersistItem) * work.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pshapes, shapes.data(), sizeof(PassParams) * shapes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_ptiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "persistent batch set-up");
    b->pnwork = (long long)work.size();
    b->pgrid = grid;
    b->pthreads = threads;
    b->psmem = smem;
    const char *env = getenv("HJLO_TEST_EXTRA_DEP");
    b->ptest_extra_dep = env ? std::max(0, atoi(env)) : 0;
    env = getenv("HJLO_TEST_WAIT_NS");
    b->pwait_ns = env ? std::max(0LL, atoll(env)) : 1000000000LL;
    b->pbuilt = true;
    return HJLO_OK;
}

// One time step of every instance in one persistent launch.
hjlo_status enqueue_persist_step(hjlo_batch *b, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b->d_pstate, 0, b->pstate_bytes, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(persistent state)");
    PersistParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.work = b->d_pwork;
    pp.nwork = b->pnwork;
    pp.shapes = b->d_pshapes;
    pp.items = b->d_pitems;
    pp.tiles = b->d_ptiles;
    pp.queue = b->d_pstate;
    pp.done = reinterpret_cast<unsigned *>(b->d_pstate + 1);
    pp.flags = b->d_flags;
    pp.count = b->count;
    pp.ndim = b->ndim;
    pp.wait_ns = b->pwait_ns;
    pp.test_extra_dep = b->ptest_extra_dep;
    return persist_launch(b->dtype, pp, b->pgrid, b->pthreads, b->psmem, st);
}

// One step of every instance: each group on its own stream, forked from and
// joined back into `st`.
hjlo_status enqueue_batch_step(hjlo_batch *b, cudaStream_t st, int nsteps_inner)
{
    cudaError_t e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord(fork)");
    for (auto &g : b->groups) {
        e = cudaStreamWaitEvent(g.stream, b->fork, 0);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent(fork)");
        for (int k = 0; k < nsteps_inner; ++k)
            for (int a = 0; a < b->ndim; ++a) {
                hjlo_status s = launch_pass_batch(g.ax[a], b->dtype, g.d_items[a], (long long)g.members.size(),
                                                  b->d_counters, b->d_flags, g.stream);
                if (s != HJLO_OK) return s;
            }
        e = cudaEventRecord(g.done, g.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g.done, 0);
        if (e != cudaSuccess) return cuda_error(e, "join");
    }
    return HJLO_OK;
}

hjlo_status capture(hjlo_batch *b, int inner, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
    hjlo_status s = HJLO_OK;
    if (b->persist) {
        for (int k = 0; k < inner && s == HJLO_OK; ++k) s = enqueue_persist_step(b, b->cap_stream);
    } else {
        s = enqueue_batch_step(b, b->cap_stream, inner);
    }
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (s != HJLO_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return cuda_error(e, "cudaGraphInstantiate"); }
    return HJLO_OK;
}

}  // namespace

extern "C" {

hjlo_status hjlo_batch_create(const hjlo_desc *descs, int32_t count, void *cuda_stream, hjlo_batch **out)
{
    if (!out) return set_error(HJLO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || count < 1) return set_error(HJLO_EINVAL, "need at least one descriptor");
    std::vector<long long> npts(count);
    for (int i = 0; i < count; ++i) {
        hjlo_status s = validate_desc(&descs[i], &npts[i]);
        if (s != HJLO_OK) return set_error(s, "instance %d: %s", i, last_error_cstr());
        if (descs[i].ndim != descs[0].ndim || descs[i].dtype != descs[0].dtype)
            return set_error(HJLO_EINVAL, "all instances must share ndim and dtype");
    }
    DeviceFacts df;
    hjlo_status s = device_facts(df);
    if (s != HJLO_OK) return s;
    if ((s = prepare_kernels()) != HJLO_OK) return s;

    hjlo_batch *b = new (std::nothrow) hjlo_batch();
    if (!b) return set_error(HJLO_ENOMEM, "host allocation");
    b->count = count;
    b->ndim = descs[0].ndim;
    b->dtype = descs[0].dtype;
    b->esize = (b->dtype == HJLO_F64) ? 8 : 4;
    b->device = df.device;
    b->stream = (cudaStream_t)cuda_stream;
    b->descs.assign(descs, descs + count);
    b->npts = npts;
    b->hv_off.resize(count);
    long long tot = 0;
    for (int i = 0; i < count; ++i) { b->hv_off[i] = tot; tot += npts[i]; }
    b->inst.resize((size_t)count * b->ndim);

    // per-instance tables; group key = shape, window size and algorithm per axis
    std::map<std::vector<long long>, int> key_to_group;
    for (int i = 0; i < count && s == HJLO_OK; ++i) {
        const hjlo_desc &d = descs[i];
        std::vector<long long> key;
        for (int a = 0; a < b->ndim && s == HJLO_OK; ++a) {
            AxisPlan &ax = b->inst[(size_t)i * b->ndim + a];
            long long inner = 1, outer = 1;
            for (int c = 0; c < a; ++c) outer *= d.shape[c];
            for (int c = a + 1; c < b->ndim; ++c) inner *= d.shape[c];
            ax.inner = inner;
            ax.outer = outer;
            double *k64 = nullptr;
            s = resolve_axis(d.shape[a], d.dx[a], d.h, d.P[a], d.window[a], ax, &k64);
            ax.t8_ok = 0;                     // the batched kernels keep 16-bit argmin offsets
            if (s != HJLO_OK) break;
            int algo = KALGO_MONGE;
            if (d.algo == HJLO_ALGO_BRUTE) algo = KALGO_BRUTE;
            if (d.algo == HJLO_ALGO_AUTO && (ax.weff < 8 || !(ax.curv > 0))) algo = KALGO_BRUTE;
            ax.algo = algo;
            cudaError_t e = cudaMalloc(&ax.d_kr64, sizeof(double) * ax.weff);
            if (e == cudaSuccess) e = cudaMemcpy(ax.d_kr64, k64, sizeof(double) * ax.weff, cudaMemcpyHostToDevice);
            free(k64);
            if (e != cudaSuccess) { s = cuda_error(e, "batch table upload"); break; }
            key.push_back(d.shape[a]);
            key.push_back(ax.weff);
            key.push_back(algo);
        }
        if (s != HJLO_OK) break;
        auto it = key_to_group.find(key);
        int gi;
        if (it == key_to_group.end()) {
            gi = (int)b->groups.size();
            key_to_group[key] = gi;
            b->groups.emplace_back();
        } else {
            gi = it->second;
        }
        b->groups[gi].members.push_back(i);
    }
    // launch shapes per group, sized for the group's instance count
    for (auto &g : b->groups) {
        if (s != HJLO_OK) break;
        const int rep = g.members[0];
        for (int a = 0; a < b->ndim && s == HJLO_OK; ++a) {
            AxisPlan ax = b->inst[(size_t)rep * b->ndim + a];
            s = shape_launch(ax, b->esize, ax.algo, df.num_sms, df.smem_optin, (long long)g.members.size(), nullptr,
                             false);
            if (s == HJLO_EUNSUPPORTED && ax.algo == KALGO_MONGE && b->descs[rep].algo == HJLO_ALGO_AUTO) {
                // lines too long for the monotone search's shared memory
                ax.algo = KALGO_BRUTE;
                s = shape_launch(ax, b->esize, ax.algo, df.num_sms, df.smem_optin, (long long)g.members.size(), nullptr,
                                 false);
            }
            if (s != HJLO_OK) break;
            apply_group_shape(b, g, a, ax);
            cudaError_t e = cudaMalloc(&g.d_items[a], sizeof(BatchItem) * g.members.size());
            if (e != cudaSuccess) { s = cuda_error(e, "cudaMalloc(batch items)"); break; }
            g.h_items[a].resize(g.members.size());
        }
        if (s == HJLO_OK) {
            cudaError_t e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
            if (e != cudaSuccess) s = cuda_error(e, "group stream");
        }
    }
    if (s == HJLO_OK) {
        cudaError_t e = cudaMalloc(&b->d_counters, sizeof(unsigned long long) * CNT_N);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_flags, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(unsigned long long) * CNT_N);
        if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_hv, sizeof(double) * std::max(1LL, tot));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e != cudaSuccess) s = cuda_error(e, "batch allocation");
    }
    if (s != HJLO_OK) {
        release(b);
        delete b;
        return s;
    }
    *out = b;
    return HJLO_OK;
}

hjlo_status hjlo_batch_destroy(hjlo_batch *b)
{
    if (!b) return HJLO_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    return HJLO_OK;
}

hjlo_status hjlo_batch_run(hjlo_batch *b, void *const *u, const double *const *V, int64_t nsteps)
{
    if (!b) return set_error(HJLO_EINVAL, "batch is NULL");
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 0) return set_error(HJLO_EINVAL, "nsteps must be >= 0");
    for (int i = 0; i < b->count; ++i)
        if (!u[i]) return set_error(HJLO_EINVAL, "u[%d] is NULL", i);
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    // h*V of every instance, then the per-instance fields of every launch
    for (int i = 0; i < b->count; ++i) {
        if (!V || !V[i]) continue;
        long long n = b->npts[i];
        long long blocks = std::min<long long>((n + 255) / 256, 2048);
        batch_scale_kernel<<<(unsigned)blocks, 256, 0, b->stream>>>(V[i], b->descs[i].h, b->d_hv + b->hv_off[i], n);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "h*V kernels");
    for (auto &g : b->groups) {
        for (int a = 0; a < b->ndim; ++a) {
            const bool last = (a == b->ndim - 1);
            for (size_t m = 0; m < g.members.size(); ++m) {
                const int i = g.members[m];
                const AxisPlan &ax = b->inst[(size_t)i * b->ndim + a];
                BatchItem &it = g.h_items[a][m];
                memset(&it, 0, sizeof(it));
                it.src = u[i];
                it.dst = u[i];
                it.hv = (last && V && V[i]) ? b->d_hv + b->hv_off[i] : nullptr;
                it.kr64 = ax.d_kr64;
                it.kmax = ax.kmax;
                it.curv = ax.curv;
                it.hoff = ax.hoff;
                it.dhi = (int)ax.dhi;
                if (ax.layout == LAYOUT_CONTIG)
                    it.use_tma = (((uintptr_t)u[i] & 15) == 0) && (((ax.N * b->esize) & 15) == 0);
                else
                    it.use_tma = encode_strided(ax, b->esize, u[i], &it.tmap) ? 1 : 0;
            }
            // pageable source: the call returns once the host array is consumed
            e = cudaMemcpyAsync(g.d_items[a], g.h_items[a].data(), sizeof(BatchItem) * g.members.size(),
                                cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(batch items)");
        }
    }
    hjlo_status s = HJLO_OK;
    if (b->persist) {
        if (!b->pbuilt) {
            drop_graphs(b);
            if ((s = build_persist(b)) != HJLO_OK) return s;
        }
        // the same per-instance fields, indexed by (axis, instance)
        b->h_pitems.resize((size_t)b->count * b->ndim);
        for (auto &g : b->groups)
            for (int a = 0; a < b->ndim; ++a)
                for (size_t m = 0; m < g.members.size(); ++m)
                    b->h_pitems[(size_t)a * b->count + g.members[m]] = g.h_items[a][m];
        e = cudaMemcpyAsync(b->d_pitems, b->h_pitems.data(), sizeof(BatchItem) * b->h_pitems.size(),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(persistent items)");
    }
    if (!b->graph_many) s = capture(b, kBatchGraphSteps, &b->graph_many);
    if (s == HJLO_OK && !b->graph_one) s = capture(b, 1, &b->graph_one);
    if (s != HJLO_OK) return s;
    long long n = 0;
    for (; n + kBatchGraphSteps <= nsteps; n += kBatchGraphSteps) {
        e = cudaGraphLaunch(b->graph_many, b->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
    }
    for (; n < nsteps; ++n) {
        e = cudaGraphLaunch(b->graph_one, b->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
    }
    b->steps += nsteps;
    return HJLO_OK;
}

hjlo_status hjlo_batch_set_persistent(hjlo_batch *b, int32_t on)
{
    if (!b) return set_error(HJLO_EINVAL, "batch is NULL");
    if (on != 0 && on != 1) return set_error(HJLO_EINVAL, "on must be 0 or 1");
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    if (on)
        for (auto &g : b->groups)
            for (int a = 0; a < b->ndim; ++a)
                if (g.ax[a].algo != KALGO_MONGE)
                    return set_error(HJLO_EUNSUPPORTED, "the persistent batch runs the monotone search only");
    if (on != b->persist) {
        drop_graphs(b);
        b->persist = on;
    }
    return HJLO_OK;
}

hjlo_status hjlo_batch_autotune(hjlo_batch *b, const void *const *u, const double *const *V, int64_t nsteps,
                                hjlo_tune_report *report)
{
    if (!b) return set_error(HJLO_EINVAL, "batch is NULL");
    if (!u) return set_error(HJLO_EINVAL, "u is NULL");
    if (nsteps < 1) return set_error(HJLO_EINVAL, "nsteps must be >= 1");
    for (int i = 0; i < b->count; ++i)
        if (!u[i]) return set_error(HJLO_EINVAL, "u[%d] is NULL", i);
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    DeviceFacts df;
    hjlo_status s = device_facts(df);
    if (s != HJLO_OK) return s;
    // trial launches do not count: the device counters are put back afterwards
    unsigned long long saved[CNT_N];
    e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(saved, b->d_counters, sizeof(saved), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "autotune counter save");
    // device copies of every instance, refreshed before each trial
    long long tot = 0;
    std::vector<long long> off(b->count);
    for (int i = 0; i < b->count; ++i) {
        off[i] = tot;
        tot += (b->npts[i] * b->esize + 255) & ~255LL;
    }
    char *scratch = nullptr;
    e = cudaMalloc(&scratch, (size_t)std::max(1LL, tot));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(autotune scratch)");
    std::vector<void *> su(b->count);
    for (int i = 0; i < b->count; ++i) su[i] = scratch + off[i];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) s = cuda_error(e, "cudaEventCreate");
    auto refresh = [&]() -> hjlo_status {
        for (int i = 0; i < b->count; ++i) {
            cudaError_t ce = cudaMemcpyAsync(su[i], u[i], (size_t)(b->npts[i] * b->esize), cudaMemcpyDeviceToDevice,
                                             b->stream);
            if (ce != cudaSuccess) return cuda_error(ce, "autotune copy");
        }
        return HJLO_OK;
    };
    // one untimed step (rebuilds the graphs of a new shape), then the best of
    // two timed runs of nsteps
    auto trial = [&](float *ms) -> hjlo_status {
        hjlo_status ts = refresh();
        if (ts == HJLO_OK) ts = hjlo_batch_run(b, su.data(), V, 1);
        float best = 1e30f;
        for (int r = 0; r < 2 && ts == HJLO_OK; ++r) {
            if ((ts = refresh()) != HJLO_OK) break;
            cudaError_t ce = cudaEventRecord(e0, b->stream);
            if (ce != cudaSuccess) return cuda_error(ce, "autotune timing");
            if ((ts = hjlo_batch_run(b, su.data(), V, nsteps)) != HJLO_OK) break;
            ce = cudaEventRecord(e1, b->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) return cuda_error(ce, "autotune timing");
            best = std::min(best, t);
        }
        *ms = best;
        return ts;
    };
    hjlo_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    const long long steps0 = b->steps;      // trials do not count as steps of the batch
    float ms0 = 0.0f;
    if (s == HJLO_OK) s = trial(&ms0);
    float cur = ms0;
    // groups by decreasing work, axis by axis
    std::vector<size_t> order(b->groups.size());
    std::vector<long long> work(b->groups.size(), 0);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        order[gi] = gi;
        for (int i : b->groups[gi].members) work[gi] += b->npts[i];
    }
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work[x] > work[y]; });
    for (size_t gi : order) {
        Group &g = b->groups[gi];
        for (int a = 0; a < b->ndim && s == HJLO_OK; ++a) {
            if (g.ax[a].algo != KALGO_MONGE) continue;
            AxisPlan best = g.ax[a];
            const AxisPlan start = g.ax[a];
            for (const ShapeHints &h : tune_candidates(start)) {
                AxisPlan t = start;
                if (shape_launch(t, b->esize, KALGO_MONGE, df.num_sms, df.smem_optin, (long long)g.members.size(),
                                 &h, false) != HJLO_OK)
                    continue;
                if (t.lpl == best.lpl && t.C == best.C && t.wide_mul == best.wide_mul && t.wide_add == best.wide_add)
                    continue;
                apply_group_shape(b, g, a, t);
                drop_graphs(b);
                float ms = 0.0f;
                s = trial(&ms);
                if (s != HJLO_OK) break;
                ++rep.trials;
                if (ms < 0.98f * cur) {
                    cur = ms;
                    best = t;
                }
            }
            apply_group_shape(b, g, a, best);
            drop_graphs(b);
        }
        if (s != HJLO_OK) break;
    }
    float ms1 = cur;
    if (s == HJLO_OK) s = trial(&ms1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    e = cudaStreamSynchronize(b->stream);
    cudaFree(scratch);
    b->steps = steps0;
    if (e == cudaSuccess) e = cudaMemcpy(b->d_counters, saved, sizeof(saved), cudaMemcpyHostToDevice);
    if (s == HJLO_OK && e != cudaSuccess) s = cuda_error(e, "autotune counter restore");
    if (s != HJLO_OK) return s;
    if (!order.empty()) {
        const Group &g = b->groups[order[0]];
        for (int a = 0; a < b->ndim; ++a) {
            if (g.ax[a].algo != KALGO_MONGE) continue;
            rep.lanes_per_line[a] = g.ax[a].lpl;
            rep.lines_per_tile[a] = g.ax[a].C;
            rep.offload[a] = (g.ax[a].wide_add < (1 << 20)) ? 1 : 0;
        }
    }
    rep.ms_initial = ms0;
    rep.ms_tuned = ms1;
    if (report) *report = rep;
    return HJLO_OK;
}

hjlo_status hjlo_batch_hbar(hjlo_batch *b, const void *const *u0, const void *const *un, int64_t nsteps,
                            double *out3)
{
    if (!b) return set_error(HJLO_EINVAL, "batch is NULL");
    if (!u0 || !un || !out3) return set_error(HJLO_EINVAL, "NULL argument");
    if (nsteps < 1) return set_error(HJLO_EINVAL, "nsteps must be >= 1");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    const long long cnt = b->count;
    std::vector<DiffArgs> args(cnt);
    for (long long i = 0; i < cnt; ++i) {
        if (!u0[i] || !un[i]) return set_error(HJLO_EINVAL, "u0/un[%lld] is NULL", i);
        args[i] = {u0[i], un[i], b->npts[i]};
    }
    if (!b->d_part) {
        e = cudaMalloc(&b->d_part, sizeof(double) * 3 * cnt * (kRedBlocks + 1) + sizeof(DiffArgs) * cnt);
        if (e != cudaSuccess) { b->d_part = nullptr; return cuda_error(e, "cudaMalloc(batch readout)"); }
    }
    double *part = b->d_part;
    double *res = part + 3 * cnt * kRedBlocks;
    DiffArgs *d_args = reinterpret_cast<DiffArgs *>(res + 3 * cnt);
    e = cudaMemcpyAsync(d_args, args.data(), sizeof(DiffArgs) * cnt, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(readout args)");
    dim3 grid(kRedBlocks, (unsigned)cnt);
    if (b->dtype == HJLO_F64)
        batch_diff_partials<double><<<grid, kRedThreads, 0, b->stream>>>(d_args, part);
    else
        batch_diff_partials<float><<<grid, kRedThreads, 0, b->stream>>>(d_args, part);
    batch_fold<<<(unsigned)((cnt + 127) / 128), 128, 0, b->stream>>>(part, kRedBlocks, cnt, res);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "readout kernels");
    std::vector<double> r(3 * cnt);
    e = cudaMemcpyAsync(r.data(), res, sizeof(double) * 3 * cnt, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_error(e, "readout copy");
    for (long long i = 0; i < cnt; ++i) {
        const double T = (double)nsteps * b->descs[i].h;
        out3[3 * i + 0] = -(r[3 * i] / (double)b->npts[i]) / T;
        out3[3 * i + 1] = -r[3 * i + 2] / T;
        out3[3 * i + 2] = -r[3 * i + 1] / T;
    }
    return HJLO_OK;
}

hjlo_status hjlo_batch_sync(hjlo_batch *b, hjlo_counters *out)
{
    if (!b) return set_error(HJLO_EINVAL, "batch is NULL");
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    unsigned long long c[CNT_N];
    int flags = 0;
    e = cudaMemcpy(c, b->d_counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "counter copy");
    if (out) {
        memset(out, 0, sizeof(*out));
        out->exact_rescans = (int64_t)c[CNT_RESCAN];
        out->brute_fallback_lines = (int64_t)c[CNT_FALLBACK];
        out->window_edge_hits = (int64_t)c[CNT_EDGE];
        out->steps = b->steps;
        out->error_flags = flags;
    }
    if (flags) {
        cudaMemset(b->d_flags, 0, sizeof(int));
        if (flags & FLAG_TIMEOUT) return set_error(HJLO_ETIMEOUT, "a bounded device wait gave up");
        return set_error(HJLO_EPRECOND, "a device precondition failed");
    }
    return HJLO_OK;
}

int32_t hjlo_batch_groups(const hjlo_batch *b) { return b ? (int32_t)b->groups.size() : 0; }

}  // extern "C"
