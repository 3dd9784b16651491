// hjlo_pass.cu -- kernel tables, launch shaping and launch of the axis pass.
//
// Kernel table (Sec. 2.3 eq. cost2 with the mechanical Lagrangian of Sec. 2.1,
// one axis at a time per Remark rk28): k[d] = h * L(d dx / h),
// L(v) = v^2/2 - P v, evaluated as
//     v = (d*dx)/h; t1 = 0.5*v; t1 = t1*v; t2 = P*v; L = t1 - t2; k = h*L
// in binary64 round-to-nearest with no contraction (this file is compiled
// with -ffp-contract=off).  Window (Sec. 3.3 eq. los; Sec. 4.2, kernel
// restricted to a support centred on its minimum): c = largest minimiser of
// k; [c-W, c+W] when W > 0 and 2W+1 < N, else the N displacements that
// realise the lift-minimised torus cost (equal costs keep the larger d).
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "hjlo_internal.h"

namespace hjlo {

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

hjlo_status set_error(hjlo_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

hjlo_status cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return set_error(HJLO_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(HJLO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char *last_error_cstr() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

// ------------------------------------------------------------------ tables

double kernel_entry(long long d, double dx, double h, double P)
{
    double v = ((double)d * dx) / h;
    double t1 = 0.5 * v;
    t1 = t1 * v;
    double t2 = P * v;
    double L = t1 - t2;
    return h * L;
}

hjlo_status resolve_window(long long N, double dx, double h, double P, long long W, AxisWindow &win)
{
    double ds = P * h / dx;
    if (!(std::fabs(ds) < 1.0e9)) return set_error(HJLO_EUNSUPPORTED, "kernel minimiser P*h/dx out of range");
    long long base = (long long)std::floor(ds);
    long long c = base - 5;
    double kc = kernel_entry(c, dx, h, P);
    for (long long d = base - 4; d <= base + 6; ++d) {
        double kd = kernel_entry(d, dx, h, P);
        if (kd <= kc) { kc = kd; c = d; }
    }
    long long lo, hi;
    if (W > 0 && 2 * W + 1 < N) {
        lo = c - W;
        hi = c + W;
    } else {
        lo = hi = c;
        while (hi - lo + 1 < N) {
            if (kernel_entry(lo - 1, dx, h, P) < kernel_entry(hi + 1, dx, h, P)) --lo; else ++hi;
        }
    }
    const long long weff = hi - lo + 1;
    if (weff > 65535) return set_error(HJLO_EUNSUPPORTED, "window of %lld displacements exceeds 65535", weff);
    if (lo < -(1LL << 30) || hi > (1LL << 30)) return set_error(HJLO_EUNSUPPORTED, "displacements out of int32 range");
    win.lo = lo;
    win.hi = hi;
    win.centre = c;
    win.kmin = kc;
    win.weff = weff;
    return HJLO_OK;
}

void fill_axis_table(long long N, double dx, double h, double P, const AxisWindow &win, AxisPlan &ax, double *k64)
{
    const long long lo = win.lo, hi = win.hi, weff = win.weff;
    double kmax = 0.0;
    for (long long t = 0; t < weff; ++t) {
        double k = kernel_entry(hi - t, dx, h, P);
        k64[t] = k;
        kmax = std::max(kmax, std::fabs(k));
    }
    // lower bound of the smallest second difference of the table (as exact
    // values); each of the three roundings is below 2^-53 of its result
    double curv = INFINITY;
    for (long long t = 1; t + 1 < weff; ++t) {
        double a = k64[t - 1] - k64[t];      // k[d+1] - k[d] with d = hi - t
        double b = k64[t] - k64[t + 1];      // k[d] - k[d-1]
        double s = a - b;
        double err = 0x1p-52 * (std::fabs(a) + std::fabs(b) + std::fabs(s));
        curv = std::min(curv, s - err);
    }
    ax.N = N;
    ax.dlo = lo;
    ax.dhi = hi;
    ax.centre = win.centre;
    ax.weff = (int)weff;
    long long ho = (-hi) % N;
    if (ho < 0) ho += N;
    ax.hoff = (int)ho;
    ax.kmin = win.kmin;
    ax.kmax = kmax;
    ax.curv = curv;
}

hjlo_status resolve_axis(long long N, double dx, double h, double P, long long W, AxisPlan &ax,
                         double **kr64_host)
{
    *kr64_host = nullptr;
    AxisWindow win;
    hjlo_status s = resolve_window(N, dx, h, P, W, win);
    if (s != HJLO_OK) return s;
    double *k64 = (double *)malloc(sizeof(double) * win.weff);
    if (!k64) return set_error(HJLO_ENOMEM, "host table allocation");
    fill_axis_table(N, dx, h, P, win, ax, k64);
    *kr64_host = k64;
    return HJLO_OK;
}

// ------------------------------------------------------------------ launch shape

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static void layout_smem(AxisPlan &ax, int esize, int algo)
{
    const int C = ax.C;
    const long long rows = (ax.layout == LAYOUT_STRIDED) ? (long long)ax.nbox * ax.by : ax.N;
    const bool monge = (algo == KALGO_MONGE);
    size_t off = 0;
    ax.off_u = 0;
    off = align_up((size_t)C * rows * esize, 128);
    ax.off_fx = (int)off;
    if (monge) off = align_up(off + (size_t)C * ax.lp * 4, 16);
    ax.off_kfx = (int)off;
    if (monge) off = align_up(off + (size_t)C * ax.weff * 4, 16);
    ax.off_t = (int)off;
    off = align_up(off + (size_t)C * ax.tp * (ax.t8 ? 1 : 2), 16);
    ax.off_k64 = (int)off;
    off = align_up(off + (size_t)ax.weff * 8, 16);
    ax.off_misc = (int)off;
    off = align_up(off + 16 + 40 * (size_t)C, 16);   // mbarrier, counters, per-line screen facts
    ax.smem = off;
}

static int odd_at_least(long long x)
{
    long long v = x < 1 ? 1 : x;
    return (int)((v & 1) ? v : v + 1);
}

static int ilog2(int x)
{
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

// Halo pitch: at least N + weff - 1 words; when several lines share a warp
// (lpl < 32) the pitch is congruent to lpl*seg mod 32, so that lane g of line
// l reads bank S*(lpl*l + g) mod 32 -- distinct across the warp.
static int halo_pitch(const AxisPlan &ax)
{
    long long L = ax.N + ax.weff - 1;
    if (ax.lpl >= 32) return (int)align_up((size_t)L, 4);
    long long want = ((long long)ax.lpl * ax.seg) % 32;
    while (L % 32 != want) ++L;
    return (int)L;
}

// Pivot group size: GS lanes share one whole-window scan (weff/GS candidates
// each) and the other GS-1 first rows are bracketed by group pivots (about
// GS*S candidates).  Returns the group size and its cost in candidates per lane.
static int pivot_group(int weff, int S, int lpl, double *cost)
{
    int best = 1;
    double bc = (double)weff;
    for (int gs = 2; gs <= 32 && gs <= lpl; gs *= 2) {
        double c = std::ceil((double)weff / gs) + (double)gs * S + 4.0 * std::log2((double)gs);
        if (c < bc) { bc = c; best = gs; }
    }
    if (cost) *cost = bc;
    return best;
}

ShapeHints env_hints()
{
    ShapeHints h;
    if (const char *e = getenv("HJLO_LANES_PER_LINE")) h.lpl = atoi(e);
    if (const char *e = getenv("HJLO_LINES_PER_TILE")) h.C = atoi(e);
    if (const char *e = getenv("HJLO_BLOCK_ROWS")) h.block_rows = atoll(e);
    if (const char *e = getenv("HJLO_OFFLOAD")) {
        int m = 0, a = 0;
        if (sscanf(e, "%d,%d", &m, &a) == 2 && m >= 0 && a >= 0) {
            h.wide_mul = m;
            h.wide_add = a;
        } else {
            h.wide_mul = 0;
            h.wide_add = 1 << 24;
        }
    }
    return h;
}

std::vector<ShapeHints> tune_candidates(const AxisPlan &ax)
{
    std::vector<ShapeHints> out;
    const int lpls[3] = {ax.lpl / 2, ax.lpl, ax.lpl * 2};
    const int Cs[3] = {ax.C / 2, ax.C, ax.C * 2};
    // row-block axes: rows per block halved / kept / doubled as well
    const long long vRs[3] = {ax.vR / 2, (long long)ax.vR, 2LL * ax.vR};
    const int nb = (ax.vblocks > 1) ? 3 : 1;
    const long long line = (ax.vblocks > 1) ? ax.vNp : ax.N;
    for (int bi = 0; bi < nb; ++bi) {
        const long long br = (nb == 3) ? vRs[bi] : 0;
        if (nb == 3 && br < 1) continue;
        for (int li = 0; li < 3; ++li) {
            if (lpls[li] < 1 || lpls[li] > 1024 || lpls[li] > line) continue;
            for (int ci = 0; ci < 3; ++ci) {
                if (Cs[ci] < 1) continue;
                for (int off = 0; off < 2; ++off) {
                    ShapeHints h;
                    h.lpl = lpls[li];
                    h.C = Cs[ci];
                    h.wide_mul = off ? 0 : 2;
                    h.wide_add = off ? (1 << 24) : 8;
                    h.block_rows = br;
                    out.push_back(h);
                }
            }
        }
    }
    return out;
}

static hjlo_status shape_lines(AxisPlan &ax, int esize, int algo, int num_sms, size_t smem_optin,
                               long long replicas, const ShapeHints *hints);

// Rows per block for a contiguous axis, or 0 to launch whole lines.  Blocks
// are used when the window is at most a quarter of the line and either a
// whole line does not fit in one CTA's shared memory or the axis has fewer
// lines than half the SMs; they hold about one SM's share of the rows, at
// least 2 (weff - 1) (a block stages vR + weff - 1 points for vR rows) and
// at most what fits.  Brute force, whose rows cost weff candidates each
// against one staged point, also takes blocks for wider windows (up to the
// full torus window) on an axis with few lines, from one row per block: a
// lone line then spreads over many SMs instead of one SM's binary64 pipe.
// A hint (hinted > 0) replaces the share, within [weff - 1 (brute: 1), what
// fits].
static long long block_rows(const AxisPlan &ax, int esize, int algo, int num_sms, size_t smem_optin,
                            long long hinted)
{
    const long long N = ax.N, w = ax.weff, lines = ax.outer;
    const bool brute = (algo == KALGO_BRUTE);
    if (ax.inner != 1 || (4 * w > N && !brute)) return 0;
    // shared memory per staged point and per window entry (layout_smem)
    const long long per_pt = esize + 2 + ((algo == KALGO_MONGE) ? 4 : 0);
    const long long per_w = 8 + ((algo == KALGO_MONGE) ? 8 : 0);
    const long long room = (long long)smem_optin - 1024 - per_w * w;
    const long long fit_pts = room > 0 ? room / per_pt : 0;         // staged points that fit
    const bool fits = N + w <= fit_pts;
    if (fits && 2 * lines >= num_sms) return 0;
    if (brute && 4 * w > N && !(2 * lines < num_sms)) return 0;     // wide windows: few lines only
    const long long least = brute ? 1 : std::max(1LL, w - 1);
    long long vR = std::max(brute ? 1 : 2 * (w - 1), (N * lines + num_sms - 1) / num_sms);
    if (hinted > 0) vR = std::max(hinted, least);
    vR = std::min(vR, fit_pts - (w - 1));
    vR = std::min(vR, N - (w - 1));                                 // a block never spans the line
    if (vR < least || vR >= N) return 0;
    return vR;
}

hjlo_status shape_launch(AxisPlan &ax, int esize, int algo, int num_sms, size_t smem_optin, long long replicas,
                         const ShapeHints *hints, bool row_blocks)
{
    ax.vblocks = 1;
    ax.vR = 0;
    ax.vNp = 0;
    ax.rows = 0;
    if ((algo == KALGO_MONGE || algo == KALGO_BRUTE) && row_blocks) {
        const ShapeHints hint = hints ? *hints : env_hints();
        const long long vR = block_rows(ax, esize, algo, num_sms, smem_optin, hint.block_rows);
        if (vR > 0) {
            AxisPlan v = ax;
            v.N = vR + ax.weff - 1;
            v.vblocks = (ax.N + vR - 1) / vR;
            v.outer = ax.outer * v.vblocks;
            v.hoff = 0;
            v.rows = vR;                      // only the block's own rows are searched
            hjlo_status s = shape_lines(v, esize, algo, num_sms, smem_optin, 1, hints);
            if (s != HJLO_OK) return s;
            // launch fields from the block lines; geometry and tables stay the axis's
            AxisPlan r = v;
            r.N = ax.N;
            r.outer = ax.outer;
            r.hoff = ax.hoff;
            r.vR = (int)vR;
            r.vNp = v.N;
            r.rows = 0;
            ax = r;
            return HJLO_OK;
        }
    }
    return shape_lines(ax, esize, algo, num_sms, smem_optin, replicas, hints);
}

static hjlo_status shape_lines(AxisPlan &ax, int esize, int algo, int num_sms, size_t smem_optin,
                               long long replicas, const ShapeHints *hints)
{
    const ShapeHints hint = hints ? *hints : env_hints();
    ax.algo = algo;
    ax.layout = (ax.inner == 1) ? LAYOUT_CONTIG : LAYOUT_STRIDED;
    const long long N = ax.N;
    const long long nlines = ax.inner * ax.outer * std::max(1LL, replicas);
    // argmin offsets: bytes for the monotone search's single-grid launches
    // with windows of at most 256 displacements (measured on the 256^3 grid:
    // 7 CTAs per SM instead of 6, 4.7 % less time per pass), else 16-bit;
    // the row pitch puts consecutive lines' rows in different banks
    ax.t8 = (algo == KALGO_MONGE && ax.t8_ok && ax.weff <= 256) ? 1 : 0;
    ax.tp = (int)N;
    if (ax.t8)
        while (ax.tp % 8 != 4) ++ax.tp;
    else
        while (ax.tp % 4 != 2) ++ax.tp;
    if (ax.layout == LAYOUT_STRIDED) {
        ax.nbox = (int)((N + 255) / 256);
        long long per = (N + ax.nbox - 1) / ax.nbox;
        ax.by = (int)align_up((size_t)per, 16);
        if (ax.by > 256) ax.by = 256;
    } else {
        ax.nbox = 1;
        ax.by = (int)N;
    }
    int cmin = 1, cmax = 32;
    if (ax.layout == LAYOUT_STRIDED) {
        cmin = (esize == 8) ? 2 : 4;
        long long p2 = 1;
        while (p2 < ax.inner && p2 < 32) p2 *= 2;
        cmax = (int)std::max<long long>(p2, cmin);
    }

    // rows searched per line (a row block searches only its own rows)
    const long long NR = (ax.rows > 0 && ax.rows < N) ? ax.rows : N;
    if (algo == KALGO_MONGE) {
        // lanes per line: maximise (occupancy efficiency) / (work per row), with
        // work per row ~ weff/S + log2(S) + 3 (pivot share, divide and conquer,
        // staging and write-back) and occupancy bounded by shared memory per
        // line; a hint (the autotuner, or the environment) overrides it.
        int best_lpl = 1;
        double best_score = -1.0;
        for (int lpl = 1; lpl <= 1024; lpl *= 2) {
            int S = odd_at_least((NR + lpl - 1) / lpl);
            AxisPlan t = ax;
            t.lpl = lpl;
            t.seg = S;
            t.C = 1;
            t.lp = halo_pitch(t);
            layout_smem(t, esize, algo);
            double lines_sm = std::min((double)nlines / num_sms, 227.0 * 1024 / (double)t.smem);
            double warps = std::min(64.0, lines_sm * lpl / 32.0);
            double eff = std::min(1.0, warps / 24.0);
            double pcost = 0.0;
            pivot_group(ax.weff, S, lpl, &pcost);
            double work = pcost / S + std::log2((double)S) + 3.0;
            double score = eff / work;
            if (hint.lpl == lpl && lpl <= N) { best_lpl = lpl; break; }
            if (S >= 3 && score > best_score * 1.0001) { best_score = score; best_lpl = lpl; }
        }
        // staging and write-back assume every lane of a line owns at most one
        // point per sweep of lpl, i.e. lpl <= N
        if (best_lpl > N) best_lpl = 1;
        ax.lpl = best_lpl;
        ax.log2lpl = ilog2(best_lpl);
        ax.seg = odd_at_least((NR + best_lpl - 1) / best_lpl);
        ax.gs = pivot_group(ax.weff, ax.seg, ax.lpl, nullptr);
        // offload rule of wide brackets: 2 x expected span + 8 unless hinted
        ax.wide_mul = 2;
        ax.wide_add = 8;
        if (hint.wide_mul >= 0 && hint.wide_add >= 0) {
            ax.wide_mul = hint.wide_mul;
            ax.wide_add = hint.wide_add;
        }
        ax.lp = halo_pitch(ax);
        ax.wpl = 1;
    } else {
        // brute force: warps per line (rows interleaved) until the grid has
        // about 48 warps per SM, at least 4 rows per warp
        ax.wpl = 1;
        while (ax.wpl < 16 && nlines * ax.wpl < 48LL * num_sms && 2LL * ax.wpl * 4 <= NR &&
               32LL * 2 * ax.wpl * cmin <= 512)
            ax.wpl *= 2;
        ax.lpl = 32 * ax.wpl;
        ax.log2lpl = ilog2(ax.lpl);
        ax.seg = 1;
        ax.gs = 1;
        ax.lp = 0;
    }
    const int lanes = (algo == KALGO_MONGE) ? ax.lpl : 32 * ax.wpl;
    // lines per CTA: at least one warp of threads, TMA-friendly for strided
    // lines, then grown while tiles stay >= 2 per SM and the shared memory
    // fits twice per SM, up to 128 threads for the monotone search (small
    // tiles balance the SMs best; measured on the 1024^2 and 256^3 grids)
    // and 512 for brute force
    int C = std::max(cmin, std::max(1, 32 / lanes));
    while (C < cmin) C *= 2;
    auto tiles_for = [&](int c) -> long long {
        if (ax.layout == LAYOUT_CONTIG) return (ax.outer + c - 1) / c;
        return ax.outer * ((ax.inner + c - 1) / c);
    };
    ax.C = C;
    layout_smem(ax, esize, algo);
    if (ax.smem > smem_optin || (long long)C * lanes > 1024)
        return set_error(HJLO_EUNSUPPORTED, "a line of %lld points does not fit in shared memory", N);
    const size_t budget = std::min<size_t>(110 * 1024, smem_optin);
    const long long cap = (algo == KALGO_MONGE) ? 128 : 512;
    while (2 * C <= std::max(cmax, C) && (long long)2 * C * lanes <= cap &&
           tiles_for(2 * C) * std::max(1LL, replicas) >= 2LL * num_sms) {
        AxisPlan t = ax;
        t.C = 2 * C;
        layout_smem(t, esize, algo);
        if (t.smem > budget) break;
        C *= 2;
    }
    // hinted lines per tile (a power of two that fits)
    if (hint.C > 0) {
        const int want = hint.C;
        if (want >= cmin && (want & (want - 1)) == 0 && (long long)want * lanes <= 1024) {
            AxisPlan t = ax;
            t.C = want;
            layout_smem(t, esize, algo);
            if (t.smem <= smem_optin) C = want;
        }
    }
    ax.C = C;
    ax.log2C = ilog2(C);
    layout_smem(ax, esize, algo);
    ax.threads = C * lanes;
    ax.tiles_per_outer = (ax.layout == LAYOUT_STRIDED) ? (ax.inner + C - 1) / C : 1;
    ax.ntiles = tiles_for(C);
    return HJLO_OK;
}

// ------------------------------------------------------------------ TMA descriptors

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 3D view {inner, N, outer} of the grid for lines along a strided axis; box
// {C, by, 1}.  Returns false if TMA cannot be used for this pointer.
bool encode_strided(const AxisPlan &ax, int esize, const void *ptr, CUtensorMap *map)
{
    if (((uintptr_t)ptr & 15) || ((ax.inner * esize) & 15) || ((ax.C * esize) & 15)) return false;
    if (ax.inner > (1LL << 32) || ax.N > (1LL << 32) || ax.outer > (1LL << 32)) return false;
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)ax.inner, (cuuint64_t)ax.N, (cuuint64_t)ax.outer};
    cuuint64_t strides[2] = {(cuuint64_t)(ax.inner * esize), (cuuint64_t)(ax.inner * ax.N * esize)};
    cuuint32_t box[3] = {(cuuint32_t)ax.C, (cuuint32_t)ax.by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ launch

// Per-device one-time set-up done outside any stream capture: shared-memory
// opt-in of every pass kernel and the driver entry point for TMA descriptors.
hjlo_status prepare_kernels()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> g(mu);
    if (dev < 64 && done[dev]) return HJLO_OK;
    hjlo_status s;
    if ((s = kern_allow_smem_f64_contig()) != HJLO_OK) return s;
    if ((s = kern_allow_smem_f64_strided()) != HJLO_OK) return s;
    if ((s = kern_allow_smem_f32_contig()) != HJLO_OK) return s;
    if ((s = kern_allow_smem_f32_strided()) != HJLO_OK) return s;
    if ((s = decomp_allow_smem()) != HJLO_OK) return s;
    if ((s = split_allow_smem()) != HJLO_OK) return s;
    if ((s = persist_allow_smem_f64()) != HJLO_OK) return s;
    if ((s = persist_allow_smem_f32()) != HJLO_OK) return s;
    encode_fn();
    if (dev < 64) done[dev] = true;
    return HJLO_OK;
}

static hjlo_status dispatch_single(const AxisPlan &ax, int dtype, const CUtensorMap &map, const PassParams &p,
                                   cudaStream_t st)
{
    const bool strided = (ax.layout == LAYOUT_STRIDED);
    if (dtype == HJLO_F64)
        return strided ? kern_single_f64_strided(ax, map, p, st) : kern_single_f64_contig(ax, map, p, st);
    return strided ? kern_single_f32_strided(ax, map, p, st) : kern_single_f32_contig(ax, map, p, st);
}

static hjlo_status dispatch_batch(const AxisPlan &ax, int dtype, const BatchItem *items, const PassParams &p,
                                  long long count, cudaStream_t st)
{
    const bool strided = (ax.layout == LAYOUT_STRIDED);
    if (dtype == HJLO_F64)
        return strided ? kern_batch_f64_strided(ax, items, p, count, st)
                       : kern_batch_f64_contig(ax, items, p, count, st);
    return strided ? kern_batch_f32_strided(ax, items, p, count, st) : kern_batch_f32_contig(ax, items, p, count, st);
}

void fill_params(const AxisPlan &ax, PassParams &p)
{
    memset(&p, 0, sizeof(p));
    p.kr64 = ax.d_kr64;
    p.N = ax.N;
    p.inner = ax.inner;
    p.outer = ax.outer;
    p.ntiles = ax.ntiles;
    p.tiles_per_outer = ax.tiles_per_outer;
    p.hoff = ax.hoff;
    p.dhi = (int)ax.dhi;
    p.weff = ax.weff;
    p.C = ax.C;
    p.log2C = ax.log2C;
    p.wpl = ax.wpl;
    p.lpl = ax.lpl;
    p.log2lpl = ax.log2lpl;
    p.seg = ax.seg;
    p.gs = ax.gs;
    p.tp = ax.tp;
    p.by = ax.by;
    p.nbox = ax.nbox;
    p.lp = ax.lp;
    p.kmax = ax.kmax;
    p.curv = ax.curv;
    p.off_u = ax.off_u;
    p.off_fx = ax.off_fx;
    p.off_kfx = ax.off_kfx;
    p.off_t = ax.off_t;
    p.off_k64 = ax.off_k64;
    p.off_misc = ax.off_misc;
    p.wait_ns = ax.wait_ns;    // 0.5 s unless a test shortens it: a tile copy takes microseconds
    p.test_extra_tx = ax.test_extra_tx;
    p.wide_mul = ax.wide_mul;
    p.wide_add = ax.wide_add;
    p.edge = (ax.weff < ax.N) ? 1 : 0;     // full torus windows have no edge
    p.rows = (int)ax.N;
    if (ax.vblocks > 1) {
        p.N = ax.vNp;
        p.outer = ax.outer * ax.vblocks;
        p.hoff = 0;
        p.vN = ax.N;
        p.vblocks = ax.vblocks;
        p.vR = ax.vR;
        p.vhoff = ax.hoff;
        p.rows = ax.vR;
    }
}

hjlo_status dmalloc(void **ptr, size_t bytes, const char *what)
{
    static std::atomic<long long> counter{0};
    static long long fail_at = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *e = getenv("HJLO_TEST_FAIL_ALLOC");
        fail_at = e ? atoll(e) : -1;
    });
    *ptr = nullptr;
    long long k = ++counter;
    if (fail_at > 0 && k == fail_at) return set_error(HJLO_ENOMEM, "%s: injected allocation failure", what);
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_error(e, what);
    }
    return HJLO_OK;
}

void apply_test_knobs(AxisPlan &ax)
{
    const char *e = getenv("HJLO_TEST_EXTRA_TX");
    ax.test_extra_tx = e ? std::max(0, atoi(e)) : 0;
    e = getenv("HJLO_TEST_WAIT_NS");
    if (e) ax.wait_ns = std::max(0LL, atoll(e));
}

hjlo_status launch_pass(const AxisPlan &ax, int dtype, const void *src, void *dst, const double *hv,
                        double hv_scale, int32_t *amin, unsigned long long *counters, int *flags,
                        cudaStream_t st)
{
    if (ax.algo == KALGO_DECOMP) {
        if (amin) return set_error(HJLO_EUNSUPPORTED, "the decomposition method records no argmins");
        if (dtype != HJLO_F64) return set_error(HJLO_EUNSUPPORTED, "the decomposition method runs in binary64");
        return ax.dsplit ? launch_split(ax, src, dst, hv, hv_scale, counters, flags, st)
                         : launch_decomp(ax, src, dst, hv, hv_scale, counters, flags, st);
    }
    const int esize = (dtype == HJLO_F64) ? 8 : 4;
    PassParams p;
    fill_params(ax, p);
    p.src = src;
    p.dst = dst;
    p.hv = hv;
    p.amin = amin;
    p.counters = counters;
    p.flags = flags;
    p.hscale = hv_scale;
    p.hv_scaled = (hv_scale != 0.0) ? 1 : 0;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (ax.layout == LAYOUT_CONTIG) {
        p.use_tma = (ax.vblocks == 1) && (((uintptr_t)src & 15) == 0) && (((ax.N * esize) & 15) == 0);
    } else {
        p.use_tma = encode_strided(ax, esize, src, &map) ? 1 : 0;
    }
    return dispatch_single(ax, dtype, map, p, st);
}


hjlo_status launch_pass_batch(const AxisPlan &ax, int dtype, const BatchItem *d_items, long long count,
                              unsigned long long *counters, int *flags, cudaStream_t st)
{
    PassParams p;
    fill_params(ax, p);
    p.counters = counters;
    p.flags = flags;
    return dispatch_batch(ax, dtype, d_items, p, count, st);
}

hjlo_status device_facts(DeviceFacts &f)
{
    cudaError_t e = cudaGetDevice(&f.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&f.num_sms, cudaDevAttrMultiProcessorCount, f.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, f.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    f.smem_optin = (size_t)optin;
    return HJLO_OK;
}

}  // namespace hjlo
