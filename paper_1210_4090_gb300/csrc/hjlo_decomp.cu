// hjlo_decomp.cu -- the paper's own fast (min,plus) convolution (Sec. 4) as
// an axis pass: every line is split into convex and concave components
// (Sec. 4.3, with the tolerance eta of Sec. 4.4), each component is
// convolved with the convex kernel in linear time (Theorem th:convex /
// Algorithm 1 for a convex component; the three parts of Lemmas lm:seg and
// lm:simplif / Theorem th:ccc / Algorithm 2 for a concave one), and the
// output is the minimum over components (Sec. 4.3 step 3).
//
// One CTA per line.  A decomposition runs over one period of the line (its
// lifted span), as Sec. 4.2-4.3 take it; where the result cannot depend on
// where the cut starts (eta = 0: every component is exactly convex or
// concave and the method is exact), or where the caller asks for it
// (hjlo_plan_set_decomp's approximate restart option), a long or lonely
// contiguous line runs in row blocks, each block decomposing its own span.
// The lifted source line and the kernel are staged in
// shared memory; the slope-increment kinds of all interior points are
// classified in parallel into two bitmaps; one thread walks the bitmaps to
// cut the components greedily (the cut is a left-to-right dependency chain,
// a few word operations per component); then each warp takes whole
// components and convolves one with its 32 lanes: every piece of the
// component and of the kernel finds its place in the merged order by a
// binary search (F(j) = the number of kernel slopes below the component's
// slope j, and for a convex piece its running maximum, which is where
// Algorithm 1's pointer stands when it takes piece j), so the sequential
// merge becomes independent searches.  Outputs are merged into per-output
// order-preserving keys with shared-memory atomicMin, so the result does not
// depend on the order in which lanes or components finish.  Every output
// value is one candidate fl(u(y) + k(d)) of the scheme, so the pass is never
// below the scheme's.
#include "hjlo_internal.h"
#include "hjlo_decomp.cuh"

namespace hjlo {

namespace {

constexpr int kDecompThreads = 1024;   // upper bound; shape_decomp picks 256 or 1024
constexpr unsigned kConvexBit = 0x80000000u;
constexpr unsigned kLongBit = 0x40000000u;     // listed for the whole CTA (see below)
constexpr unsigned kIndexMask = 0x3fffffffu;
constexpr int kLongComponent = 512;    // components of at least this many pieces: the whole CTA
constexpr int kMaxLong = 64;           // listed long components per CTA (the rest stay with a warp)
constexpr int kMiscWarpTotals = 4;     // misc[4..36): warp totals of a block scan
constexpr int kMiscLongList = 36;      // misc[36..36+kMaxLong): indices of the long components
constexpr long long kSplitMinPoints = 4096;   // shorter lonely lines stay in one CTA (one launch, not five)

struct DecompParams {
    const double *src;
    double *dst;
    const double *hv;
    double hscale;
    int hv_scaled;
    const double *kr64;          // kr64[t] = k[dhi - t]; f(i) = k[dlo + i] = kr64[n - i]
    unsigned long long *counters;
    int *flags;
    long long N, inner, outer;
    int n;                       // window length - 1
    int hoff;                    // (-dhi) mod N
    int L;                       // N + n source points
    int nwords;                  // (L + 31) / 32
    double eta;
    int off_f, off_r, off_keys, off_cv, off_cc, off_comp, off_fm, off_misc;
    // row blocks (contiguous lines; vN = 0 otherwise): a line of vN points is
    // cut into vblocks blocks of N rows; block b of real line rl is CTA
    // rl * vblocks + b, with sources (b N + y + hoff) mod vN, y in [0, L)
    long long vN, vblocks;
};

// Candidate v for output x = z - n.  Most candidates lose: a plain read of
// the current key skips the atomic for them (keys only decrease, so a stale
// read can only cause an unneeded atomic, never a missed one).
__device__ __forceinline__ void emit(unsigned long long *keys, int n, int N, int z, double v)
{
    const int x = z - n;
    if (x >= 0 && x < N) {
        unsigned khi, klo;
        dkey32(v, khi, klo);
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(&keys[x]);
        const unsigned chi = (unsigned)(cur >> 32), clo = (unsigned)cur;
        if (khi < chi || (khi == chi && klo < clo))       // 32-bit compares (see dkey32)
            atomicMin(&keys[x], ((unsigned long long)khi << 32) | klo);
    }
}

// First point q in [from, to] whose bit is clear, or `none`.
__device__ int next_clear(const unsigned *bits, int from, int to, int none)
{
    if (from > to) return none;
    int w = from >> 5;
    unsigned word = ~bits[w] & (0xffffffffu << (from & 31));
    const int wlast = to >> 5;
    for (;;) {
        if (w == wlast) word &= (to & 31) == 31 ? 0xffffffffu : ((1u << ((to & 31) + 1)) - 1u);
        if (word) return (w << 5) + __ffs(word) - 1;
        if (++w > wlast) return none;
        word = ~bits[w];
    }
}

// Number of entries of the non-decreasing F[0..m) that are <= i.
__device__ __forceinline__ int upto(const int *F, int m, int i)
{
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (F[mid] <= i) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One component g[0..m] (source points s..s+m) convolved by a whole warp.
// F[0..m) is scratch.  Convex kind (Algorithm 1): Algorithm 1 takes kernel
// pieces while their slope is strictly below the component's current one,
// so when it takes component piece j its kernel pointer is
// Fmax(j) = max_{j' <= j} F(j') and the vertex after it is
// (Fmax(j), j + 1); kernel piece i is taken after J(i) = #{j : Fmax(j) <= i}
// component pieces, giving the vertex (i + 1, J(i)).  Concave kind: alpha_j =
// F(j) and the three parts of Theorem th:ccc.
__device__ void conv_component_warp(const double *f, const unsigned *rk, int n, const double *g, int m, int s,
                                    bool convex, int *F, unsigned long long *keys, int N)
{
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < m; j += 32) F[j] = below(rk, rk + n, n, __dsub_rn(g[j + 1], g[j]));
    __syncwarp();
    if (convex || m == 0) {
        int carry = 0;
        for (int j0 = 0; j0 < m; j0 += 32) {
            int v = (j0 + lane < m) ? F[j0 + lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int w = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = max(v, w);
            }
            v = max(v, carry);
            if (j0 + lane < m) F[j0 + lane] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
        __syncwarp();
        if (lane == 0) emit(keys, n, N, s, __dadd_rn(f[0], g[0]));
        for (int j = lane; j < m; j += 32) {
            const int i = F[j];
            emit(keys, n, N, s + i + j + 1, __dadd_rn(f[i], g[j + 1]));
        }
        for (int i = lane; i < n; i += 32) {
            const int J = upto(F, m, i);
            emit(keys, n, N, s + i + 1 + J, __dadd_rn(f[i + 1], g[J]));
        }
    } else {
        const int a0 = F[0], am = F[m - 1];
        for (int x = lane; x <= a0; x += 32) emit(keys, n, N, s + x, __dadd_rn(f[x], g[0]));
        for (int j = lane; j < m; j += 32) {
            const int a = F[j];
            emit(keys, n, N, s + j + a, __dadd_rn(f[a], g[j]));
            emit(keys, n, N, s + j + 1 + a, __dadd_rn(f[a], g[j + 1]));
        }
        for (int x = m + am + lane; x <= m + n; x += 32) emit(keys, n, N, s + x, __dadd_rn(f[x - m], g[m]));
    }
    __syncwarp();
}

// The same convolution as conv_component_warp by the whole CTA (every thread
// calls it): the pieces' searches and the emissions are spread over all
// threads and the running maximum of F is a block-wide scan (warp scans,
// then a scan of the warps' totals in wtot[0..32)).  For the long components
// that tolerance eta > 0 leaves, which would keep one warp busy while the
// others wait at the barrier.
__device__ void conv_component_block(const double *f, const unsigned *rk, int n, const double *g, int m, int s,
                                     bool convex, int *F, unsigned long long *keys, int N, int *wtot)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    for (int j = tid; j < m; j += nthr) F[j] = below(rk, rk + n, n, __dsub_rn(g[j + 1], g[j]));
    __syncthreads();
    if (convex || m == 0) {
        int carry = 0;
        for (int j0 = 0; j0 < m; j0 += nthr) {
            const int j = j0 + tid;
            int v = (j < m) ? F[j] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int w = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = max(v, w);
            }
            if (lane == 31) wtot[warp] = v;
            __syncthreads();
            if (warp == 0) {
                int t = (lane < nw) ? wtot[lane] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int w = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t = max(t, w);
                }
                if (lane < nw) wtot[lane] = t;
            }
            __syncthreads();
            v = max(v, carry);
            if (warp > 0) v = max(v, wtot[warp - 1]);
            if (j < m) F[j] = v;
            const int next = max(carry, wtot[nw - 1]);
            __syncthreads();                         // wtot is rewritten by the next chunk
            carry = next;
        }
        __syncthreads();
        if (tid == 0) emit(keys, n, N, s, __dadd_rn(f[0], g[0]));
        for (int j = tid; j < m; j += nthr) {
            const int i = F[j];
            emit(keys, n, N, s + i + j + 1, __dadd_rn(f[i], g[j + 1]));
        }
        for (int i = tid; i < n; i += nthr) {
            const int J = upto(F, m, i);
            emit(keys, n, N, s + i + 1 + J, __dadd_rn(f[i + 1], g[J]));
        }
    } else {
        const int a0 = F[0], am = F[m - 1];
        for (int x = tid; x <= a0; x += nthr) emit(keys, n, N, s + x, __dadd_rn(f[x], g[0]));
        for (int j = tid; j < m; j += nthr) {
            const int a = F[j];
            emit(keys, n, N, s + j + a, __dadd_rn(f[a], g[j]));
            emit(keys, n, N, s + j + 1 + a, __dadd_rn(f[a], g[j + 1]));
        }
        for (int x = m + am + tid; x <= m + n; x += nthr) emit(keys, n, N, s + x, __dadd_rn(f[x - m], g[m]));
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDecompThreads) decomp_kernel(DecompParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *g = reinterpret_cast<double *>(smem);
    double *f = reinterpret_cast<double *>(smem + p.off_f);
    unsigned *rk = reinterpret_cast<unsigned *>(smem + p.off_r);   // slope keys: high words, then low
    int *fm = reinterpret_cast<int *>(smem + p.off_fm);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem + p.off_keys);
    unsigned *cv = reinterpret_cast<unsigned *>(smem + p.off_cv);
    unsigned *cc = reinterpret_cast<unsigned *>(smem + p.off_cc);
    unsigned *comp = reinterpret_cast<unsigned *>(smem + p.off_comp);
    int *misc = reinterpret_cast<int *>(smem + p.off_misc);

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    const long long line = blockIdx.x;
    const int N = (int)p.N, n = p.n, L = p.L;
    long long base, stride;
    int rows = N;                               // outputs written back
    if (p.vN) {
        const long long rl = line / p.vblocks;
        const long long r0 = (line - rl * p.vblocks) * p.N;
        const long long left = p.vN - r0;
        rows = (int)(left < p.N ? left : p.N);
        base = rl * p.vN + r0;
        stride = 1;
        // ---- stage the block's span: g[y] = u((r0 + y - dhi) mod vN) (L <= vN: one wrap)
        const double *ls = p.src + rl * p.vN;
        const long long q0 = (r0 + p.hoff) % p.vN;
        for (int y = tid; y < L; y += nthr) {
            long long q = q0 + y;
            q = (q >= p.vN) ? q - p.vN : q;
            g[y] = ls[q];
        }
    } else {
        const long long o = line / p.inner, in = line - o * p.inner;
        base = o * p.N * p.inner + in;
        stride = p.inner;
        // ---- stage: g[y] = u((y - dhi) mod N)
        for (int y = tid; y < L; y += nthr) g[y] = p.src[base + (long long)((y + p.hoff) % N) * stride];
    }
    // f(i) = k[dlo + i]
    for (int i = tid; i <= n; i += nthr) f[i] = p.kr64[n - i];
    for (int x = tid; x < N; x += nthr) keys[x] = ~0ull;
    __syncthreads();
    for (int i = tid; i < n; i += nthr) dkey32(__dsub_rn(f[i + 1], f[i]), rk[i], rk[n + i]);   // kernel slopes

    // ---- kinds of the slope increment at every interior point q:
    // convex rule (increment >= -eta) and concave rule (increment <= 0)
    for (int b0 = (tid >> 5) << 5; b0 < (p.nwords << 5); b0 += nthr) {
        const int q = b0 + lane;
        bool okv = false, okc = false;
        if (q >= 1 && q <= L - 2) {
            const double inc = __dsub_rn(__dsub_rn(g[q + 1], g[q]), __dsub_rn(g[q], g[q - 1]));
            okv = inc >= -p.eta;
            okc = inc <= 0.0;
        }
        const unsigned wv = __ballot_sync(0xffffffffu, okv);
        const unsigned wc = __ballot_sync(0xffffffffu, okc);
        if (lane == 0) {
            cv[b0 >> 5] = wv;
            cc[b0 >> 5] = wc;
        }
    }
    __syncthreads();

    // ---- greedy cut: a component starting at s takes the kind of the
    // increment at s + 1 and ends at the first later point that breaks it;
    // components of kLongComponent pieces or more (up to kMaxLong of them)
    // are flagged and listed for the whole CTA
    if (tid == 0) {
        int nc = 0, nl = 0;
        if (L == 1) {
            comp[nc++] = 0u | kConvexBit;
            comp[nc] = 0u;
        } else {
            int s = 0;
            while (s < L - 1) {
                bool convex = true;
                int e = L - 1;
                if (s + 1 < L - 1) {
                    convex = (cv[(s + 1) >> 5] >> ((s + 1) & 31)) & 1u;
                    e = next_clear(convex ? cv : cc, s + 2, L - 2, L - 1);
                }
                const bool is_long = (e - s >= kLongComponent) && nl < kMaxLong;
                if (is_long) misc[kMiscLongList + nl++] = nc;
                comp[nc++] = (unsigned)s | (convex ? kConvexBit : 0u) | (is_long ? kLongBit : 0u);
                s = e;
            }
            comp[nc] = (unsigned)(L - 1);
        }
        misc[0] = nc;
        misc[1] = nl;
        atomicAdd(&p.counters[CNT_COMPONENTS], (unsigned long long)nc);
    }
    __syncthreads();

    // ---- convolve the components, minimum into the keys: long ones by the
    // whole CTA one after another, the others a warp each (the keys' minimum
    // does not depend on the order)
    const int nc = misc[0], nl = misc[1];
    for (int q = 0; q < nl; ++q) {
        const int c = misc[kMiscLongList + q];
        const int s = (int)(comp[c] & kIndexMask);
        const int e = (int)(comp[c + 1] & kIndexMask);
        conv_component_block(f, rk, n, g + s, e - s, s, (comp[c] & kConvexBit) != 0, fm + s, keys, N,
                             misc + kMiscWarpTotals);
    }
    for (int c = tid >> 5; c < nc; c += nthr >> 5) {
        if (comp[c] & kLongBit) continue;
        const int s = (int)(comp[c] & kIndexMask);
        const bool convex = (comp[c] & kConvexBit) != 0;
        const int e = (int)(comp[c + 1] & kIndexMask);
        conv_component_warp(f, rk, n, g + s, e - s, s, convex, fm + s, keys, N);
    }
    __syncthreads();

    // ---- values, potential term, stores
    for (int x = tid; x < rows; x += nthr) {
        const unsigned long long k = keys[x];
        if (k == ~0ull) {                  // no component reached x: cannot happen for a convex kernel
            atomicOr(p.flags, FLAG_PRECOND);
            continue;
        }
        double m = dkey_decode(k);
        const long long at = base + (long long)x * stride;
        if (p.hv) m = __dsub_rn(m, p.hv_scaled ? __dmul_rn(p.hscale, p.hv[at]) : p.hv[at]);
        p.dst[at] = m;
    }
}

// Shared memory of one CTA for lines (or row blocks) of N outputs.
size_t decomp_smem(const AxisPlan &ax, long long N, DecompParams *p)
{
    const long long n = ax.weff - 1, L = N + n, nwords = (L + 31) / 32;
    size_t off = 0;
    off += sizeof(double) * L;                                  // g
    const size_t off_f = off;
    off += sizeof(double) * (n + 1);
    const size_t off_r = off;                                   // n slope keys (two words each)
    off += sizeof(double) * (n + 1);
    off = (off + 15) & ~size_t(15);
    const size_t off_keys = off;
    off += sizeof(unsigned long long) * N;
    const size_t off_cv = off;
    off += sizeof(unsigned) * nwords;
    const size_t off_cc = off;
    off += sizeof(unsigned) * nwords;
    const size_t off_comp = off;
    off += sizeof(unsigned) * (L + 1);
    const size_t off_fm = off;
    off += sizeof(int) * (L + 1);
    const size_t off_misc = off;
    off += sizeof(int) * (kMiscLongList + kMaxLong);            // counts, warp totals, long list
    if (p) {
        p->off_f = (int)off_f;
        p->off_r = (int)off_r;
        p->off_fm = (int)off_fm;
        p->off_keys = (int)off_keys;
        p->off_cv = (int)off_cv;
        p->off_cc = (int)off_cc;
        p->off_comp = (int)off_comp;
        p->off_misc = (int)off_misc;
        p->n = (int)n;
        p->L = (int)L;
        p->nwords = (int)nwords;
    }
    return off;
}

}  // namespace

hjlo_status decomp_allow_smem()
{
    cudaError_t e = cudaFuncSetAttribute(decomp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return e == cudaSuccess ? HJLO_OK : cuda_error(e, "cudaFuncSetAttribute(decomp)");
}

hjlo_status shape_decomp(AxisPlan &ax, size_t smem_optin, int num_sms, bool blocks_ok)
{
    ax.algo = KALGO_DECOMP;
    ax.layout = (ax.inner == 1) ? LAYOUT_CONTIG : LAYOUT_STRIDED;
    ax.vblocks = 1;
    ax.vR = 0;
    ax.vNp = 0;
    ax.dsplit = 0;
    if (ax.weff >= 3 && !(ax.curv > 0))
        return set_error(HJLO_EPRECOND, "the decomposition pass needs a strictly convex kernel table");
    // Row blocks for a contiguous axis (blocks_ok), as for the other passes:
    // when the window is at most a quarter of the line and either a whole
    // line does not fit or the axis has fewer lines than half the SMs.  Each
    // block is decomposed on its own span (the cut restarts at the block's
    // first source).  Blocks hold one SM's share of the rows, at least
    // weff - 1 (the span is at most twice the rows: on the 2^18-point
    // pendulum at eta = dx, 161 blocks of 1636 rows ran 22 % faster than 81
    // of 3272).
    const long long N = ax.N, w = ax.weff, lines = ax.outer;
    const bool fits = decomp_smem(ax, N, nullptr) <= smem_optin;
    // whole periods (eta > 0) of a few long lines would leave most SMs idle
    // with one CTA per line: spread each period across CTAs instead (the
    // 2 x 4096-point pendulum at eta = dx, 289 steps: 7.7 ms against 14.7)
    if (!blocks_ok && N >= kSplitMinPoints && 2 * lines * ax.inner < num_sms)
        return shape_split(ax, smem_optin, num_sms);
    if (blocks_ok && ax.inner == 1 && 4 * w <= N && (!fits || 2 * lines < num_sms)) {
        long long vR = std::max(std::max(1LL, w - 1), (N * lines + num_sms - 1) / num_sms);
        const ShapeHints hint = env_hints();
        if (hint.block_rows > 0) vR = std::max(hint.block_rows, std::max(1LL, w - 1));
        while (vR > w - 1 && decomp_smem(ax, vR, nullptr) > smem_optin) vR = vR * 3 / 4;
        vR = std::min(vR, N - (w - 1));                  // span vR + weff - 1 <= N: one wrap
        if (vR >= std::max(1LL, w - 1) && vR < N && decomp_smem(ax, vR, nullptr) <= smem_optin) {
            ax.vR = (int)vR;
            ax.vblocks = (N + vR - 1) / vR;
        }
    }
    const long long rowsN = (ax.vblocks > 1) ? ax.vR : N;
    ax.smem = decomp_smem(ax, rowsN, nullptr);
    // a line that fits neither one CTA nor row blocks (eta > 0 without
    // restarts, a strided axis, a wide window): the period's cut and
    // convolutions across CTAs (hjlo_split.cu); HJLO_DECOMP_SPLIT=1 takes
    // that path for every line (tests)
    const char *force = getenv("HJLO_DECOMP_SPLIT");
    if ((force && atoi(force) == 1) || ax.smem > smem_optin || rowsN + ax.weff > (1LL << 30))
        return shape_split(ax, smem_optin, num_sms);
    if (ax.smem > smem_optin || rowsN + ax.weff > (1LL << 30))
        return set_error(HJLO_EUNSUPPORTED, "a line of %lld points does not fit the decomposition pass", ax.N);
    ax.ntiles = ax.inner * ax.outer * ax.vblocks;
    // one CTA per line: few lines (a 1D problem) get 32 warps each to hide
    // the latency of their components' searches; many lines get 8 warps
    // (measured: 2 x 4096-point pendulum 137 -> 100 ms, 1024^2 law 51 ms at
    // 256 threads against 64 ms at 1024)
    ax.threads = (ax.ntiles < 2LL * num_sms) ? kDecompThreads : 256;
    if (ax.ntiles > 0x7fffffffLL) return set_error(HJLO_EUNSUPPORTED, "too many lines");
    ax.C = 1;
    ax.log2C = 0;
    return HJLO_OK;
}

hjlo_status launch_decomp(const AxisPlan &ax, const void *src, void *dst, const double *hv, double hv_scale,
                          unsigned long long *counters, int *flags, cudaStream_t st)
{
    DecompParams p;
    memset(&p, 0, sizeof(p));
    const bool blocks = ax.vblocks > 1;
    decomp_smem(ax, blocks ? ax.vR : ax.N, &p);
    p.src = reinterpret_cast<const double *>(src);
    p.dst = reinterpret_cast<double *>(dst);
    p.hv = hv;
    p.hscale = hv_scale;
    p.hv_scaled = (hv_scale != 0.0) ? 1 : 0;
    p.kr64 = ax.d_kr64;
    p.counters = counters;
    p.flags = flags;
    p.N = blocks ? ax.vR : ax.N;
    p.inner = ax.inner;
    p.outer = ax.outer;
    p.hoff = ax.hoff;
    p.eta = ax.eta;
    if (blocks) {
        p.vN = ax.N;
        p.vblocks = ax.vblocks;
    }
    decomp_kernel<<<(unsigned)ax.ntiles, ax.threads, ax.smem, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decomposition kernel launch");
    return HJLO_OK;
}

}  // namespace hjlo
