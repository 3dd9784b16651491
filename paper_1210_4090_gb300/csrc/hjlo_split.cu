// hjlo_split.cu -- the decomposition method of Sec. 4 over one whole period
// of a line too long for one CTA.  Sec. 4.2-4.3 decompose the function over
// a period of the torus; at tolerance eta > 0 the result depends on the cut,
// so a long line cannot be cut into independently decomposed row blocks.
// Here the period's cut and convolutions are spread over many CTAs and give
// exactly what one CTA holding the whole line would (hjlo_decomp.cu):
//
//  1. classify   every interior point's slope increment (convex rule
//                >= -eta, concave rule <= 0) into two bitmaps, and every
//                piece's F = the number of kernel slopes strictly below its
//                slope (the quantity both Algorithm 1 and Algorithm 2 use);
//  2. local cut  per chunk of the span, the greedy cut of Sec. 4.3 started at
//                the chunk's first point as if a component began there;
//  3. stitch     per line, one warp walks the true cut from point 0: where
//                it reaches a start of a chunk's local cut the rest of that
//                chunk's cut is the true one (the cut is a deterministic
//                chain), so it jumps to the chunk's exit; elsewhere it takes
//                single greedy steps.  Then the true starts are marked and
//                the running state of the chain at each chunk's first piece
//                (its component's start and max of F so far) is scanned;
//  4. pieces     per chunk, each piece's component kind and A = the running
//                maximum of F from its component's start (convex: Algorithm
//                1's kernel pointer) or F itself (concave: alpha of Theorem
//                th:ccc);
//  5. emit       per block of outputs, every vertex of every component's
//                merged sequence that lands in the block -- each one a
//                candidate fl(f(d) + g(y)) of the scheme -- is minimised into
//                shared-memory keys, then stored with the potential term.
//
// Step 5 uses that every output vertex of a component is either a piece
// vertex (convex: (A(p), p + 1); concave: (A(p), p) and (A(p), p + 1)) or a
// point vertex (y, d) with d in an interval fixed by A at the point's two
// pieces and whether the point starts or ends its component, so a block
// needs only A, the kind bits and the start bits of the points and pieces
// whose vertices can reach it: its outputs plus one window to the left.
#include "hjlo_internal.h"
#include "hjlo_decomp.cuh"

#include <climits>

namespace hjlo {

namespace {

constexpr int kSplitThreads = 256;
constexpr int kEmitThreads = 1024;
constexpr int kStitchThreads = 1024;
constexpr int kCutWarps = 4;                 // chunks per CTA in the local cut (a warp each)
constexpr int kMaxChunkWords = 128;          // chunks of at most 4096 points
constexpr int kDefaultChunk = 1024;
constexpr size_t kStitchStage = 200 * 1024;  // the stitch walk's data staged in shared memory up to this size

struct SplitParams {
    const double *src;
    double *dst;
    const double *hv;
    double hscale;
    int hv_scaled;
    const double *kr64;          // kr64[t] = k[dhi - t]; f(d) = k[dlo + d] = kr64[n - d]
    unsigned long long *counters;
    int *flags;
    long long N, inner, lines;
    int n;                       // window length - 1
    int hoff;                    // (-dhi) mod N: lifted point y is grid point (y + hoff) mod N
    int L;                       // N + n points in the lifted span
    int CH, CW, B;               // chunk points (a multiple of 32), its words, chunks per line
    long long Wl;                // bitmap words per line (B * CW)
    long long Pl;                // per-piece ints per line (B * CH)
    int vR;                      // outputs per write-back block
    long long nblk;              // write-back blocks per line
    double eta;
    // scratch: bitmaps (Wl words per line), per-piece ints (Pl per line),
    // per-chunk ints (B per line)
    unsigned *cv, *cc;           // convex / concave rule holds at the point
    unsigned *ts;                // local cut starts, then the true starts
    unsigned *ms;                // starts the stitch walk took by single steps
    unsigned *pk;                // piece's component is convex
    unsigned *rk;                // the n kernel slopes' keys: high words, then low (set once per plan)
    int *F, *A;
    int *wmax;                   // max F over each word's 32 pieces (INT_MIN past the span)
    int *fcv, *fcc;              // first point of the chunk whose rule fails (-1: none)
    int *mall;                   // max F over the chunk's pieces
    int *X;                      // local cut: first chain point at or after the chunk's end
    int *lastl;                  // local cut: last start in the chunk (-1: none)
    int *mtl;                    // max F over the pieces from lastl to the chunk's end
    int *entry;                  // stitch: first true start that is a local start (-1: none)
    int *lsm;                    // stitch: last start taken by a single step (-1: none)
    int *cs, *cm;                // chain state at the chunk's first piece: start, max F so far
};

__device__ __forceinline__ long long line_base(const SplitParams &p, long long line)
{
    const long long o = line / p.inner, in = line - o * p.inner;
    return o * p.N * p.inner + in;
}

// Grid point of lifted point y in [0, L) (L < 2N).
__device__ __forceinline__ long long lifted(const SplitParams &p, int y)
{
    long long q = (long long)y + p.hoff;
    q -= (q >= p.N) ? p.N : 0;
    q -= (q >= p.N) ? p.N : 0;
    return q;
}

__device__ __forceinline__ bool bit_at(const unsigned *bits, int q) { return (bits[q >> 5] >> (q & 31)) & 1u; }

// f(d) = k[dlo + d], d in [0, n].
__device__ __forceinline__ double fval(const SplitParams &p, int d) { return __ldg(p.kr64 + (p.n - d)); }

// Kind of the component starting at s: the convex rule at s + 1 (a
// component of one piece, at the span's end, counts as convex).
__device__ __forceinline__ bool kind_at(const SplitParams &p, const unsigned *cv, int s)
{
    return (s + 1 < p.L - 1) ? bit_at(cv, s + 1) : true;
}

__device__ __forceinline__ int warp_min(int v)
{
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v)
{
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// First point q >= from whose bit is clear, by the whole warp (every lane
// calls it with the same arguments): the rest of from's chunk 32 words at a
// time, then the chunks' first clear points 32 chunks at a time.  The
// point L - 1 and every point after it are clear, so it returns at most
// L - 1 for from <= L - 1.
__device__ int warp_next_clear(const SplitParams &p, const unsigned *bits, const int *first, int from)
{
    const int lane = threadIdx.x & 31;
    if (from >= p.L - 1) return p.L - 1;
    const int cb = from / p.CH;
    const int wend = (cb + 1) * p.CW;
    const int w0 = from >> 5;
    for (int w = w0; w < wend; w += 32) {
        const int wi = w + lane;
        unsigned word = (wi < wend) ? ~bits[wi] : 0u;
        if (wi == w0) word &= 0xffffffffu << (from & 31);
        const unsigned has = __ballot_sync(0xffffffffu, word != 0u);
        if (has) {
            const int l = __ffs(has) - 1;
            const unsigned wl = __shfl_sync(0xffffffffu, word, l);
            return ((w + l) << 5) + __ffs(wl) - 1;
        }
    }
    for (int c = cb + 1; c < p.B; c += 32) {
        const int v = (c + lane < p.B) ? first[c + lane] : -1;
        const unsigned has = __ballot_sync(0xffffffffu, v >= 0);
        if (has) return __shfl_sync(0xffffffffu, v, __ffs(has) - 1);
    }
    return p.L - 1;
}

// The greedy cut's next start after a component starting at s (s < L - 1),
// by the whole warp, from the bitmaps in global memory.
__device__ int warp_next_start(const SplitParams &p, const unsigned *cv, const unsigned *cc, const int *fcv,
                               const int *fcc, int s)
{
    if (s + 1 >= p.L - 1) return p.L - 1;
    const bool convex = bit_at(cv, s + 1);
    return warp_next_clear(p, convex ? cv : cc, convex ? fcv : fcc, s + 2);
}

// The kernel's slopes f(i + 1) - f(i) as order-preserving keys (once per
// plan: the table does not change).
__global__ void split_slopes(SplitParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.n) dkey32(__dsub_rn(fval(p, i + 1), fval(p, i)), p.rk[i], p.rk[p.n + i]);
}

// ---------------------------------------------------------------- 1. classify

// One CTA per chunk.  Bits of points outside [1, L - 2] are clear, F of
// pieces outside [0, L - 2] is 0.
__global__ void __launch_bounds__(kSplitThreads) split_classify(SplitParams p)
{
    constexpr int G = 4;                                   // words per warp whose loads go out together
    __shared__ int s_fcv, s_fcc, s_mall;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const long long line = blockIdx.x / p.B;
    const int b = (int)(blockIdx.x - line * p.B);
    const long long base = line_base(p, line);
    const int n = p.n, L = p.L;
    if (tid == 0) {
        s_fcv = INT_MAX;
        s_fcc = INT_MAX;
        s_mall = INT_MIN;
    }
    __syncthreads();
    int fv = INT_MAX, fc = INT_MAX, mx = INT_MIN;
    unsigned *cv = p.cv + line * p.Wl, *cc = p.cc + line * p.Wl;
    int *F = p.F + line * p.Pl, *wmax = p.wmax + line * p.Wl;
    for (int w0 = warp; w0 < p.CW; w0 += G * nw) {
        double gm[G], g0[G], g1[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int q = b * p.CH + ((w0 + k * nw) << 5) + lane;
            const bool in = (w0 + k * nw < p.CW) && q < L - 1;
            g0[k] = in ? p.src[base + lifted(p, q) * p.inner] : 0.0;
            g1[k] = in ? p.src[base + lifted(p, q + 1) * p.inner] : 0.0;
            gm[k] = (in && q >= 1) ? p.src[base + lifted(p, q - 1) * p.inner] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int w = w0 + k * nw;
            if (w >= p.CW) break;                          // warp-uniform
            const int q = b * p.CH + (w << 5) + lane;
            bool okv = false, okc = false;
            int f = 0, fm = INT_MIN;
            if (q < L - 1) {
                const double r1 = __dsub_rn(g1[k], g0[k]);
                f = below(p.rk, p.rk + n, n, r1);
                fm = f;
                if (q >= 1) {
                    const double inc = __dsub_rn(r1, __dsub_rn(g0[k], gm[k]));
                    okv = inc >= -p.eta;
                    okc = inc <= 0.0;
                }
            }
            F[q] = f;
            fm = warp_max(fm);
            mx = max(mx, fm);
            const unsigned wv = __ballot_sync(0xffffffffu, okv), wc = __ballot_sync(0xffffffffu, okc);
            const int wq = b * p.CH + (w << 5);
            if (lane == 0) {
                cv[b * p.CW + w] = wv;
                cc[b * p.CW + w] = wc;
                wmax[b * p.CW + w] = fm;
            }
            if (~wv) fv = min(fv, wq + __ffs(~wv) - 1);
            if (~wc) fc = min(fc, wq + __ffs(~wc) - 1);
        }
    }
    if (lane == 0) {
        atomicMin(&s_fcv, fv);
        atomicMin(&s_fcc, fc);
        atomicMax(&s_mall, mx);
    }
    __syncthreads();
    if (tid == 0) {
        const long long c = line * p.B + b;
        p.fcv[c] = (s_fcv == INT_MAX) ? -1 : s_fcv;
        p.fcc[c] = (s_fcc == INT_MAX) ? -1 : s_fcc;
        p.mall[c] = s_mall;
    }
}

// Max of F over the pieces [q0, chunk end) of one chunk (pieces past L - 2
// count as INT_MIN), by the whole warp: the partial word of q0 from F, the
// chunk's later words from their maxima.
__device__ __forceinline__ int warp_tail_max(const SplitParams &p, const int *F, const int *wmax, int q0, int c1)
{
    const int lane = threadIdx.x & 31;
    const int wq = q0 >> 5;
    const int q = q0 + lane;
    int m = (q < ((wq + 1) << 5) && q < p.L - 1) ? F[q] : INT_MIN;
    for (int w = wq + 1 + lane; w < (c1 >> 5); w += 32) m = max(m, wmax[w]);
    return warp_max(m);
}

// ---------------------------------------------------------------- 2. local cut

// First clear bit at a position >= from (relative to the chunk's first
// point) among the staged words [0, nwords), or -1.
__device__ __forceinline__ int staged_next_clear(const unsigned *sw, int from, int nwords)
{
    int w = from >> 5;
    if (w >= nwords) return -1;
    unsigned word = ~sw[w] & (0xffffffffu << (from & 31));
    for (;;) {
        if (word) return (w << 5) + __ffs(word) - 1;
        if (++w >= nwords) return -1;
        word = ~sw[w];
    }
}

// One warp per chunk: the greedy cut of Sec. 4.3 from the chunk's first
// point, with the chunk's words (and the next chunk's first word) staged in
// shared memory.  Every lane walks the same chain (the values are
// warp-uniform); a component that runs past the staged words is finished
// by the warp from global memory.
__global__ void __launch_bounds__(32 * kCutWarps) split_local_cut(SplitParams p)
{
    __shared__ unsigned s_v[kCutWarps][kMaxChunkWords + 1];
    __shared__ unsigned s_c[kCutWarps][kMaxChunkWords + 1];
    __shared__ unsigned s_t[kCutWarps][kMaxChunkWords];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long gc = (long long)blockIdx.x * kCutWarps + wid;
    if (gc >= p.lines * p.B) return;                       // the whole warp
    const long long line = gc / p.B;
    const int b = (int)(gc - line * p.B);
    const unsigned *cv = p.cv + line * p.Wl, *cc = p.cc + line * p.Wl;
    const int *fcv = p.fcv + line * p.B, *fcc = p.fcc + line * p.B;
    const int c0 = b * p.CH, c1 = c0 + p.CH, w0 = b * p.CW, L = p.L;
    unsigned *sv = s_v[wid], *sc = s_c[wid], *st = s_t[wid];
#pragma unroll
    for (int r = 0; r < (kMaxChunkWords + 32) / 32; ++r) {   // loads of all rounds issued together
        const int i = lane + 32 * r;
        if (i > p.CW) continue;
        const bool in = (i < p.CW) || (b + 1 < p.B);
        sv[i] = in ? cv[w0 + i] : 0u;
        sc[i] = in ? cc[w0 + i] : 0u;
        if (i < p.CW) st[i] = 0u;
    }
    __syncwarp();
    int s = c0, last = -1, it = 0;
    while (s < c1 && s < L - 1 && it++ <= p.CH) {        // s advances every step
        last = s;
        if (lane == 0) st[(s - c0) >> 5] |= 1u << ((s - c0) & 31);
        int e = L - 1;
        if (s + 1 < L - 1) {
            const int r = s + 1 - c0;                      // <= CH: inside the staged words
            const bool convex = (sv[r >> 5] >> (r & 31)) & 1u;
            const int q = staged_next_clear(convex ? sv : sc, s + 2 - c0, p.CW + 1);
            e = (q >= 0) ? c0 + q
                         : warp_next_clear(p, convex ? cv : cc, convex ? fcv : fcc, c1 + 32);
        }
        s = e;
    }
    __syncwarp();
    const long long cw = line * p.Wl + w0;
    for (int i = lane; i < p.CW; i += 32) {
        p.ts[cw + i] = st[i];
        p.ms[cw + i] = 0u;
    }
    const int mt = (last >= 0) ? warp_tail_max(p, p.F + line * p.Pl, p.wmax + line * p.Wl, last, c1) : INT_MIN;
    if (lane == 0) {
        p.X[gc] = s;
        p.lastl[gc] = last;
        p.mtl[gc] = mt;
        p.entry[gc] = -1;
        p.lsm[gc] = -1;
    }
}

// ---------------------------------------------------------------- 3. stitch

// Running state of the chain at a piece: the start s of its component and
// the max of F from s (s < 0: no start seen in the part it summarises).
struct Run {
    int s, m;
};
__device__ __forceinline__ Run run_join(Run x, Run y) { return (y.s >= 0) ? y : Run{x.s, max(x.m, y.m)}; }
__device__ __forceinline__ Run run_shfl_up(Run r, int o)
{
    return Run{__shfl_up_sync(0xffffffffu, r.s, o), __shfl_up_sync(0xffffffffu, r.m, o)};
}

// Inclusive scan of one Run per thread over the CTA (every thread calls it;
// wt: 32 Runs of shared memory).  Returns the thread's inclusive prefix;
// *total = the CTA's whole join.
__device__ Run block_scan_run(Run v, Run *wt, Run *total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const Run u = run_shfl_up(v, o);
        if (lane >= o) v = run_join(u, v);
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
        Run t = (lane < nw) ? wt[lane] : Run{-1, INT_MIN};
        for (int o = 1; o < 32; o <<= 1) {
            const Run u = run_shfl_up(t, o);
            if (lane >= o) t = run_join(u, t);
        }
        if (lane < nw) wt[lane] = t;
    }
    __syncthreads();
    if (warp > 0) v = run_join(wt[warp - 1], v);
    *total = wt[nw - 1];
    __syncthreads();                                       // wt is reused by the next call
    return v;
}

// One CTA per line.  Warp 0 walks the true cut from point 0, on the local
// starts, rule bitmaps and chunk summaries staged in shared memory when they
// fit (stage = 1; lines up to about 2^19 points);
// then the CTA scans the chain's state at every chunk's first piece.  The
// chunks mark their true starts themselves (split_pieces).
__global__ void __launch_bounds__(kStitchThreads) split_stitch(SplitParams p, int stage)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Run s_wt[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const long long line = blockIdx.x;
    const int L = p.L, B = p.B;
    const unsigned *cv = p.cv + line * p.Wl, *cc = p.cc + line * p.Wl;
    const unsigned *ts = p.ts + line * p.Wl;
    unsigned *ms = p.ms + line * p.Wl;
    const int *fcv = p.fcv + line * B, *fcc = p.fcc + line * B;
    const int *X = p.X + line * B;
    int *lastl = p.lastl + line * B, *mtl = p.mtl + line * B;
    const int *mall = p.mall + line * B;
    int *entry = p.entry + line * B, *lsm = p.lsm + line * B;
    int *cs = p.cs + line * B, *cm = p.cm + line * B;
    const int *F = p.F + line * p.Pl;
    if (stage) {
        // the walk's reads, all of them, from shared memory: local starts,
        // both rule bitmaps, the chunks' exits and first failing points
        unsigned *sts = reinterpret_cast<unsigned *>(smem), *scv = sts + p.Wl, *scc = scv + p.Wl;
        int *sx = reinterpret_cast<int *>(scc + p.Wl), *sfv = sx + B, *sfc = sfv + B;
#pragma unroll 4
        for (long long i = tid; i < p.Wl; i += blockDim.x) {
            sts[i] = ts[i];
            scv[i] = cv[i];
            scc[i] = cc[i];
        }
#pragma unroll 2
        for (int i = tid; i < B; i += blockDim.x) {
            sx[i] = X[i];
            sfv[i] = fcv[i];
            sfc[i] = fcc[i];
        }
        ts = sts;
        cv = scv;
        cc = scc;
        X = sx;
        fcv = sfv;
        fcc = sfc;
        __syncthreads();
    }
    if (warp == 0) {
        // every iteration moves s forward (X[b] >= the chunk's end > s; a
        // greedy step ends after its start), so the walk ends within L steps
        int s = 0;
        long long it = 0;
        while (s < L - 1 && it++ <= (long long)L) {
            const int b = s / p.CH;
            if (bit_at(ts, s)) {
                if (lane == 0) entry[b] = s;
                s = X[b];
            } else {
                if (lane == 0) {
                    ms[s >> 5] |= 1u << (s & 31);
                    lsm[b] = s;
                }
                s = warp_next_start(p, cv, cc, fcv, fcc, s);
            }
            __syncwarp();
        }
        if (s < L - 1 && lane == 0) atomicOr(p.flags, FLAG_PRECOND);   // not reached: s always advances
    }
    __syncthreads();
    // the chunks' last true starts and max of F from there: a chunk that
    // joined its local cut ends with it; one that did not, with its last
    // single step (its max of F taken here, a warp per chunk, into the local
    // cut's slots, which that chunk no longer needs)
    for (int b = warp; b < B; b += nw) {
        if (entry[b] >= 0 || lsm[b] < 0) continue;
        const int mt = warp_tail_max(p, F, p.wmax + line * p.Wl, lsm[b], (b + 1) * p.CH);
        if (lane == 0) {
            lastl[b] = lsm[b];
            mtl[b] = mt;
        }
    }
    __syncthreads();
    // chain state at each chunk's first piece: scan of the chunks' summaries
    // (last start and max of F from it, or no start and the chunk's max)
    Run carry{0, INT_MIN};
    for (int b0 = 0; b0 < B; b0 += blockDim.x) {
        const int b = b0 + tid;
        Run v{-1, INT_MIN};
        if (b < B) v = (entry[b] >= 0 || lsm[b] >= 0) ? Run{lastl[b], mtl[b]} : Run{-1, mall[b]};
        Run total;
        const Run inc = block_scan_run(v, s_wt, &total);
        const Run ex = run_join(carry, inc);              // state after chunk b
        if (b + 1 < B) {
            cs[b + 1] = ex.s;
            cm[b + 1] = ex.m;
        }
        if (b0 == 0 && tid == 0) {
            cs[0] = 0;
            cm[0] = INT_MIN;
        }
        carry = run_join(carry, total);
    }
}

// ---------------------------------------------------------------- 4. pieces

// One CTA per chunk.  First the chunk's true starts: its local starts from
// the stitch's join on, and the single steps (counted as the components).
// Then each thread takes a run of consecutive pieces; the chain state at
// each run's first piece comes from a scan over the runs seeded with the
// chunk's state (cs, cm).
__global__ void __launch_bounds__(kSplitThreads) split_pieces(SplitParams p)
{
    __shared__ Run s_wt[32];
    __shared__ unsigned s_ts[kMaxChunkWords], s_pk[kMaxChunkWords];
    __shared__ unsigned long long s_count;
    const int tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
    const long long line = blockIdx.x / p.B;
    const int b = (int)(blockIdx.x - line * p.B);
    const long long cb = line * p.B + b;
    const int L = p.L;
    const unsigned *cv = p.cv + line * p.Wl;
    unsigned *ts = p.ts + line * p.Wl + (long long)b * p.CW;
    const unsigned *ms = p.ms + line * p.Wl + (long long)b * p.CW;
    const int *F = p.F + line * p.Pl;
    int *A = p.A + line * p.Pl;
    const int c0 = b * p.CH;
    if (tid == 0) s_count = (L == 1 && b == 0) ? 1ull : 0ull;   // a span of one point: one component
    __syncthreads();
    const int e = p.entry[cb];
    unsigned long long cnt = 0;
    for (int i = tid; i < p.CW; i += nthr) {
        const int q0 = c0 + (i << 5);
        unsigned keep = 0u;
        if (e >= 0) {
            if (q0 >= e) keep = 0xffffffffu;
            else if (q0 + 31 >= e) keep = 0xffffffffu << (e - q0);
        }
        const unsigned t = (ts[i] & keep) | ms[i];
        s_ts[i] = t;
        s_pk[i] = 0u;
        ts[i] = t;
        cnt += __popc(t);
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(&s_count, cnt);
    __syncthreads();
    const int run = (p.CH + nthr - 1) / nthr;
    const int q0 = c0 + min(tid * run, p.CH), q1 = c0 + min((tid + 1) * run, p.CH);
    const int qe = min(q1, L - 1);                         // pieces [q0, qe) exist
    Run v{-1, INT_MIN};
#pragma unroll 4
    for (int q = q0; q < qe; ++q) v = bit_at(s_ts, q - c0) ? Run{q, F[q]} : Run{v.s, max(v.m, F[q])};
    Run total;
    const Run inc = block_scan_run(v, s_wt, &total);
    // exclusive prefix: the state before this run
    Run prev = Run{__shfl_up_sync(0xffffffffu, inc.s, 1), __shfl_up_sync(0xffffffffu, inc.m, 1)};
    if (lane == 0) prev = (tid >> 5) ? s_wt[(tid >> 5) - 1] : Run{-1, INT_MIN};
    Run st = run_join(Run{p.cs[cb], p.cm[cb]}, prev);
    int ks = -1;
    bool convex = true;
    for (int q = q0; q < q1; ++q) {
        if (q >= qe) {
            A[q] = 0;
            continue;
        }
        st = bit_at(s_ts, q - c0) ? Run{q, F[q]} : Run{st.s, max(st.m, F[q])};
        if (st.s != ks) {
            ks = st.s;
            convex = kind_at(p, cv, ks);
        }
        A[q] = convex ? st.m : F[q];
        if (convex) atomicOr(&s_pk[(q - c0) >> 5], 1u << ((q - c0) & 31));
    }
    __syncthreads();
    for (int i = tid; i < p.CW; i += nthr) p.pk[line * p.Wl + (long long)b * p.CW + i] = s_pk[i];
    if (tid == 0 && s_count) atomicAdd(&p.counters[CNT_COMPONENTS], s_count);
}

// ---------------------------------------------------------------- 5. emit

// Output vertex at z = y + d of value fl(f(d) + g(y)) into the block's keys
// (z in [zlo, zlo + nkeys)).  A plain read skips the atomic for candidates
// that lose (keys only decrease).
__device__ __forceinline__ void emit_key(unsigned long long *keys, int zlo, int nkeys, int z, double v)
{
    const int x = z - zlo;
    if (x < 0 || x >= nkeys) return;
    unsigned khi, klo;
    dkey32(v, khi, klo);
    const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(&keys[x]);
    const unsigned chi = (unsigned)(cur >> 32), clo = (unsigned)cur;
    if (khi < chi || (khi == chi && klo < clo)) atomicMin(&keys[x], ((unsigned long long)khi << 32) | klo);
}

// The block's staged view of a line: points and pieces [gy0, gy1], their
// values g, A, and the start and kind bits (words from wb on).
struct Stage {
    const double *g;
    const int *A;
    const unsigned *ts, *pk;
    int gy0, wb;
    __device__ __forceinline__ bool start_bit(int q) const
    {
        return (ts[(q >> 5) - wb] >> (q & 31)) & 1u;
    }
    __device__ __forceinline__ bool convex_bit(int q) const
    {
        return (pk[(q >> 5) - wb] >> (q & 31)) & 1u;
    }
    __device__ __forceinline__ int a(int q) const { return A[q - gy0]; }
};

// The (up to two) intervals [a0, b0) and [a1, b1) of output positions z
// that point y reaches as a vertex (y, z - y) of its components' merged
// sequences, clipped to [zlo, zhi):
//   y starts a component (y <= L - 2):   [y, y + A(y) + 1)
//       (convex: the vertex (0, y) and kernel pieces i < A(y); concave: the
//       fan d in [0, A(y)])
//   y ends a component (y >= 1):          [y + A(y-1) + c, y + n + 1), c = 1 if convex
//       (convex: kernel pieces i >= A(y - 1); concave: the fan d in [A(y - 1), n])
//   y inside a convex component:          [y + A(y-1) + 1, y + A(y) + 1)
struct Spans {
    int a0, b0, a1, b1;
};
__device__ __forceinline__ Spans point_spans(const SplitParams &p, const Stage &sg, int y, int zlo, int zhi)
{
    const int L = p.L, n = p.n;
    Spans r{0, 0, 0, 0};
    const bool st = (y == 0) || (y < L - 1 && sg.start_bit(y));
    const bool en = (y == L - 1) || (y > 0 && sg.start_bit(y));
    if (st || en) {
        if (st && (y <= L - 2 || L == 1)) {           // L = 1: one point, the vertex (0, 0)
            r.a0 = y;
            r.b0 = y + sg.a(y) + 1;
        }
        if (en && y >= 1) {
            r.a1 = y + sg.a(y - 1) + (sg.convex_bit(y - 1) ? 1 : 0);
            r.b1 = y + n + 1;
        }
    } else if (sg.convex_bit(y)) {
        r.a0 = y + sg.a(y - 1) + 1;
        r.b0 = y + sg.a(y) + 1;
    }
    r.a0 = max(r.a0, zlo);
    r.b0 = max(min(r.b0, zhi), r.a0);
    r.a1 = max(r.a1, zlo);
    r.b1 = max(min(r.b1, zhi), r.a1);
    return r;
}

// Shared memory of the emit kernel for blocks of vR outputs: keys, g, A,
// the point vertices' offsets, two bit ranges.
size_t emit_smem(int vR, int n)
{
    const size_t span = (size_t)vR + n + 2;
    return sizeof(unsigned long long) * (size_t)vR + (sizeof(double) + 2 * sizeof(int)) * span +
           2 * sizeof(unsigned) * (span / 32 + 2);
}

// One CTA per block of vR outputs x in [x0, x1) of a line, z = x + n in
// [zlo, zhi).  Vertices reaching the block come from points y in
// [x0, x1 + n) and pieces p in [x0 - 1, x1 + n), all staged in shared
// memory; the point vertices are spread evenly over the threads by a scan
// of their counts (each thread a contiguous range of them).
__global__ void __launch_bounds__(kEmitThreads) split_emit(SplitParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nw = nthr >> 5;
    const long long line = blockIdx.x / p.nblk;
    const long long blk = blockIdx.x - line * p.nblk;
    const int n = p.n, L = p.L;
    const int x0 = (int)(blk * p.vR), x1 = (int)min((long long)x0 + p.vR, p.N);
    const int zlo = x0 + n, zhi = x1 + n, nkeys = x1 - x0;
    const int gy0 = max(0, x0 - 1), gy1 = min(L - 1, x1 + n);        // staged points [gy0, gy1]
    const int ylo = x0, yhi = min(L - 1, x1 + n - 1);                  // points [ylo, yhi]
    const int np = yhi - ylo + 1;
    const int qlo = gy0, qhi = min(L - 2, x1 + n - 1);                 // pieces [qlo, qhi]
    const int wb = gy0 >> 5, nwords = (gy1 >> 5) - wb + 1;
    const size_t span = (size_t)p.vR + n + 2;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem);
    double *g = reinterpret_cast<double *>(keys + p.vR);
    int *sA = reinterpret_cast<int *>(g + span);
    int *off = sA + span;                                              // [np + 1]
    unsigned *sts = reinterpret_cast<unsigned *>(off + span);
    unsigned *spk = sts + (span / 32 + 2);
    const long long base = line_base(p, line);
    const unsigned *ts = p.ts + line * p.Wl, *pk = p.pk + line * p.Wl;
    const int *A = p.A + line * p.Pl;
#pragma unroll 4
    for (int y = gy0 + tid; y <= gy1; y += nthr) {
        g[y - gy0] = p.src[base + lifted(p, y) * p.inner];
        sA[y - gy0] = (y <= L - 2) ? A[y] : 0;
    }
#pragma unroll 2
    for (int i = tid; i < nwords; i += nthr) {
        sts[i] = ts[wb + i];
        spk[i] = pk[wb + i];
    }
    for (int i = tid; i < nkeys; i += nthr) keys[i] = ~0ull;
    __syncthreads();
    const Stage sg{g, sA, sts, spk, gy0, wb};
    // counts of the point vertices: a run of points per thread, then a scan
    const int run = (np + nthr - 1) / nthr;
    const int i0 = min(tid * run, np), i1 = min(i0 + run, np);
    int sum = 0;
    for (int i = i0; i < i1; ++i) {
        const Spans r = point_spans(p, sg, ylo + i, zlo, zhi);
        off[i] = (r.b0 - r.a0) + (r.b1 - r.a1);
        sum += off[i];
    }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = (lane < nw) ? s_wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < nw) s_wsum[lane] = t;
    }
    __syncthreads();
    int acc = incl - sum + (warp ? s_wsum[warp - 1] : 0);   // exclusive prefix of this run
    for (int i = i0; i < i1; ++i) {
        const int c = off[i];
        off[i] = acc;
        acc += c;
    }
    const int total = s_wsum[nw - 1];
    if (tid == 0) off[np] = total;
    __syncthreads();
    // piece vertices
    for (int q = qlo + tid; q <= qhi; q += nthr) {
        const int a = sg.a(q);
        const double fa = fval(p, a);
        if (sg.convex_bit(q)) {
            emit_key(keys, zlo, nkeys, q + 1 + a, __dadd_rn(fa, g[q + 1 - gy0]));
        } else {
            emit_key(keys, zlo, nkeys, q + a, __dadd_rn(fa, g[q - gy0]));
            emit_key(keys, zlo, nkeys, q + 1 + a, __dadd_rn(fa, g[q + 1 - gy0]));
        }
    }
    // point vertices: thread t takes vertices [k0, k1); the first belongs to
    // the last point whose offset is <= k0, the others follow in order
    const long long per = ((long long)total + nthr - 1) / nthr;
    const int k0 = (int)min((long long)total, per * tid), k1 = (int)min((long long)total, per * (tid + 1));
    if (k0 < k1) {
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= k0) lo = mid; else hi = mid - 1;
        }
        int i = lo, k = k0;
        while (k < k1 && i < np) {
            const int y = ylo + i;
            const Spans r = point_spans(p, sg, y, zlo, zhi);
            const double gy = g[y - gy0];
            const int len0 = r.b0 - r.a0;
            const int end = min(k1, off[i + 1]);
            for (; k < end; ++k) {
                const int j = k - off[i];
                const int z = (j < len0) ? r.a0 + j : r.a1 + (j - len0);
                emit_key(keys, zlo, nkeys, z, __dadd_rn(fval(p, z - y), gy));
            }
            ++i;
        }
    }
    __syncthreads();
    // values, potential term, stores
    for (int i = tid; i < nkeys; i += nthr) {
        const unsigned long long k = keys[i];
        if (k == ~0ull) {                  // no vertex reached x: cannot happen for a convex kernel
            atomicOr(p.flags, FLAG_PRECOND);
            continue;
        }
        double m = dkey_decode(k);
        const long long at = base + (long long)(x0 + i) * p.inner;
        if (p.hv) m = __dsub_rn(m, p.hv_scaled ? __dmul_rn(p.hscale, p.hv[at]) : p.hv[at]);
        p.dst[at] = m;
    }
}

}  // namespace

// The kernels' static shared memory (a few hundred bytes) comes out of the
// CTA's; their dynamic shared memory is kept kStaticReserve below it.
constexpr size_t kStaticReserve = 1024;

hjlo_status split_allow_smem()
{
    const int dyn = 227 * 1024 - (int)kStaticReserve;
    cudaError_t e = cudaFuncSetAttribute(split_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(split_stitch, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    return e == cudaSuccess ? HJLO_OK : cuda_error(e, "cudaFuncSetAttribute(split)");
}

// Chunks of kDefaultChunk points (HJLO_DECOMP_CHUNK: a multiple of 32 in
// [64, 4096], for tests that want many chunks on short lines or few on long
// ones); write-back blocks of about one per SM over all lines, at least 256
// rows (HJLO_DECOMP_SPLIT_ROWS sets them), fewer while their shared memory
// does not fit (the 2^18-point pendulum at eta = dx, a whole run: 152
// blocks of 1725 rows 53 us per pass, 304 of 862 55 us, 76 of 3450 73 us).
hjlo_status shape_split(AxisPlan &ax, size_t smem_optin, int num_sms)
{
    smem_optin = (smem_optin > kStaticReserve) ? smem_optin - kStaticReserve : 0;
    const long long N = ax.N, n = ax.weff - 1, lines = ax.inner * ax.outer, L = N + n;
    if (L + n + 2 >= (1LL << 31) - 64)
        return set_error(HJLO_EUNSUPPORTED, "a line of %lld points is too long for the decomposition pass", N);
    int CH = kDefaultChunk;
    if (const char *e = getenv("HJLO_DECOMP_CHUNK")) {
        const int c = atoi(e);
        if (c >= 64 && c <= 32 * kMaxChunkWords && c % 32 == 0) CH = c;
    }
    const long long B = (L + CH - 1) / CH;
    long long vR = std::max(256LL, (N * lines + num_sms - 1) / num_sms);
    if (const char *e = getenv("HJLO_DECOMP_SPLIT_ROWS")) {
        const long long r = atoll(e);
        if (r >= 1) vR = r;
    }
    vR = std::min(vR, N);
    while (vR > 1 && emit_smem((int)vR, (int)n) > smem_optin) vR = vR * 3 / 4;
    if (emit_smem((int)vR, (int)n) > smem_optin)
        return set_error(HJLO_EUNSUPPORTED, "a window of %lld displacements is too wide for the decomposition pass",
                         (long long)ax.weff);
    const long long nblk = (N + vR - 1) / vR;
    if (lines * B > 0x7fffffffLL || lines * nblk > 0x7fffffffLL || lines > 0x7fffffffLL)
        return set_error(HJLO_EUNSUPPORTED, "too many lines or chunks for the decomposition pass");
    ax.algo = KALGO_DECOMP;
    ax.layout = (ax.inner == 1) ? LAYOUT_CONTIG : LAYOUT_STRIDED;
    ax.vblocks = 1;
    ax.vR = 0;
    ax.vNp = 0;
    ax.dsplit = 1;
    ax.dchunk = CH;
    ax.dB = (int)B;
    ax.dvR = (int)vR;
    ax.dnblk = nblk;
    ax.smem = emit_smem((int)vR, (int)n);
    ax.threads = kEmitThreads;                 // the write-back launch, which ntiles counts
    ax.ntiles = lines * nblk;
    ax.C = 1;
    ax.log2C = 0;
    return HJLO_OK;
}

namespace {

// Scratch layout of an axis (offsets into d_split; every array 16-byte aligned).
struct SplitLayout {
    size_t cv, cc, ts, ms, pk, rk, F, A, wmax, chunk[10], bytes;
};
SplitLayout split_layout(const AxisPlan &ax)
{
    SplitLayout s;
    const size_t lines = (size_t)(ax.inner * ax.outer), B = (size_t)ax.dB, CH = (size_t)ax.dchunk;
    const size_t words = lines * B * (CH / 32), pieces = lines * B * CH, chunks = lines * B;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 15) & ~size_t(15);
        return at;
    };
    s.cv = take(4 * words);
    s.cc = take(4 * words);
    s.ts = take(4 * words);
    s.ms = take(4 * words);
    s.pk = take(4 * words);
    s.rk = take(8 * (size_t)(ax.weff - 1));
    s.F = take(4 * pieces);
    s.A = take(4 * pieces);
    s.wmax = take(4 * words);
    for (int i = 0; i < 10; ++i) s.chunk[i] = take(4 * chunks);
    s.bytes = off;
    return s;
}

}  // namespace

size_t split_scratch_bytes(const AxisPlan &ax) { return ax.dsplit ? split_layout(ax).bytes : 0; }

namespace {

SplitParams split_params(const AxisPlan &ax)
{
    const SplitLayout lay = split_layout(ax);
    unsigned char *w = reinterpret_cast<unsigned char *>(ax.d_split);
    SplitParams p;
    memset(&p, 0, sizeof(p));
    p.kr64 = ax.d_kr64;
    p.N = ax.N;
    p.inner = ax.inner;
    p.lines = ax.inner * ax.outer;
    p.n = ax.weff - 1;
    p.hoff = ax.hoff;
    p.L = (int)(ax.N + ax.weff - 1);
    p.CH = ax.dchunk;
    p.CW = ax.dchunk / 32;
    p.B = ax.dB;
    p.Wl = (long long)ax.dB * p.CW;
    p.Pl = (long long)ax.dB * ax.dchunk;
    p.vR = ax.dvR;
    p.nblk = ax.dnblk;
    p.eta = ax.eta;
    p.cv = reinterpret_cast<unsigned *>(w + lay.cv);
    p.cc = reinterpret_cast<unsigned *>(w + lay.cc);
    p.ts = reinterpret_cast<unsigned *>(w + lay.ts);
    p.ms = reinterpret_cast<unsigned *>(w + lay.ms);
    p.pk = reinterpret_cast<unsigned *>(w + lay.pk);
    p.rk = reinterpret_cast<unsigned *>(w + lay.rk);
    p.F = reinterpret_cast<int *>(w + lay.F);
    p.A = reinterpret_cast<int *>(w + lay.A);
    p.wmax = reinterpret_cast<int *>(w + lay.wmax);
    int **chunk_arrays[10] = {&p.fcv, &p.fcc, &p.mall, &p.X, &p.lastl, &p.mtl, &p.entry, &p.lsm, &p.cs, &p.cm};
    for (int i = 0; i < 10; ++i) *chunk_arrays[i] = reinterpret_cast<int *>(w + lay.chunk[i]);
    return p;
}

}  // namespace

hjlo_status split_prepare(const AxisPlan &ax, cudaStream_t st)
{
    if (!ax.dsplit) return HJLO_OK;
    if (!ax.d_split || ax.split_bytes < split_scratch_bytes(ax))
        return set_error(HJLO_ECUDA, "decomposition scratch missing");
    const SplitParams p = split_params(ax);
    if (p.n > 0) split_slopes<<<(unsigned)((p.n + 255) / 256), 256, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HJLO_OK : cuda_error(e, "decomposition slopes launch");
}

hjlo_status launch_split(const AxisPlan &ax, const void *src, void *dst, const double *hv, double hv_scale,
                         unsigned long long *counters, int *flags, cudaStream_t st)
{
    if (!ax.d_split || ax.split_bytes < split_scratch_bytes(ax))
        return set_error(HJLO_ECUDA, "decomposition scratch missing");
    SplitParams p = split_params(ax);
    p.src = reinterpret_cast<const double *>(src);
    p.dst = reinterpret_cast<double *>(dst);
    p.hv = hv;
    p.hscale = hv_scale;
    p.hv_scaled = (hv_scale != 0.0) ? 1 : 0;
    p.counters = counters;
    p.flags = flags;
    const long long chunks = p.lines * p.B;
    split_classify<<<(unsigned)chunks, kSplitThreads, 0, st>>>(p);
    split_local_cut<<<(unsigned)((chunks + kCutWarps - 1) / kCutWarps), 32 * kCutWarps, 0, st>>>(p);
    const size_t stage = sizeof(int) * 3 * (size_t)(p.Wl + p.B);
    const bool staged = stage <= kStitchStage;
    split_stitch<<<(unsigned)p.lines, kStitchThreads, staged ? stage : 0, st>>>(p, staged ? 1 : 0);
    split_pieces<<<(unsigned)chunks, kSplitThreads, 0, st>>>(p);
    split_emit<<<(unsigned)(p.lines * p.nblk), kEmitThreads, ax.smem, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "decomposition kernel launch");
    return HJLO_OK;
}

}  // namespace hjlo
