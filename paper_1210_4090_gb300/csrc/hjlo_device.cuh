// hjlo_device.cuh -- device code of the axis pass (one min-plus convolution
// along one axis of the grid, Remark rk28 of Bouillard, Faou & Zavidovique,
// with the potential term of eq. eqconvol fused into the last axis).
//
// A CTA owns a tile of C lines x N positions.  It stages the tile in shared
// memory (TMA: one bulk copy for lines along the contiguous axis, a 3D tensor
// copy for lines along a strided axis), finds for every output i the argmin
// offset t (displacement d = dhi - t) and then writes
//     m_i = fl(u[(i-d) mod N] + k[d])          (one binary64 add)
//     u'_i = fl(m_i - hV_i)                    (last axis only)
// so each output costs exactly the binary64 operations of the definition.
//
// Halo index space.  For row i the window of lifted sources j = i - d,
// d in [dlo, dhi], is shifted to jj = j + dhi in [i, i + weff - 1]; the source
// position is (jj + hoff) mod N with hoff = (-dhi) mod N, and the kernel entry
// is kr[jj - i] = k[dhi - (jj - i)] (the table stored reversed).  Ascending jj
// is ascending lifted source, so a strict '<' scan keeps the smallest source
// among equal values (the library's tie rule).
//
// MONGE search.  u[j] + k[i-j] is a Monge matrix with margin
// a = min second difference of k > 0 (k convex, hypothesis (i)): the leftmost
// row argmin is non-decreasing in i, and along the periodic line
// argmin(i+N) = argmin(i) + N.  Lane g of the line's lpl lanes owns the rows
// [s_g, s_{g+1}), s_g = min(g*S, N) with S odd (so that lanes reading rows S
// apart fall in different shared-memory banks): it scans the whole window for
// its first row (the pivot) and then fills its segment by divide and conquer,
// each row searching only between the argmins of two rows already known.  Every
// comparison is made first on an int32 fixed-point screen: per line,
// (u - min u)/2^q and k/2^q truncated, 2^q chosen so that the line's range
// fills 29 bits; each screened candidate is within 3 units of the exact sum.
// When another candidate lies within 6 units (+ one binary64 ulp of the
// values, in units) of the screened minimum, the row is re-scanned in binary64
// over the surviving candidates, so the argmin (and the value) is the binary64
// one.  Ties in binary64 sit within the bracket as long as
// a > 8 ulp(max|u| + max|k|); a line that fails this margin (or holds
// non-finite values) is handed to the brute-force scan.  The conversions use
// integer instructions only: on this part the binary64 pipe is the scarce
// unit, and it is kept for the one add per output of the definition.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hjlo {

enum { LAYOUT_CONTIG = 0, LAYOUT_STRIDED = 1 };
enum { KALGO_BRUTE = 1, KALGO_MONGE = 2, KALGO_DECOMP = 3 };
enum { FLAG_PRECOND = 1, FLAG_TIMEOUT = 2 };
enum { CNT_RESCAN = 0, CNT_FALLBACK = 1, CNT_COMPONENTS = 2, CNT_EDGE = 3, CNT_N = 4 };

struct PassParams {
    const void *src;          // tile source (global)
    void *dst;                // output (global); may equal src
    const double *hv;         // h*V for the potential term, or nullptr
    int32_t *amin;            // argmin displacement d per point, or nullptr
    const double *kr64;       // kr64[t] = k[dhi - t], t in [0, weff)
    unsigned long long *counters;
    int *flags;
    long long N, inner, outer;
    long long ntiles;
    long long tiles_per_outer;  // STRIDED: ceil(inner / C)
    int hoff;                 // (-dhi) mod N
    int dhi;                  // argmin output: d = dhi - t
    int weff;                 // window size (<= N)
    int C, log2C;             // lines per tile (power of two)
    int wpl;                  // BRUTE: warps per line
    int lpl, log2lpl;         // MONGE: lanes per line (power of two)
    int seg;                  // MONGE: rows per lane segment (odd)
    int gs;                   // MONGE: lanes sharing one full-window pivot scan (power of two <= 32)
    int tp;                   // pitch (uint16) of a line's argmin offsets; tp % 4 == 2
    int use_tma;
    int by, nbox;             // STRIDED TMA: rows per box, boxes per tile
    int lp;                   // pitch (int32 words) of a line in the fixed-point halo
    double kmax;              // max |k| over the window
    double curv;              // lower bound of the min second difference of k (inf if weff < 3)
    int off_u, off_fx, off_kfx, off_t, off_k64, off_misc;  // shared memory offsets (bytes)
    long long wait_ns;        // bound on the first mbarrier wait of a tile
    int test_extra_tx;        // test knob: bytes the barrier expects beyond the copy (0 in use)
    double hscale;            // hv_scaled: potential term fl(m - fl(hscale * hv[x]))
    int hv_scaled;            // 0: hv already holds h*V
    int wide_mul, wide_add;   // MONGE: a bracket of more than wide_mul * (expected span) + wide_add
                              // offsets is searched by the whole warp
    int edge;                 // partial window: count argmins on its first or last displacement
    int rows;                 // rows searched per line: N, or in row-block mode the block's vR
    // Row blocks (contiguous lines only; vN = 0 otherwise).  A line of vN points
    // is cut into vblocks blocks of vR rows; block b of real line rl is the
    // tile line rl * vblocks + b, staged as a periodic line of N = vR + weff - 1
    // points: halo index jj <-> real position (b * vR + jj + vhoff) mod vN.
    // Its first vR rows see no wrap, so their minima are the real rows', and
    // only they are searched: the last segment's right bracket is row N,
    // the periodic image of row 0, a valid bracket for every row of the line.
    long long vN, vblocks;
    int vR, vhoff;
};

// Real line, first row and row count of tile line vl in row-block mode.
struct RowBlock {
    long long base;   // global index of the block's first row
    int rows;         // real rows of the block
};
__device__ __forceinline__ RowBlock row_block(const PassParams &p, long long vl)
{
    const long long rl = vl / p.vblocks;
    const long long r0 = (vl - rl * p.vblocks) * p.vR;
    const long long left = p.vN - r0;
    return RowBlock{rl * p.vN + r0, (int)(left < p.vR ? left : p.vR)};
}

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier for at most `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit_ns)
{
    unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_tensor_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                                   uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Hint: bring [p, p + bytes) of global memory into L2 ahead of use (whole
// 16-byte units inside the range only; the ragged ends load normally).
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned long long bytes)
{
    const unsigned long long a = (unsigned long long)__cvta_generic_to_global(p);
    unsigned long long s = (a + 15ull) & ~15ull;
    const unsigned long long e = (a + bytes) & ~15ull;
    while (s < e) {
        const unsigned long long n = (e - s < (1ull << 20)) ? e - s : (1ull << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)n) : "memory");
        s += n;
    }
}

// ------------------------------------------------------------------ number helpers

// Order-preserving integer key of a binary64 value, as two 32-bit words
// (high, low): negative values have every bit flipped, the others the sign
// bit set; -0 maps to +0's key so that equal values (IEEE ==) have equal
// keys.  Finite inputs only.  32-bit integer instructions only: on this GPU
// 64-bit integer compares share the binary64 pipe with the candidate adds.
__device__ __forceinline__ void dkey32(double x, unsigned &khi, unsigned &klo)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned neg = (unsigned)((int)hi >> 31);
    const bool mzero = (hi == 0x80000000u) && (lo == 0u);
    khi = mzero ? 0x80000000u : (hi ^ (neg | 0x80000000u));
    klo = mzero ? 0u : (lo ^ neg);
}

// The same key as one 64-bit word (for 64-bit atomics).
__device__ __forceinline__ unsigned long long dkey(double x)
{
    unsigned khi, klo;
    dkey32(x, khi, klo);
    return ((unsigned long long)khi << 32) | klo;
}

// dkey held as two 32-bit words, compared and shuffled with 32-bit
// instructions.
struct Key2 {
    unsigned hi, lo;
};
__device__ __forceinline__ Key2 key2_max() { return Key2{0xffffffffu, 0xffffffffu}; }
__device__ __forceinline__ Key2 key2(double x)
{
    Key2 k;
    dkey32(x, k.hi, k.lo);
    return k;
}
__device__ __forceinline__ bool key2_less(Key2 a, Key2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool key2_eq(Key2 a, Key2 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ Key2 key2_shfl_xor(Key2 a, int w)
{
    return Key2{__shfl_xor_sync(0xffffffffu, a.hi, w), __shfl_xor_sync(0xffffffffu, a.lo, w)};
}

// Inverse of dkey for keys of finite values.
__device__ __forceinline__ double dkey_decode(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k ^ 0x8000000000000000ull) : ~k;
    return __longlong_as_double((long long)b);
}

// Unbiased binary exponent of |x| (x finite, nonzero normal or subnormal).
__device__ __forceinline__ int expo(double x)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int eb = (int)((b >> 52) & 0x7ff);
    return (eb ? eb : 1) - 1023;
}

// x / 2^q truncated toward zero, modulo 2^32 (two's complement), with 32-bit
// integer instructions only.  The difference of two such values is exact
// modulo 2^32 up to the two truncations (each below one unit), so it is
// correct whenever the true difference fits in an int32 -- however large
// |x| / 2^q itself is.
__device__ __forceinline__ unsigned fixq32(double x, int q)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int eb = (int)((hi >> 20) & 0x7ffu);
    const unsigned mh = (hi & 0xfffffu) | (eb ? 0x100000u : 0u);   // significand = mh:lo (53 bits)
    const int k = 1075 + q - (eb ? eb : 1);                        // |x| / 2^q = significand / 2^k
    // k > 0: the low word of significand >> k, as two clamped funnel shifts
    // (>> min(k, 32), then >> min(k - 32, 32)), so k >= 64 gives 0;
    // k <= 0: the low word of significand << -k (0 from 32 on).  No branches.
    const unsigned a = __funnelshift_rc(lo, mh, (unsigned)max(k, 0));
    const unsigned vr = __funnelshift_rc(a, 0u, (unsigned)max(k - 32, 0));
    const unsigned vl = __funnelshift_lc(0u, lo, (unsigned)max(-k, 0));
    const unsigned v = (k > 0) ? vr : vl;
    const unsigned sg = (unsigned)((int)hi >> 31);
    return (v ^ sg) - sg;
}

// Exact binary32 -> binary64 (integer ops for normal numbers).
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x)
{
    unsigned b = __float_as_uint(x);
    unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;   // zero, subnormal, inf, nan
    unsigned long long r = ((unsigned long long)(b & 0x80000000u) << 32) |
                           ((unsigned long long)(e - 127u + 1023u) << 52) |
                           ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)r);
}

__device__ __forceinline__ void store_val(double *p, double m) { *p = m; }
__device__ __forceinline__ void store_val(float *p, double m) { *p = __double2float_rn(m); }

// Order-preserving int32 key of the high word of a binary64 value: keys of
// two values compare like the values, up to the discarded low word.
__device__ __forceinline__ int hikey(double x)
{
    int hi = (int)((unsigned long long)__double_as_longlong(x) >> 32);
    return hi ^ ((hi >> 31) & 0x7fffffff);
}

// A binary64 bound from a high-word key: the smallest (lower = true) or the
// largest value whose high word has this key.
__device__ __forceinline__ double hikey_bound(int key, bool lower)
{
    int hi = key ^ ((key >> 31) & 0x7fffffff);
    bool neg = hi < 0;
    unsigned lo = (neg == lower) ? 0xffffffffu : 0u;
    unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | lo;
    return __longlong_as_double((long long)b);
}

// ------------------------------------------------------------------ tile geometry

template <int LAYOUT>
struct Tile {
    long long base;     // global element index of (line 0, position 0)
    long long lstride;  // global stride between lines of the tile
    long long pstride;  // global stride between positions of a line
    int valid;          // lines of the tile that exist
};

template <int LAYOUT>
__device__ __forceinline__ Tile<LAYOUT> tile_of(const PassParams &p, long long tile)
{
    Tile<LAYOUT> t;
    if (LAYOUT == LAYOUT_CONTIG) {
        long long l0 = tile << p.log2C;
        t.base = l0 * p.N;
        t.lstride = p.N;
        t.pstride = 1;
        long long rem = p.outer - l0;
        t.valid = (int)(rem < p.C ? rem : p.C);
    } else {
        long long o = tile / p.tiles_per_outer;
        long long in0 = (tile - o * p.tiles_per_outer) << p.log2C;
        t.base = o * p.N * p.inner + in0;
        t.lstride = 1;
        t.pstride = p.inner;
        long long rem = p.inner - in0;
        t.valid = (int)(rem < p.C ? rem : p.C);
    }
    return t;
}

// shared-memory index of (line l, position i) in the staged tile
template <int LAYOUT>
__device__ __forceinline__ int uidx(const PassParams &p, int l, int i)
{
    return (LAYOUT == LAYOUT_CONTIG) ? (l * (int)p.N + i) : ((i << p.log2C) + l);
}

__device__ __forceinline__ int wrapN(int x, int N)
{
    x = (x >= N) ? x - N : x;
    return (x >= N) ? x - N : x;
}

// Exact scan of halo indices [lo, hi] for row r: smallest key, ascending jj.
template <typename T, int LAYOUT>
__device__ __forceinline__ void exact_scan(const PassParams &p, const T *su, const double *kr64, int l, int r,
                                           int lo, int hi, Key2 &best, int &bt)
{
    const int N = (int)p.N;
    int pos = wrapN(lo + p.hoff, N);
    for (int jj = lo; jj <= hi; ++jj) {
        const Key2 key = key2(__dadd_rn(widen(su[uidx<LAYOUT>(p, l, pos)]), kr64[jj - r]));
        if (key2_less(key, best)) { best = key; bt = jj - r; }
        pos = (pos + 1 == N) ? 0 : pos + 1;
    }
}

// Screened search of row r over the offsets t in [tlo, thi] (halo index
// r + t); f = the line's fixed-point halo shifted to row r, k = the line's
// fixed-point kernel table.  Returns the argmin offset t.  `rescans` counts
// rows that needed the binary64 re-scan.
template <typename T, int LAYOUT>
__device__ __forceinline__ int screened_row(const PassParams &p, const T *su, const int *f, const int *k,
                                            const double *kr64, int l, int r, int tlo, int thi, int thr_add,
                                            int &rescans)
{
    int m1 = 0x7fffffff, m2 = 0x7fffffff, t1 = tlo;
    if (thi - tlo < 4) {
        // short brackets (most rows of the divide and conquer): four
        // candidates without a loop, those past thi masked
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = min(tlo + q, thi);
            const int c = (tlo + q <= thi) ? f[t] + k[t] : 0x7fffffff;
            m2 = min(m2, max(m1, c));
            t1 = (c < m1) ? t : t1;
            m1 = min(m1, c);
        }
    } else {
#pragma unroll 4
        for (int t = tlo; t <= thi; ++t) {
            int c = f[t] + k[t];
            m2 = min(m2, max(m1, c));
            t1 = (c < m1) ? t : t1;
            m1 = min(m1, c);
        }
    }
    const int thr = m1 + thr_add;
    if (m2 > thr) return t1;
    // another candidate is within the screen's error: binary64 over the survivors
    ++rescans;
    const int N = (int)p.N;
    Key2 best = key2_max();
    int bt = t1;
    for (int t = tlo; t <= thi; ++t) {
        int c = f[t] + k[t];
        if (c <= thr) {
            int pos = wrapN(r + t + p.hoff, N);
            const Key2 key = key2(__dadd_rn(widen(su[uidx<LAYOUT>(p, l, pos)]), kr64[t]));
            if (key2_less(key, best)) { best = key; bt = t; }
        }
    }
    return bt;
}

// Search of one row per lane with offload: lanes whose bracket [tlo, thi]
// is at least `wide` offsets long (rows next to a shock of the argmin map)
// hand their rows to the warp, which splits into k groups of 32/k lanes
// (k = the number of such rows, rounded up to a power of two) that search
// them side by side; the other lanes scan their own rows first.  Each group
// returns what the sequential screened_row returns (smallest screened value,
// first offset on ties; binary64 re-scan of the survivors when a second
// candidate is within the screen's error).  Every lane of the warp must call
// it (has = false for lanes without a row).  Returns this lane's offset.
template <typename T, int LAYOUT>
__device__ __forceinline__ int row_or_offload(const PassParams &p, const T *su, const int *fx, const int *kfx,
                                              const double *kr64, int line, int r, int tlo, int thi,
                                              int thr_add, bool has, int wide, int &rescans)
{
    const bool longj = has && (thi - tlo >= wide);
    int t = 0;
    if (has && !longj)
        t = screened_row<T, LAYOUT>(p, su, fx + line * p.lp + r, kfx + line * p.weff, kr64, line, r, tlo, thi,
                                    thr_add, rescans);
    const unsigned mask = __ballot_sync(0xffffffffu, longj);
    if (mask == 0u) return t;
    const int lane = threadIdx.x & 31;
    const int k = __popc(mask);
    int lgG = 5;                                   // group size G = 2^lgG = 32 / next_pow2(k)
    while ((1 << (5 - lgG)) < k) --lgG;
    const int G = 1 << lgG;
    const int job = lane >> lgG, sl = lane & (G - 1);
    const bool gact = job < k;
    // the lane holding the job-th long row
    unsigned m = mask;
    for (int i = 0; i < job && m; ++i) m &= m - 1;
    const int src = (gact && m) ? __ffs(m) - 1 : lane;
    const int rb = __shfl_sync(0xffffffffu, r, src);
    const int lob = __shfl_sync(0xffffffffu, tlo, src);
    const int hib = __shfl_sync(0xffffffffu, thi, src);
    const int lnb = __shfl_sync(0xffffffffu, line, src);
    const int thb = __shfl_sync(0xffffffffu, thr_add, src);
    const int *f = fx + lnb * p.lp + rb;
    const int *kk = kfx + lnb * p.weff;
    int m1 = 0x7fffffff, m2 = 0x7fffffff, t1 = 0x7fffffff;
    if (gact) {
        for (int tt = lob + sl; tt <= hib; tt += G) {
            const int c = f[tt] + kk[tt];
            m2 = min(m2, max(m1, c));
            t1 = (c < m1) ? tt : t1;
            m1 = min(m1, c);
        }
    }
    for (int w = G >> 1; w; w >>= 1) {
        const int om1 = __shfl_xor_sync(0xffffffffu, m1, w);
        const int om2 = __shfl_xor_sync(0xffffffffu, m2, w);
        const int ot1 = __shfl_xor_sync(0xffffffffu, t1, w);
        const int nm2 = min(max(m1, om1), min(m2, om2));
        if (om1 < m1 || (om1 == m1 && ot1 < t1)) { m1 = om1; t1 = ot1; }
        m2 = nm2;
    }
    const int thr = gact ? m1 + thb : 0;
    const bool need = gact && !(m2 > thr);
    int res = t1;
    if (__any_sync(0xffffffffu, need)) {
        const int N = (int)p.N;
        Key2 bk = key2_max();
        int bt = 0x7fffffff;
        if (need) {
            for (int tt = lob + sl; tt <= hib; tt += G) {
                if (f[tt] + kk[tt] <= thr) {
                    const int pos = wrapN(rb + tt + p.hoff, N);
                    const Key2 key = key2(__dadd_rn(widen(su[uidx<LAYOUT>(p, lnb, pos)]), kr64[tt]));
                    if (key2_less(key, bk)) { bk = key; bt = tt; }
                }
            }
        }
        for (int w = G >> 1; w; w >>= 1) {
            const Key2 ok = key2_shfl_xor(bk, w);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, w);
            if (key2_less(ok, bk) || (key2_eq(ok, bk) && ot < bt)) { bk = ok; bt = ot; }
        }
        if (need) res = bt;
    }
    // the owner of the j-th long row reads lane j * G (its group's first lane)
    const int rank = __popc(mask & ((1u << lane) - 1u));
    const int from = longj ? (rank << lgG) : lane;
    const int got = __shfl_sync(0xffffffffu, res, from);
    const int gneed = __shfl_sync(0xffffffffu, need ? 1 : 0, from);
    if (longj) {
        t = got;
        rescans += gneed;
    }
    return t;
}

// ------------------------------------------------------------------ the pass kernel

// 1 when offset t is the first or last of the window (t = 0 or weff - 1).
__device__ __forceinline__ int on_edge(int t, int weff) { return (unsigned)(t - 1) >= (unsigned)(weff - 2) ? 1 : 0; }

// Adds the threads' window-edge argmins of this tile to the plan's counter;
// every lane of the warp must call it.
__device__ __forceinline__ void count_edges(const PassParams &p, int edges)
{
    if (!p.edge) return;
    const int we = __reduce_add_sync(0xffffffffu, edges);
    if ((threadIdx.x & 31) == 0 && we) atomicAdd(&p.counters[CNT_EDGE], (unsigned long long)we);
}

// Write-back of rows i = i0, i0 + step, ... < i1 of one contiguous line: the
// exact value fl(u[src] + k[d]) at the recorded argmin, minus fl(h V) when
// the pass carries the potential term, stored (binary32: rounded), with the
// optional argmin.  Four rows per thread at a time, their potential-term
// loads issued together.  Returns how many of the rows' argmins sit on the
// window's edge.
template <typename T, typename OFF>
__device__ __forceinline__ int write_rows_contig(const PassParams &p, const T *lu, const OFF *lt,
                                                  const double *kr64, T *dst, long long xb, int i0, int i1, int step)
{
    const int N = (int)p.N;
    T *gd = dst + xb;
    const double *gh = p.hv ? p.hv + xb : nullptr;
    int32_t *ga = p.amin ? p.amin + xb : nullptr;
    int edges = 0;
    int i = i0;
    for (; i + 3 * step < i1; i += 4 * step) {
        double hvb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) hvb[b] = gh ? __ldg(gh + i + b * step) : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ii = i + b * step;
            const int t = lt[ii];
            const int pos = wrapN(ii + t + p.hoff, N);
            double m = __dadd_rn(widen(lu[pos]), kr64[t]);
            if (gh) m = __dsub_rn(m, p.hv_scaled ? __dmul_rn(p.hscale, hvb[b]) : hvb[b]);
            store_val(gd + ii, m);
            if (ga) ga[ii] = p.dhi - t;
            edges += on_edge(t, p.weff);
        }
    }
    for (; i < i1; i += step) {
        const int t = lt[i];
        const int pos = wrapN(i + t + p.hoff, N);
        double m = __dadd_rn(widen(lu[pos]), kr64[t]);
        if (gh) m = __dsub_rn(m, p.hv_scaled ? __dmul_rn(p.hscale, gh[i]) : gh[i]);
        store_val(gd + i, m);
        if (ga) ga[i] = p.dhi - t;
        edges += on_edge(t, p.weff);
    }
    return edges;
}

// Per-line facts of the fixed-point screen, in shared memory.
struct LineInfo {
    unsigned fref;                  // fixq32(lower bound of u, q)
    int pad0;
    int kmin, kmax;                 // hikey of min u and max u over the line
    int q;                          // unit 2^q
    int thr_add;                    // survivors: screened value <= min + thr_add
    int fallback;                   // 1: brute force for this line
    int pad;
};

// One tile of one axis pass (everything a CTA does).  `tmap` is the 3D TMA
// descriptor of the source for strided lines (unused otherwise).  OFF holds
// the rows' argmin offsets in shared memory: bytes when the window has at
// most 256 displacements (more lines per SM), else 16-bit words.
template <typename T, int LAYOUT, int ALGO, typename OFF = unsigned short>
__device__ __forceinline__ void pass_tile(const CUtensorMap *tmap, const PassParams &p, long long tile)
{
    extern __shared__ __align__(128) unsigned char smem[];
    T *su = reinterpret_cast<T *>(smem + p.off_u);
    int *fx = reinterpret_cast<int *>(smem + p.off_fx);
    int *kfx = reinterpret_cast<int *>(smem + p.off_kfx);
    OFF *tt = reinterpret_cast<OFF *>(smem + p.off_t);
    double *kr64 = reinterpret_cast<double *>(smem + p.off_k64);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + p.off_misc);
    LineInfo *li = reinterpret_cast<LineInfo *>(smem + p.off_misc + 16);         // [C]

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int N = (int)p.N, C = p.C, weff = p.weff;
    const Tile<LAYOUT> tl = tile_of<LAYOUT>(p, tile);
    const T *src = reinterpret_cast<const T *>(p.src);

    // ---- stage the tile
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (ALGO == KALGO_MONGE && tid < C) {
        li[tid].kmin = 0x7fffffff;
        li[tid].kmax = (int)0x80000000;
    }
    __syncthreads();
    if (p.use_tma) {
        if (tid == 0) {
            if (LAYOUT == LAYOUT_CONTIG) {
                uint32_t bytes = (uint32_t)((long long)tl.valid * N * (long long)sizeof(T));
                mbar_arrive_expect_tx(bar, bytes + (uint32_t)p.test_extra_tx);
                tma_bulk_load(su, src + tl.base, bytes, bar);
            } else {
                uint32_t bytes = (uint32_t)(p.nbox * p.by * C * (int)sizeof(T));
                mbar_arrive_expect_tx(bar, bytes + (uint32_t)p.test_extra_tx);
                long long o = tile / p.tiles_per_outer;
                int x0 = (int)((tile - o * p.tiles_per_outer) << p.log2C);
                for (int b = 0; b < p.nbox; ++b)
                    tma_tensor_load_3d(su + (long long)b * p.by * C, tmap, x0, b * p.by, (int)o, bar);
            }
        }
    } else if (LAYOUT == LAYOUT_CONTIG && p.vN) {
        // row blocks: gather each block's window span from its real line
        // (N <= vN, so one wrap at most)
        for (int l = 0; l < tl.valid; ++l) {
            const long long vl = (tile << p.log2C) + l;
            const long long rl = vl / p.vblocks;
            const T *ls = src + rl * p.vN;
            const long long s0 = ((vl - rl * p.vblocks) * p.vR + p.vhoff) % p.vN;
            for (int i = tid; i < N; i += nthr) {
                long long q = s0 + i;
                q = (q >= p.vN) ? q - p.vN : q;
                su[l * N + i] = ls[q];
            }
        }
    } else {
        for (int l = 0; l < tl.valid; ++l)
            for (int i = tid; i < N; i += nthr)
                su[uidx<LAYOUT>(p, l, i)] = src[tl.base + l * tl.lstride + (long long)i * tl.pstride];
    }
    // the potential term of a contiguous tile is read at the very end: start
    // moving it towards L2 now, behind the search
    if (LAYOUT == LAYOUT_CONTIG && p.hv && !p.vN && tid == nthr - 1)
        prefetch_l2(p.hv + tl.base, (unsigned long long)tl.valid * N * sizeof(double));
    for (int i = tid; i < weff; i += nthr) kr64[i] = p.kr64[i];
    if (p.use_tma) {
        bool ok = mbar_wait_bounded(bar, 0, p.wait_ns);
        if (__syncthreads_or(!ok)) {
            // the copy did not land in time: flag it, give it one more bounded
            // wait so nothing is still writing our shared memory, and leave
            if (tid == 0) atomicOr(p.flags, FLAG_TIMEOUT);
            mbar_wait_bounded(bar, 0, 500000000LL);
            return;
        }
    } else {
        __syncthreads();
    }

    const int lane = tid & 31, warp = tid >> 5;

    if (ALGO == KALGO_MONGE) {
        const int lpl = p.lpl;
        // line-major thread groups for the contiguous layout: lpl consecutive
        // threads per line (nthr = C * lpl)
        const int cl = tid >> p.log2lpl, sub = tid & (lpl - 1);
        // ---- per-line range from high-word keys (integer instructions only)
        {
            int mn = 0x7fffffff, mx = (int)0x80000000;
            if (LAYOUT == LAYOUT_CONTIG) {
                if (cl < tl.valid)
                    for (int i = sub; i < N; i += lpl) {
                        int k = hikey(widen(su[cl * N + i]));
                        mn = min(mn, k);
                        mx = max(mx, k);
                    }
                const int lim = lpl < 32 ? lpl : 32;
                for (int o = lim >> 1; o; o >>= 1) {
                    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                }
                if ((lane & (lim - 1)) == 0 && cl < tl.valid) {
                    atomicMin(&li[cl].kmin, mn);
                    atomicMax(&li[cl].kmax, mx);
                }
            } else {
                // line index fastest: consecutive threads read consecutive
                // words; each thread keeps one line (nthr is a multiple of C)
                const int l = tid & (C - 1);
                for (int idx = tid; idx < C * N; idx += nthr) {
                    int k = hikey(widen(su[idx]));
                    mn = min(mn, k);
                    mx = max(mx, k);
                }
                for (int o = 16; o >= C; o >>= 1) {
                    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                }
                if (lane < C && l < tl.valid) {
                    atomicMin(&li[l].kmin, mn);
                    atomicMax(&li[l].kmax, mx);
                }
            }
        }
        __syncthreads();
        // ---- per-line scale, survivor threshold and Monge margin
        if (tid < tl.valid) {
            LineInfo &L = li[tid];
            const double umin = hikey_bound(L.kmin, true), umax = hikey_bound(L.kmax, false);
            const double R = __dsub_ru(umax, umin);
            const double Rk = __dadd_ru(R, __dmul_ru(2.0, p.kmax));
            const double cmax = __dadd_ru(fmax(fabs(umin), fabs(umax)), p.kmax);
            const bool finite = isfinite(Rk) && isfinite(cmax);
            const int q = (finite && Rk > 0.0) ? expo(Rk) - 28 : -1074;
            int tie = finite ? expo(cmax) - 52 - q : 0;
            tie = tie < 0 ? 0 : (tie > 28 ? 28 : tie);
            L.q = q;
            L.fref = fixq32(umin, q);
            L.thr_add = 7 + (1 << tie);
            L.fallback = (!finite || !(p.curv > __dmul_ru(cmax, 0x1p-49))) ? 1 : 0;
        }
        __syncthreads();
        // ---- fixed-point halo of every line and the line's kernel table.  The
        // halo holds N + weff - 1 entries; entry jj + N repeats entry jj (same
        // position one period later), so each position is converted once.
        if (LAYOUT == LAYOUT_CONTIG) {
            if (cl < tl.valid) {
                const int q = li[cl].q;
                const unsigned fref = li[cl].fref;
                int *lfx = fx + cl * p.lp;
                const T *lu = su + cl * N;
                int pos = (sub + p.hoff) % N;
                for (int jj = sub; jj < N; jj += lpl) {
                    const int v = (int)(fixq32(widen(lu[pos]), q) - fref);
                    lfx[jj] = v;
                    if (jj < weff - 1) lfx[jj + N] = v;
                    pos += lpl;                      // lpl <= N
                    pos = (pos >= N) ? pos - N : pos;
                }
                for (int t = sub; t < weff; t += lpl) kfx[cl * weff + t] = (int)fixq32(kr64[t], q);
            }
        } else {
            const int l = tid & (C - 1);
            if (l < tl.valid) {
                const int q = li[l].q;
                const unsigned fref = li[l].fref;
                const int step = nthr >> p.log2C;
                int *lfx = fx + l * p.lp;
                int jj = tid >> p.log2C;
                int pos = (jj + p.hoff) % N;
                const int stepN = step % N;
                for (; jj < N; jj += step) {
                    const int v = (int)(fixq32(widen(su[(pos << p.log2C) + l]), q) - fref);
                    lfx[jj] = v;
                    if (jj < weff - 1) lfx[jj + N] = v;
                    pos += stepN;
                    pos = (pos >= N) ? pos - N : pos;
                }
                for (int t = tid >> p.log2C; t < weff; t += step) kfx[l * weff + t] = (int)fixq32(kr64[t], q);
            }
        }
        __syncthreads();
        // ---- monotone search: lane g of line `line` owns rows [s0, s1).
        // Every barrier and shuffle below is reached by all threads of the
        // block; the work between them is predicated per thread (lines of one
        // warp may differ in validity and in fallback).
        const int line = cl;
        const int g = sub;
        const bool active = line < tl.valid;
        const int lsafe = active ? line : 0;
        const int thr_add = li[lsafe].thr_add;
        const bool fallback = li[lsafe].fallback != 0;
        const int *lfx = fx + lsafe * p.lp;
        const int *lk = kfx + lsafe * weff;
        OFF *lt = tt + lsafe * p.tp;
        const bool work = active && !fallback;
        int rescans = 0;
        const int S = p.seg, GS = p.gs;
        const int NR = p.rows;                // rows searched (N, or a row block's vR)
        const int s0 = min(g * S, NR), s1 = min((g + 1) * S, NR);
        const int o = g & (GS - 1);
        const int rp = min((g - o) * S, NR);  // the group's pivot row
        if (active && fallback) {
            // brute force over each lane's own segment of rows
            for (int r = s0; r < s1; ++r) {
                Key2 best = key2_max();
                int bt = 0;
                exact_scan<T, LAYOUT>(p, su, kr64, line, r, r, r + weff - 1, best, bt);
                lt[r] = (OFF)bt;
            }
            if (g == 0) atomicAdd(&p.counters[CNT_FALLBACK], 1ull);
        }
        if (GS == 1) {
            // P1: every segment's first row scans the whole window
            if (work && s0 < s1)
                lt[s0] = (OFF)screened_row<T, LAYOUT>(p, su, lfx + s0, lk, kr64, line, s0, 0, weff - 1,
                                                                thr_add, rescans);
            __syncthreads();
        } else {
            // P1: the GS lanes of a group share the whole-window scan of the
            // group's first row; partial minima merge by shuffles
            const int ch = (weff + GS - 1) / GS;
            const int tlo = o * ch, thi = min(tlo + ch, weff) - 1;
            const bool hp = work && rp < NR;
            int m1 = 0x7fffffff, m2 = 0x7fffffff, t1 = 0x7fffffff;
            if (hp) {
                const int *f = lfx + rp;
#pragma unroll 4
                for (int t = tlo; t <= thi; ++t) {
                    int c = f[t] + lk[t];
                    m2 = min(m2, max(m1, c));
                    t1 = (c < m1) ? t : t1;
                    m1 = min(m1, c);
                }
            }
            for (int w = 1; w < GS; w <<= 1) {
                int om1 = __shfl_xor_sync(0xffffffffu, m1, w);
                int om2 = __shfl_xor_sync(0xffffffffu, m2, w);
                int ot1 = __shfl_xor_sync(0xffffffffu, t1, w);
                int nm2 = min(max(m1, om1), min(m2, om2));
                if (om1 < m1 || (om1 == m1 && ot1 < t1)) { m1 = om1; t1 = ot1; }
                m2 = nm2;
            }
            const int thr = hp ? m1 + thr_add : 0;
            const bool need = hp && !(m2 > thr);
            int tpiv = t1;
            if (__any_sync(0xffffffffu, need)) {
                Key2 bk = key2_max();
                int bt = 0x7fffffff;
                if (need) {
                    const int *f = lfx + rp;
                    for (int t = tlo; t <= thi; ++t) {
                        if (f[t] + lk[t] <= thr) {
                            int pos = wrapN(rp + t + p.hoff, N);
                            const Key2 key = key2(__dadd_rn(widen(su[uidx<LAYOUT>(p, line, pos)]), kr64[t]));
                            if (key2_less(key, bk)) { bk = key; bt = t; }
                        }
                    }
                }
                for (int w = 1; w < GS; w <<= 1) {
                    const Key2 ok = key2_shfl_xor(bk, w);
                    const int ot = __shfl_xor_sync(0xffffffffu, bt, w);
                    if (key2_less(ok, bk) || (key2_eq(ok, bk) && ot < bt)) { bk = ok; bt = ot; }
                }
                if (need) tpiv = bt;
                if (need && o == 0) ++rescans;
            }
            if (hp && o == 0) lt[rp] = (OFF)tpiv;
            __syncthreads();
            // P2: the other segments' first rows, bracketed by the argmins of
            // this group's and the next group's pivot rows (about GS * S
            // offsets away from shocks; wider brackets go to the warp)
            {
                const bool has = work && o != 0 && s0 < s1;
                int lo = 0, hi = 0;
                if (has) {
                    const int jl = rp + lt[rp];
                    const int rn = min((g - o + GS) * S, NR);
                    const int jr = (rn < NR) ? rn + lt[rn] : N + lt[0];
                    lo = max(jl - s0, 0);
                    hi = min(jr - s0, weff - 1);
                    if (lo > hi) { lo = 0; hi = weff - 1; }   // never for a Monge matrix
                }
                const int t = row_or_offload<T, LAYOUT>(p, su, fx, kfx, kr64, lsafe, s0, lo, hi, thr_add, has,
                                                        p.wide_mul * GS * S + p.wide_add, rescans);
                if (has) lt[s0] = (OFF)t;
            }
            __syncthreads();
        }
        // P3: the rest of each segment by divide and conquer; right
        // bracket: the next segment's first row, or the first row shifted by
        // one period
        {
            // every lane walks the block-uniform segment length S (rows past
            // its segment's end are predicated off)
            const bool dc = work && s1 - s0 >= 2;
            const int jnext = dc ? ((s1 < NR) ? (s1 + lt[s1]) : (N + lt[0])) : 0;
            const int nr = s1 - s0;
            int step = 1;
            while (step * 2 < S) step *= 2;
            for (; step >= 1; step >>= 1) {
                for (int rr = step; rr < S; rr += 2 * step) {
                    const bool has = dc && rr < nr;
                    const int r = s0 + rr;
                    int tlo = 0, thi = 0;
                    if (has) {
                        const int jl = (r - step) + lt[r - step];
                        const int qq = r + step;
                        const int jr = (qq < s1) ? qq + lt[qq] : jnext;
                        tlo = max(jl - r, 0);
                        thi = min(jr - r, weff - 1);
                        if (tlo > thi) { tlo = 0; thi = weff - 1; }   // never for a Monge matrix
                    }
                    const int t = row_or_offload<T, LAYOUT>(p, su, fx, kfx, kr64, lsafe, r, tlo, thi, thr_add, has,
                                                            p.wide_mul * (2 * step + 1) + p.wide_add, rescans);
                    if (has) lt[r] = (OFF)t;
                }
            }
        }
        {
            const int wr = __reduce_add_sync(0xffffffffu, rescans);
            if (lane == 0 && wr) atomicAdd(&p.counters[CNT_RESCAN], (unsigned long long)wr);
        }
        if (LAYOUT == LAYOUT_CONTIG) {
            // Every row's argmin was found by a lane of the warp that owns the
            // row's segment (divide and conquer, offload and fallback lines all
            // stay inside the warp after P2), so each warp writes its own rows
            // back as soon as it is done: no block barrier, coalesced stores.
            __syncwarp();
            T *dst = reinterpret_cast<T *>(p.dst);
            const int nl = (lpl >= 32) ? 1 : (32 >> p.log2lpl);     // lines held by this warp
            int edges = 0;
            for (int k = 0; k < nl; ++k) {
                int l = cl, r0 = 0, r1 = N;
                if (lpl >= 32) {
                    const int w0 = (g >> 5) << 5;                    // first lane of the warp in the line
                    r0 = min(w0 * S, NR);
                    r1 = min((w0 + 32) * S, NR);
                } else {
                    l = ((warp << 5) >> p.log2lpl) + k;
                }
                if (l >= tl.valid) continue;
                long long xb = tl.base + l * tl.lstride;
                if (p.vN) {
                    const RowBlock rb = row_block(p, (tile << p.log2C) + l);
                    xb = rb.base;
                    r1 = min(r1, rb.rows);
                }
                edges += write_rows_contig<T, OFF>(p, su + l * N, tt + l * p.tp, kr64, dst, xb, r0 + lane, r1, 32);
            }
            count_edges(p, edges);
            return;
        }
    } else {
        // ---- brute force: every row scanned by a whole warp, shuffle reduction
        const int line = warp / p.wpl;
        if (line < tl.valid) {
            OFF *lt = tt + line * p.tp;
            const int wl = warp - line * p.wpl;
            for (int r = wl; r < p.rows; r += p.wpl) {
                // running minimum as a Key2: the binary64 pipe only does the adds
                Key2 best = key2_max();
                int bt = 0;
                const int lo = r + lane, hi = r + weff - 1;
                if (lo <= hi) {
                    int pos = wrapN(lo + p.hoff, N);
                    for (int jj = lo; jj <= hi; jj += 32) {
                        const Key2 key = key2(__dadd_rn(widen(su[uidx<LAYOUT>(p, line, pos)]), kr64[jj - r]));
                        const bool less = key2_less(key, best);
                        best = less ? key : best;
                        bt = less ? jj - r : bt;
                        pos += 32;
                        while (pos >= N) pos -= N;
                    }
                }
                for (int o = 16; o; o >>= 1) {
                    const Key2 ok = key2_shfl_xor(best, o);
                    const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
                    if (key2_less(ok, best) || (key2_eq(ok, best) && ot < bt)) { best = ok; bt = ot; }
                }
                if (lane == 0) lt[r] = (OFF)bt;
            }
        }
    }
    __syncthreads();

    // ---- exact values, potential term, stores (coalesced order)
    T *dst = reinterpret_cast<T *>(p.dst);
    int edges = 0;
    if (LAYOUT == LAYOUT_CONTIG) {
        const int lanes = nthr >> p.log2C;              // threads per line
        const int l = tid / lanes, sub = tid - l * lanes;
        if (l < tl.valid) {
            long long xb = tl.base + l * tl.lstride;
            int rows = N;
            if (p.vN) {
                const RowBlock rb = row_block(p, (tile << p.log2C) + l);
                xb = rb.base;
                rows = rb.rows;
            }
            edges = write_rows_contig<T, OFF>(p, su + l * N, tt + l * p.tp, kr64, dst, xb, sub, rows, lanes);
        }
    } else {
        const int l = tid & (C - 1);
        if (l < tl.valid) {
            const int step = nthr >> p.log2C;
            const OFF *lt = tt + l * p.tp;
            const long long xb = tl.base + l;
            const long long xs = (long long)step * tl.pstride;
            int i = tid >> p.log2C;
            long long x = xb + (long long)i * tl.pstride;
            for (; i < N; i += step, x += xs) {
                const int t = lt[i];
                const int pos = wrapN(i + t + p.hoff, N);
                double m = __dadd_rn(widen(su[(pos << p.log2C) + l]), kr64[t]);
                if (p.hv) m = __dsub_rn(m, p.hv_scaled ? __dmul_rn(p.hscale, p.hv[x]) : p.hv[x]);
                store_val(dst + x, m);
                if (p.amin) p.amin[x] = p.dhi - t;
                edges += on_edge(t, p.weff);
            }
        }
    }
    count_edges(p, edges);
}

template <typename T, int LAYOUT, int ALGO, typename OFF>
__global__ void __launch_bounds__(1024) pass_kernel(const __grid_constant__ CUtensorMap tmap, PassParams p)
{
    const long long tile = blockIdx.x;
    if (tile >= p.ntiles) return;
    pass_tile<T, LAYOUT, ALGO, OFF>(&tmap, p, tile);
}

// Per-instance fields of a batched pass: one entry per grid of the batch.
struct BatchItem {
    CUtensorMap tmap;          // 3D TMA descriptor of this instance's u (strided lines)
    const void *src;
    void *dst;
    const double *hv;          // this instance's h*V (last axis) or nullptr
    const double *kr64;        // this instance's reversed kernel table
    double kmax, curv;
    int hoff, dhi;
    int use_tma, pad;
};

// One axis pass over many grids of the same launch shape: block b handles
// tile (b mod tiles) of instance (b / tiles).  Fields that differ between
// instances come from `items`; the rest of `p` is shared.
template <typename T, int LAYOUT, int ALGO>
__global__ void __launch_bounds__(1024) pass_kernel_batch(const BatchItem *__restrict__ items, PassParams p,
                                                          long long count)
{
    const long long inst = blockIdx.x / p.ntiles;
    const long long tile = blockIdx.x - inst * p.ntiles;
    if (inst >= count) return;
    const BatchItem *it = items + inst;
    PassParams q = p;
    q.src = it->src;
    q.dst = it->dst;
    q.hv = it->hv;
    q.kr64 = it->kr64;
    q.kmax = it->kmax;
    q.curv = it->curv;
    q.hoff = it->hoff;
    q.dhi = it->dhi;
    q.use_tma = it->use_tma;
    if (q.use_tma && LAYOUT == LAYOUT_STRIDED && threadIdx.x == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&it->tmap) : "memory");
    pass_tile<T, LAYOUT, ALGO>(&it->tmap, q, tile);
}

}  // namespace hjlo
