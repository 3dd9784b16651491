// hjlo_decomp.cuh -- device helpers shared by the two decomposition passes
// (one CTA per line, and a period cut across CTAs).
#pragma once

namespace hjlo {

// Number of kernel slopes strictly below rho (the slopes increase).  The
// slopes are held as order-preserving keys (kh, kl: dkey32's words, which
// compare as the finite values do, -0 with +0), so the search uses 32-bit
// integer compares and leaves the binary64 pipe to the candidates' adds.
__device__ __forceinline__ int below(const unsigned *kh, const unsigned *kl, int n, double rho)
{
    unsigned h, l;
    dkey32(rho, h, l);
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const unsigned a = kh[mid];
        if (a < h || (a == h && kl[mid] < l)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace hjlo
