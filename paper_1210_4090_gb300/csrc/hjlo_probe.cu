// hjlo_probe.cu -- the binary64 add rate of the GPU (a measurement helper
// with no counterpart in the paper): the brute-force pass is bound by one
// binary64 add per window candidate, so its roofline needs the rate at which
// the device retires independent binary64 adds.
//
// Every thread runs 8 independent chains x_c = fl(x_c + y_c), unrolled so the
// adds of a chain are 8 apart in program order; the chains' results are
// combined and stored once so nothing is removed.  The grid is a multiple of
// the SM count with several CTAs per SM.
#include "hjlo_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) dadd_rate_kernel(long long iters, double seed, double *sink)
{
    double x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = seed * (double)(threadIdx.x + c + 1);
        y[c] = 0x1p-40 * (double)(c + 1);
    }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __dadd_rn(x[c], y[c]);
    }
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc = __dadd_rn(acc, x[c]);
    if (acc == 1.2345e300) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // never true for these inputs
}

}  // namespace

extern "C" hjlo_status hjlo_probe_fp64_add(int64_t iters, void *cuda_stream, double *adds_per_s)
{
    using namespace hjlo;
    clear_error();
    if (iters < 1 || iters > (1LL << 30) || !adds_per_s) return set_error(HJLO_EINVAL, "invalid probe arguments");
    DeviceFacts df;
    hjlo_status s = device_facts(df);
    if (s != HJLO_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = df.num_sms * 8, threads = 256;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_error(e, "cudaEventCreate");
    }
    // warm-up launch, then the timed one
    dadd_rate_kernel<<<blocks, threads, 0, st>>>(iters / 8 + 1, 1.0, nullptr);
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) dadd_rate_kernel<<<blocks, threads, 0, st>>>(iters, 1.0, nullptr);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_error(e, "binary64 add-rate probe");
    const double adds = (double)blocks * threads * (double)iters * kChains;
    *adds_per_s = (ms > 0.0f) ? adds / ((double)ms * 1e-3) : 0.0;
    return HJLO_OK;
}
