// Measurement utility: the FP64 fused multiply-add rate of the device, the
// denominator of the roofline of the FP64 step (which is bound by the FP64
// units, not by HBM).  Every thread runs kChains independent chains
// a <- a * b + c of `iters` FMAs each, so that the pipe never waits on a
// dependency; the caller times the launch with CUDA events on `stream`.
#include <cuda_runtime.h>

#include "fdlbm.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma(int iters, double b, double c, double *out)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // a store the compiler cannot drop, taken (almost) never
    if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

extern "C" {

fdlbm_status fdlbm_probe_fp64_fma(int blocks, int iters, double *out, void *stream,
                                  double *flop)
{
    if (blocks < 1 || iters < 1 || !out) return FDLBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // b slightly below 1 and c small keep the chains finite for any iters
    k_fp64_fma<<<blocks, kThreads, 0, s>>>(iters, 0.9999999, 1e-7, out);
    if (flop) *flop = 2.0 * kChains * (double)iters * kThreads * (double)blocks;
    return cudaGetLastError() == cudaSuccess ? FDLBM_OK : FDLBM_ECUDA;
}

}  // extern "C"
