// FP64 pipe throughput probe (measurement support, not part of the method): the roofline of the
// FP64 kernels is the device's DFMA rate, which is measured here with independent FMA chains.
#include "mrom_internal.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

// Every thread runs kChains independent dependency chains x <- x * a + b for `iters` steps, so
// the FP64 pipe, not latency, bounds the rate.  The result goes to sink so nothing is removed.
__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s < 0.0) sink[0] = s;  // never true (every x stays near 1); keeps the chains live
}

}  // namespace

using namespace mrom;

extern "C" mrom_status mrom_fp64_peak(mrom_handle h, int32_t iters, double* tflops, double* ms) {
  if (!h || !tflops || iters < 1) return MROM_EINVAL;
  cudaSetDevice(h->device);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_probe_kernel, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int grid = h->num_sms * per_sm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a = 1 - 2^-30, b = 2^-30: x stays near 1, no overflow or denormals
  const double a = 1.0 - 9.313225746154785e-10, b = 9.313225746154785e-10;
  dfma_probe_kernel<<<grid, kThreads, 0, h->stream>>>(iters / 8 + 1, a, b, nullptr);  // warm-up
  cudaEventRecord(e0, h->stream);
  dfma_probe_kernel<<<grid, kThreads, 0, h->stream>>>(iters, a, b, nullptr);
  cudaEventRecord(e1, h->stream);
  h->launches += 2;
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_fp64_peak");
  const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return MROM_OK;
}
