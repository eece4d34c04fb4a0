// Arithmetic-throughput probe of the CUDA cores (a diagnostic, not part of the method): the
// FP64 and FP32 FMA rates that bound the factorization's small dense kernels, measured on
// the device the library runs on instead of derived from unit counts and clocks.
#include <algorithm>

#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int PR_CHAINS = 8;      // independent FMA chains per thread (hide the FMA latency)
constexpr int PR_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PR_THREADS) fma_probe_kernel(T* out, int iters, T a, T b, int store) {
  T x[PR_CHAINS];
#pragma unroll
  for (int i = 0; i < PR_CHAINS; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PR_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < PR_CHAINS; ++i) s += x[i];
  if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // store = 0: kept only as a use
}

template <typename T>
spalu_status run(int iters, double* flops, cudaStream_t s) {
  const int blocks = sm_count() * 8;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SPALU_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SPALU_ERR_CUDA; }
  double best = 0.0;
  spalu_status st = SPALU_OK;
  for (int rep = 0; rep < 4 && st == SPALU_OK; ++rep) {      // first launch warms up
    cudaEventRecord(e0, s);
    note_launch();
    fma_probe_kernel<T><<<blocks, PR_THREADS, 0, s>>>(nullptr, iters, T(0.999), T(1e-4), 0);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = SPALU_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * PR_CHAINS * (double)iters * blocks * PR_THREADS / (ms * 1e-3);
    if (rep > 0) best = std::max(best, f);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops = best;
  return st;
}

}  // namespace
}  // namespace spalu

extern "C" spalu_status spalu_measure_fma_peak(int precision, double* flops, spalu_stream_t stream) {
  if (!flops || (precision != 0 && precision != 1)) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == 0 ? spalu::run<double>(1 << 12, flops, s) : spalu::run<float>(1 << 16, flops, s);
}
