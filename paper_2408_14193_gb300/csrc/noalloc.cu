// Residual norms without any device allocation.
//
// spalu_refine measures ||b - A x|| / ||b|| with buffers it allocates on first use (the
// residual vectors and the partial sums of its reductions).  Some callers cannot let the
// library allocate at that point: hosts that hand every byte of device memory to their own
// pool (a framework's caching allocator, a serving runtime with a fixed memory budget) and
// forbid allocations from libraries after start-up, and processes already at the edge of
// device memory, where a new cudaMalloc would fail.  spalu_residual_noalloc serves them: the
// residual is formed on the fly and reduced through a fixed scratch array that lives in this
// file for the whole life of the process.
//
// The array's device address is looked up once per device and kept.  A cudaDeviceReset (or
// any reset of the primary context) unloads this module and makes that address stale, so
// the entry point must not be used across such a reset.
#include <mutex>

#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int NA_BLOCKS = 512;      // blocks of the first reduction pass
constexpr int NA_MAX_RHS = 64;      // largest nrhs one call accepts

// [NA_MAX_RHS][NA_BLOCKS][2] partial sums (||r||^2, ||b||^2), then NA_MAX_RHS results.
// Every call overwrites the partials it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_RHS * NA_BLOCKS * 2 + NA_MAX_RHS];

constexpr int NA_MAX_DEVICES = 64;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

__global__ void resid_partial_kernel(int n, const int* rowptr, const int* colind, const double* val,
                                     const double* B, const double* X, int ld, double* part) {
  __shared__ double red[2][32];
  const int c = blockIdx.y;
  double rr = 0.0, bb = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * X[colind[p] + (size_t)ld * c];
    const double b = B[i + (size_t)ld * c];
    const double r = b - acc;
    rr += r * r;
    bb += b * b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    double a = threadIdx.x < nw ? red[0][threadIdx.x] : 0.0;
    double b = threadIdx.x < nw ? red[1][threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      part[((size_t)c * gridDim.x + blockIdx.x) * 2] = a;
      part[((size_t)c * gridDim.x + blockIdx.x) * 2 + 1] = b;
    }
  }
}

__global__ void resid_final_kernel(const double* part, int nb, double* out) {
  const int c = blockIdx.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nb; ++k) {             // fixed order: the result is deterministic
      a += part[((size_t)c * nb + k) * 2];
      b += part[((size_t)c * nb + k) * 2 + 1];
    }
    out[c] = b > 0.0 ? sqrt(a / b) : 0.0;
  }
}

// Device address of the scratch array for the current device, looked up once per device.
double* scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}

}  // namespace

spalu_status residual_noalloc(int n, const int* rowptr, const int* colind, const double* val,
                              const double* B, const double* X, int nrhs, int ld, double* relres,
                              cudaStream_t s) {
  if (nrhs < 0 || nrhs > NA_MAX_RHS || !B || !X || !relres || ld < n) return SPALU_ERR_ARG;
  if (nrhs == 0) return SPALU_OK;
  double* scratch = scratch_for_current_device();
  if (!scratch) return SPALU_ERR_CUDA;
  double* part = scratch;
  double* out = scratch + (size_t)NA_MAX_RHS * NA_BLOCKS * 2;
  note_launch();
  resid_partial_kernel<<<dim3(NA_BLOCKS, nrhs), 256, 0, s>>>(n, rowptr, colind, val, B, X, ld, part);
  note_launch();
  resid_final_kernel<<<nrhs, 32, 0, s>>>(part, NA_BLOCKS, out);
  if (cudaGetLastError() != cudaSuccess) return SPALU_ERR_CUDA;
  if (cudaMemcpyAsync(relres, out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SPALU_ERR_CUDA;
  return SPALU_OK;
}

}  // namespace spalu
