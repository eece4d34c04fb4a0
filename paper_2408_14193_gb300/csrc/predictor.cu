// Learned rank predictor: training and inference kernels of the 16 -> 64 (ReLU) -> 2
// network that predicts a segment's ID rank k and one-pass sketch size h (the paper finds k
// adaptively, Sec. 4.2.3; this network is not in the paper).
//
//   * training in FP32: forward and backward over a batch (one warp per row, lane j owning
//     hidden units j and j + 32), per-block partial gradients, a deterministic reduction
//     over blocks, and Adam (beta1 0.9, beta2 0.999, eps 1e-8) which also refreshes the
//     bfloat16 inference copy;  loss = sum (o - y)^2 / (2 n) over the n rows of a batch;
//   * inference in BF16 (mlp_infer_block, shared with the sparsification kernel, serves the
//     stand-alone inference kernel here too);
//   * feature standardisation (mean, 1/std with std < 1e-6 -> 1) in FP64;
//   * export of the (features, targets) rows recorded by a factorization, in level and
//     segment order: y0 = log2(1 + k), y1 = log2(min(far rows, k + p)).
#include <cmath>

#include "pred_infer.cuh"
#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int GW = 8;                  // warps per block of the gradient kernel
constexpr int NACC = PRED_NPARAM + 1;  // gradient entries + the loss sum

// Per grid node u of the original matrix (features 5-10 of the segments): log d_u with
// d_u = |A_uu|, log(d_u / s_u) with s_u = sum_{j != u} |A_uj|, |sum_j A_uj| / d_u, and
// sum_{j!=u} |A_uj - A_ju| / sum_{j!=u} (|A_uj| + |A_ju|); computed in the precision of the
// value array (FP64, or its FP32 copy in the mixed path), stored as float.
template <typename V>
__global__ void node_stats_kernel(const int* __restrict__ rowptr, const int* __restrict__ colind,
                                  const V* __restrict__ val, int n, float4* __restrict__ out) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    V dd = V(0), off = V(0), rs = V(0), num = V(0), den = V(0);
    for (int p = rowptr[u]; p < rowptr[u + 1]; ++p) {
      const int j = colind[p];
      const V a = val[p];
      rs += a;
      if (j == u) { dd += a; continue; }
      off += fabs(a);
      V aj = V(0);
      for (int q = rowptr[j]; q < rowptr[j + 1]; ++q)
        if (colind[q] == u) aj += val[q];
      num += fabs(a - aj);
      den += fabs(a) + fabs(aj);
    }
    dd = fabs(dd);
    float4 r;
    if constexpr (sizeof(V) == 4) {     // FP32 copy of the values (mixed path): FP32 logs
      r.x = dd > 0.f ? logf(dd) : -690.7755f;              // log(1e-300) when dd vanishes
      r.y = (off > 0.f && dd > 0.f) ? logf(dd / off) : 0.f;
      r.z = dd > 0.f ? fabsf(rs) / dd : 0.f;
      r.w = den > 0.f ? num / den : 0.f;
    } else {
      r.x = (float)(dd > 0.0 ? log(dd) : log(1e-300));
      r.y = (float)((off > 0.0 && dd > 0.0) ? log(dd / off) : 0.0);
      r.z = (float)(dd > 0.0 ? fabs(rs) / dd : 0.0);
      r.w = (float)(den > 0.0 ? num / den : 0.0);
    }
    out[u] = r;
  }
}

__global__ void pred_fit_norm_kernel(const float* X, int n, PredDev* P) {
  __shared__ double red[32];
  const int col = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s += (double)X[(size_t)r * PRED_NFEAT + col];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double mean = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mean += red[w];
  mean /= n;
  __syncthreads();
  double v = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double dv = (double)X[(size_t)r * PRED_NFEAT + col] - mean;
    v += dv * dv;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double var = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) var += red[w];
    const double sd = sqrt(var / n);
    P->mu[col] = (float)mean;
    P->isd[col] = sd < 1e-6 ? 1.0f : (float)(1.0 / sd);
  }
}

// Forward + backward of rows [r0, r0 + nb); partial[blockIdx.x][*] receives this block's
// gradient sums (scaled by inv_n) and its sum of squared residuals.
__global__ void __launch_bounds__(GW * 32) pred_grad_kernel(const float* __restrict__ params,
                                                             const PredDev* __restrict__ P,
                                                             const float* __restrict__ X,
                                                             const float* __restrict__ Y, int r0, int nb,
                                                             float inv_n, float* __restrict__ partial) {
  __shared__ float acc[NACC];
  __shared__ float mu[PRED_NFEAT], isd[PRED_NFEAT];
  for (int i = threadIdx.x; i < NACC; i += blockDim.x) acc[i] = 0.0f;
  if (threadIdx.x < PRED_NFEAT) { mu[threadIdx.x] = P->mu[threadIdx.x]; isd[threadIdx.x] = P->isd[threadIdx.x]; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j0 = lane, j1 = lane + 32;
  float w1a[PRED_NFEAT], w1b[PRED_NFEAT], g1a[PRED_NFEAT], g1b[PRED_NFEAT];
#pragma unroll
  for (int i = 0; i < PRED_NFEAT; ++i) {
    w1a[i] = params[j0 * PRED_NFEAT + i];
    w1b[i] = params[j1 * PRED_NFEAT + i];
    g1a[i] = 0.0f;
    g1b[i] = 0.0f;
  }
  const float b1a = params[PRED_OFF_B1 + j0], b1b = params[PRED_OFF_B1 + j1];
  const float w20a = params[PRED_OFF_W2 + j0], w20b = params[PRED_OFF_W2 + j1];
  const float w21a = params[PRED_OFF_W2 + PRED_NHID + j0], w21b = params[PRED_OFF_W2 + PRED_NHID + j1];
  const float b20 = params[PRED_OFF_B2], b21 = params[PRED_OFF_B2 + 1];
  float gb1a = 0.f, gb1b = 0.f, g20a = 0.f, g20b = 0.f, g21a = 0.f, g21b = 0.f, gb20 = 0.f, gb21 = 0.f, lsum = 0.f;
  for (int s = blockIdx.x * GW + warp; s < nb; s += gridDim.x * GW) {
    const float* x = X + (size_t)(r0 + s) * PRED_NFEAT;
    float z[PRED_NFEAT];
#pragma unroll
    for (int i = 0; i < PRED_NFEAT; ++i) z[i] = (x[i] - mu[i]) * isd[i];
    float aa = b1a, ab = b1b;
#pragma unroll
    for (int i = 0; i < PRED_NFEAT; ++i) { aa = fmaf(w1a[i], z[i], aa); ab = fmaf(w1b[i], z[i], ab); }
    const float ha = fmaxf(aa, 0.f), hb = fmaxf(ab, 0.f);
    float o0 = w20a * ha + w20b * hb, o1 = w21a * ha + w21b * hb;
    for (int o = 16; o > 0; o >>= 1) {
      o0 += __shfl_xor_sync(0xffffffffu, o0, o);
      o1 += __shfl_xor_sync(0xffffffffu, o1, o);
    }
    const float r0v = (o0 + b20) - Y[(size_t)(r0 + s) * 2];
    const float r1v = (o1 + b21) - Y[(size_t)(r0 + s) * 2 + 1];
    const float d0 = r0v * inv_n, d1 = r1v * inv_n;
    if (lane == 0) { lsum += r0v * r0v + r1v * r1v; gb20 += d0; gb21 += d1; }
    g20a += d0 * ha; g20b += d0 * hb;
    g21a += d1 * ha; g21b += d1 * hb;
    const float da = aa > 0.f ? w20a * d0 + w21a * d1 : 0.f;
    const float db = ab > 0.f ? w20b * d0 + w21b * d1 : 0.f;
    gb1a += da; gb1b += db;
#pragma unroll
    for (int i = 0; i < PRED_NFEAT; ++i) { g1a[i] = fmaf(da, z[i], g1a[i]); g1b[i] = fmaf(db, z[i], g1b[i]); }
  }
#pragma unroll
  for (int i = 0; i < PRED_NFEAT; ++i) {
    atomicAdd(&acc[j0 * PRED_NFEAT + i], g1a[i]);
    atomicAdd(&acc[j1 * PRED_NFEAT + i], g1b[i]);
  }
  atomicAdd(&acc[PRED_OFF_B1 + j0], gb1a);
  atomicAdd(&acc[PRED_OFF_B1 + j1], gb1b);
  atomicAdd(&acc[PRED_OFF_W2 + j0], g20a);
  atomicAdd(&acc[PRED_OFF_W2 + j1], g20b);
  atomicAdd(&acc[PRED_OFF_W2 + PRED_NHID + j0], g21a);
  atomicAdd(&acc[PRED_OFF_W2 + PRED_NHID + j1], g21b);
  if (lane == 0) {
    atomicAdd(&acc[PRED_OFF_B2], gb20);
    atomicAdd(&acc[PRED_OFF_B2 + 1], gb21);
    atomicAdd(&acc[PRED_NPARAM], lsum);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NACC; i += blockDim.x) partial[(size_t)blockIdx.x * NACC + i] = acc[i];
}

// grad[i] = sum over blocks b (in order) of partial[b][i]; also advances the Adam step
__global__ void pred_reduce_kernel(const float* __restrict__ partial, int nblk, float* __restrict__ grad,
                                   int* step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && step) *step += 1;
  if (i >= NACC) return;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * NACC + i];
  grad[i] = s;
}

__global__ void pred_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                 const float* __restrict__ grad, const int* step, float lr, PredDev* P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= PRED_NPARAM) return;
  const int t = *step;
  const double bc1 = 1.0 - pow(0.9, (double)t), bc2 = 1.0 - pow(0.999, (double)t);
  const float g = grad[i];
  const float mi = 0.9f * m[i] + 0.1f * g;
  const float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  const float mh = (float)(mi / bc1), vh = (float)(vi / bc2);
  const float p = params[i] - lr * mh / (sqrtf(vh) + 1e-8f);
  params[i] = p;
  P->wb[i] = __float2bfloat16_rn(p);
}

__global__ void pred_to_bf16_kernel(const float* __restrict__ params, PredDev* P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < PRED_NPARAM) P->wb[i] = __float2bfloat16_rn(params[i]);
}

__global__ void pred_infer_kernel(const PredDev* __restrict__ P, const float* __restrict__ X, int n,
                                  float* __restrict__ out) {
  __shared__ float xf[PRED_NFEAT], zs[PRED_NFEAT], hid[PRED_NHID], o[PRED_NOUT];
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    if (threadIdx.x < PRED_NFEAT) xf[threadIdx.x] = X[(size_t)r * PRED_NFEAT + threadIdx.x];
    __syncthreads();
    mlp_infer_block(*P, xf, zs, hid, o);
    if (threadIdx.x < PRED_NOUT) out[(size_t)r * PRED_NOUT + threadIdx.x] = o[threadIdx.x];
    __syncthreads();
  }
}

// Ordered compaction of the recorded rows of one level (one block of 1024 threads): rows
// land at *count + (rank among the valid segments of this level), segment order kept.
__global__ void __launch_bounds__(1024) pred_export_kernel(const float* __restrict__ feat, const int* __restrict__ tgt,
                                                           int nseg, int p, float* __restrict__ X,
                                                           float* __restrict__ Y, int cap, int* count) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = *count;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s0 = 0; s0 < nseg; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const bool valid = s < nseg && tgt[(size_t)s * 4 + 2] != 0;
    const unsigned b = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 32; ++w) { if (w < warp) before += wsum[w]; total += wsum[w]; }
    const int pos = base + before + __popc(b & ((1u << lane) - 1u));
    if (valid && pos < cap) {
      for (int i = 0; i < PRED_NFEAT; ++i) X[(size_t)pos * PRED_NFEAT + i] = feat[(size_t)s * PRED_NFEAT + i];
      const int k = tgt[(size_t)s * 4], nF = tgt[(size_t)s * 4 + 1];
      const int hs = max(1, min(nF, k + p));
      Y[(size_t)pos * 2] = (float)log2(1.0 + k);
      Y[(size_t)pos * 2 + 1] = (float)log2((double)hs);
    }
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

}  // namespace

int pred_grad_blocks(int nb) {
  int g = (nb + GW * 8 - 1) / (GW * 8);
  return g < 1 ? 1 : (g > PRED_MAXBLK ? PRED_MAXBLK : g);
}

void launch_node_stats(const int* rowptr, const int* colind, const double* val, const float* fval, int n,
                       float4* out, cudaStream_t s) {
  if (n <= 0) return;
  int g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  note_launch();
  if (fval) node_stats_kernel<float><<<g, 256, 0, s>>>(rowptr, colind, fval, n, out);
  else node_stats_kernel<double><<<g, 256, 0, s>>>(rowptr, colind, val, n, out);
}

void launch_pred_fit_norm(const float* X, int n, PredDev* P, cudaStream_t s) {
  note_launch();
  pred_fit_norm_kernel<<<PRED_NFEAT, 256, 0, s>>>(X, n, P);
}

void launch_pred_grad(const float* params, const PredDev* P, const float* X, const float* Y, int r0, int nb,
                      float* partial, float* grad, int* step, cudaStream_t s) {
  const int g = pred_grad_blocks(nb);
  note_launch();
  pred_grad_kernel<<<g, GW * 32, 0, s>>>(params, P, X, Y, r0, nb, 1.0f / nb, partial);
  note_launch();
  pred_reduce_kernel<<<(NACC + 255) / 256, 256, 0, s>>>(partial, g, grad, step);
}

void launch_pred_adam(float* params, float* m, float* v, const float* grad, const int* step, float lr,
                      PredDev* P, cudaStream_t s) {
  note_launch();
  pred_adam_kernel<<<(PRED_NPARAM + 255) / 256, 256, 0, s>>>(params, m, v, grad, step, lr, P);
}

void launch_pred_to_bf16(const float* params, PredDev* P, cudaStream_t s) {
  note_launch();
  pred_to_bf16_kernel<<<(PRED_NPARAM + 255) / 256, 256, 0, s>>>(params, P);
}

void launch_pred_infer(const PredDev* P, const float* X, int n, float* out, cudaStream_t s) {
  if (n <= 0) return;
  note_launch();
  pred_infer_kernel<<<n < 4096 ? n : 4096, 64, 0, s>>>(P, X, n, out);
}

void launch_pred_export(const float* feat, const int* tgt, int nseg, int p, float* X, float* Y, int cap,
                        int* count, cudaStream_t s) {
  if (nseg <= 0) return;
  note_launch();
  pred_export_kernel<<<1, 1024, 0, s>>>(feat, tgt, nseg, p, X, Y, cap, count);
}

}  // namespace spalu
