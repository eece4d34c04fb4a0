// BF16 inference of the learned rank predictor (16 -> 64 ReLU -> 2; no counterpart in the
// paper), shared by the sparsification kernel and the stand-alone inference kernel.
#pragma once
#include "spalu_internal.h"

namespace spalu {

// BF16 inference of one feature row held in shared memory (needs >= 64 threads; every
// thread of the block calls it).  Hidden unit j and output k accumulate in float32 in a
// fixed order; products of bfloat16 values are exact in float32.
__device__ __forceinline__ void mlp_infer_block(const PredDev& P, const float* xf, float* zs, float* hid, float* out) {
  const int t = threadIdx.x;
  if (t < PRED_NFEAT)
    zs[t] = __bfloat162float(__float2bfloat16_rn(__fmul_rn(__fsub_rn(xf[t], P.mu[t]), P.isd[t])));
  __syncthreads();
  if (t < PRED_NHID) {
    float acc = __bfloat162float(P.wb[PRED_OFF_B1 + t]);
    for (int i = 0; i < PRED_NFEAT; ++i)
      acc = __fmaf_rn(__bfloat162float(P.wb[t * PRED_NFEAT + i]), zs[i], acc);
    hid[t] = __bfloat162float(__float2bfloat16_rn(fmaxf(acc, 0.0f)));
  }
  __syncthreads();
  if (t < PRED_NOUT) {
    float acc = __bfloat162float(P.wb[PRED_OFF_B2 + t]);
    for (int j = 0; j < PRED_NHID; ++j)
      acc = __fmaf_rn(__bfloat162float(P.wb[PRED_OFF_W2 + t * PRED_NHID + j]), hid[j], acc);
    out[t] = acc;
  }
  __syncthreads();
}

// One-pass sketch size from the network outputs (float32 arithmetic)
__device__ __forceinline__ int pred_sketch_size(const float* o, int nF, int e, int p, int h0, double margin) {
  const float o0 = fminf(fmaxf(o[0], -30.0f), 30.0f);
  const float o1 = fminf(fmaxf(o[1], -30.0f), 30.0f);
  const float m1 = 1.0f + (float)margin;
  const int hh = (int)ceilf(__fmul_rn(exp2f(o1), m1));
  const int kh = (int)ceilf(__fmul_rn(__fsub_rn(exp2f(o0), 1.0f), m1)) + p;
  int h = max(max(hh, kh), 1);
  return min(min(h, nF), max(h0, 2 * (e + p)));
}

}  // namespace spalu
