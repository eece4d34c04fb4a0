// Algorithmic work counts of the factorization (floating-point operations; a multiply-add
// counts 2), accumulated per level by the sparsify and merge kernels so that throughput can
// be stated against a roofline.  They follow the cost terms of Sec. 5.2 (the sampled
// interaction block, the pivoted QR of each ID, the interpolation matrix, the sparsifying
// transforms, the block eliminations); the exact sums are definitions of this library,
// counting the operations the method needs on the compressed sizes (not padded tiles):
//   lu(n)            LU with partial pivoting of order n: at step j, n-j-1 divisions and an
//                    (n-j-1)^2 rank-one update;
//   sketch(h, f, e)  G (h x f) times B_F (f x e);
//   qr(m, e, k)      k Householder steps on m x e: reflector norm 2 (m-j) and its application
//                    to the e-j-1 trailing columns 4 (m-j)(e-j-1);
//   interp(k, e)     T = R_11^{-1} R_12: e-k back substitutions of order k;
//   apply(e, k)      column and row operations of Eq. (UtALt) on the e x e own block;
//   elim(p, q)       p unknowns eliminated against q (Eq. (L^-1 A U^-1)): lu(p), W and Z
//                    (p^2 q each), Schur update 2 q^2 p.
#pragma once

namespace spalu {
namespace work {

__host__ __device__ inline unsigned long long lu(long long n) {
  return n > 0 ? (unsigned long long)(n * (n - 1) * (4 * n + 1) / 6) : 0ull;
}
__host__ __device__ inline unsigned long long sketch(long long h, long long f, long long e) {
  return (unsigned long long)(2 * h * f * e);
}
__host__ __device__ inline unsigned long long qr(long long m, long long e, long long k) {
  long long s = k < m ? k : m;
  s = s < e ? s : e;
  unsigned long long t = 0;
  for (long long j = 0; j < s; ++j) t += (unsigned long long)(2 * (m - j) + 4 * (m - j) * (e - j - 1));
  return t;
}
__host__ __device__ inline unsigned long long interp(long long k, long long e) {
  return (unsigned long long)(k * k * (e - k));
}
__host__ __device__ inline unsigned long long apply(long long e, long long k) {
  return (unsigned long long)(4 * e * k * (e - k));
}
__host__ __device__ inline unsigned long long elim(long long p, long long q) {
  return lu(p) + (unsigned long long)(2 * p * p * q + 2 * q * q * p);
}

}  // namespace work
}  // namespace spalu
