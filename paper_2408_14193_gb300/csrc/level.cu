// One level of the spaLU factorization (Sec. 4.3, Alg. 2, l = L..1) and its solve.
//
// Data model: the Schur complement A^(l) is the sum over the depth-l boxes of dense
// "frontal" blocks over each box's boundary unknowns (its four sides and corners); a side
// shared by two boxes is one segment.  Per level:
//   sparsify_kernel   one CTA per segment: hybrid sketch Y = [B_N; G B_F / sqrt(h)] of
//                     B = [A_{n,i}; A_{i,n}^T] (Eqs. (Phi), (ID [A_ni; A_in])), column-pivoted
//                     QR and T = R_1^{-1} R_2 (Eqs. (RRQR 1), (RRQR 2)), the transform of the
//                     segment's own block by U_t, L_t (Eq. (UtALt)), LU of the remainder and
//                     its Schur update onto the skeleton (Eq. (L^-1 * A * U^-1)).
//   merge_*_kernels   one parent (depth l-1 box) at a time: extend-add of its two children
//                     restricted to skeletons (the permutation E_(l)), LU of the level-l
//                     separator's skeleton block and the Schur update onto the parent's
//                     boundary, which is the parent's frontal for level l-1.
// The neighbour couplings of a remainder are dropped (they are O(eps) after the
// transform), and the couplings between skeletons are unchanged by the transforms, so only
// the segment's own diagonal block is transformed.
//
// Every kernel is templated on the working precision T (double; float in mixed mode).
// Column norms, pivots and the truncation test of the column-pivoted QR stay in FP64.
// GB300 runs FP64 at 2 FMA per clock per SM, so per-column scalars (Householder coefficients,
// norm downdates) are computed once for 32 columns at a time (one lane per column) and
// divisions are replaced by stored reciprocals.
#include <cfloat>
#include <cmath>

#include "pred_infer.cuh"
#include "spalu_internal.h"
#include "work.cuh"

namespace spalu {
namespace {

constexpr int NEAR_MAX = 16;      // near unknowns per segment (the geometry gives <= 10)
constexpr int RUN_MAX = 16;
constexpr int SK_CHUNK = 16;      // far unknowns per chunk of the sketch product (at least)
constexpr int SK_CHUNK_MAX = 64;  // ... and at most, where the shared-memory budget has room
constexpr int NW = 8;             // warps per CTA of the sparsify kernel (segments with e > 32)
constexpr int NW_SMALL = 2;       // ... and for levels whose segments have at most 16 unknowns
constexpr double TIE_RTOL = 1e-12;
constexpr int RSTAGE = 96;        // triangular blocks up to this order are staged in shared memory

// ------------------------------------------------------------ Philox4x32-10 (SC'11)
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Entries of the sampling matrix G for sketch rows 4 g .. 4 g + 3 of one far row: counter
// (g, node, 2l+t, sid), key = seed; the four output words give u1..u4 (odd multiples of
// 2^-24), and float32 Box-Muller turns each pair into two normals:
// z = {R1 cos(2 pi u2), R1 sin(2 pi u2), R2 cos(2 pi u4), R2 sin(2 pi u4)}, R = sqrt(-2 log u).
__device__ __forceinline__ void sketch_gauss4(unsigned long long seed, int l, int sid, int g, int node, int t,
                                              float (&z)[4]) {
  uint32_t c[4] = {(uint32_t)g, (uint32_t)node, (uint32_t)(2 * l + t), (uint32_t)sid};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
  float u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) u[i] = (float)(((c[i] >> 9) << 1) | 1u) * 0x1p-24f;
  const float r1 = sqrtf(-2.0f * logf(u[0])), r2 = sqrtf(-2.0f * logf(u[2]));
  const float a1 = 6.283185307179586f * u[1], a2 = 6.283185307179586f * u[3];
  z[0] = r1 * cosf(a1);
  z[1] = r1 * sinf(a1);
  z[2] = r2 * cosf(a2);
  z[3] = r2 * sinf(a2);
}

// ------------------------------------------------------------ neighbour runs of a segment
struct Run {
  int p1, p2, len, ref;   // positions in box 1 / box 2 (-1: absent), count, seg id or -2-node
};

struct SegCtx {
  int sid, e, b1, b2, s1, s2;   // boxes (b1 = lower/left owner) and position of the segment
  int horiz, line, lo, hi;      // geometric extent
  int nrun, nb;
  Run run[RUN_MAX];
};

__device__ void seg_context(const LevelDev& d, int sid, SegCtx& S) {
  const Geo g = d.g;
  int I1, J1, I2, J2;
  S.sid = sid;
  S.e = d.cnt[sid];
  if (sid < g.nh()) {
    int I = sid % g.bx, J = sid / g.bx + 1;
    I1 = I; J1 = J - 1; I2 = I; J2 = J;
    S.s1 = g.side_pos(SIDE_TOP);
    S.s2 = g.side_pos(SIDE_BOTTOM);
    S.horiz = 1;
    S.line = J * (g.h + 1) - 1;
    S.lo = I * (g.w + 1);
    S.hi = S.lo + g.w - 1;
  } else {
    int t = sid - g.nh();
    int I = t % (g.bx - 1) + 1, J = t / (g.bx - 1);
    I1 = I - 1; J1 = J; I2 = I; J2 = J;
    S.s1 = g.side_pos(SIDE_RIGHT);
    S.s2 = g.side_pos(SIDE_LEFT);
    S.horiz = 0;
    S.line = I * (g.w + 1) - 1;
    S.lo = J * (g.h + 1);
    S.hi = S.lo + g.h - 1;
  }
  S.b1 = I1 + g.bx * J1;
  S.b2 = I2 + g.bx * J2;
  const int skip1 = S.horiz ? SIDE_TOP : SIDE_RIGHT;
  const int skip2 = S.horiz ? SIDE_BOTTOM : SIDE_LEFT;
  int n = 0, nb = 0;
  for (int side = 0; side < 4; ++side) {
    if (side == skip1) continue;
    int sg = g.box_side(I1, J1, side);
    if (sg >= 0) { S.run[n] = {g.side_pos(side), -1, d.cnt[sg], sg}; nb += S.run[n].len; ++n; }
  }
  for (int side = 0; side < 4; ++side) {
    if (side == skip2) continue;
    int sg = g.box_side(I2, J2, side);
    if (sg >= 0) { S.run[n] = {-1, g.side_pos(side), d.cnt[sg], sg}; nb += S.run[n].len; ++n; }
  }
  // shared corners: horizontal (b1 below b2): b1.TL = b2.BL, b1.TR = b2.BR;
  //                 vertical (b1 left of b2):  b1.BR = b2.BL, b1.TR = b2.TL
  for (int c = 0; c < 4; ++c) {
    int cid = g.box_corner(I1, J1, c);
    if (cid < 0) continue;
    int c2 = -1;
    if (S.horiz) { if (c == C_TL) c2 = C_BL; else if (c == C_TR) c2 = C_BR; }
    else { if (c == C_BR) c2 = C_BL; else if (c == C_TR) c2 = C_TL; }
    S.run[n] = {g.corner_pos(c), c2 >= 0 ? g.corner_pos(c2) : -1, 1, -2 - g.junction_node(cid, d.nx)};
    ++nb; ++n;
  }
  for (int c = 0; c < 4; ++c) {
    int cid = g.box_corner(I2, J2, c);
    if (cid < 0) continue;
    bool shared = S.horiz ? (c == C_BL || c == C_BR) : (c == C_BL || c == C_TL);
    if (shared) continue;
    S.run[n] = {-1, g.corner_pos(c), 1, -2 - g.junction_node(cid, d.nx)};
    ++nb; ++n;
  }
  S.nrun = n;
  S.nb = nb;
}

__device__ __forceinline__ void locate(const SegCtx& S, int f, int& r, int& i) {
  r = 0;
  while (f >= S.run[r].len) { f -= S.run[r].len; ++r; }
  i = f;
}

__device__ __forceinline__ int run_node(const LevelDev& d, const Run& R, int i) {
  return R.ref >= 0 ? d.nodes[(size_t)R.ref * d.capS + i] : (-2 - R.ref);
}

__device__ __forceinline__ int cheb(const SegCtx& S, int node, int nx) {
  int x = node % nx, y = node / nx;
  int a = S.horiz ? y : x, b = S.horiz ? x : y;
  int da = abs(a - S.line);
  int db = max(0, max(S.lo - b, b - S.hi));
  return max(da, db);
}

// B entry for neighbour (run R, element i), half t (0: A[v, s_c], 1: A[s_c, v]), column c
template <typename T>
__device__ __forceinline__ T bval(const LevelDev& d, const SegCtx& S, const T* F1, const T* F2,
                                  const Run& R, int i, int t, int c) {
  const size_t ld = d.ldF;
  T v = T(0);
  if (R.p1 >= 0) {
    int p = R.p1 + i;
    v += t == 0 ? F1[p + ld * (S.s1 + c)] : F1[(S.s1 + c) + ld * p];
  }
  if (R.p2 >= 0) {
    int p = R.p2 + i;
    v += t == 0 ? F2[p + ld * (S.s2 + c)] : F2[(S.s2 + c) + ld * p];
  }
  return v;
}

// Neighbour table of a segment (shared memory, built once per segment when it has at most
// NB_MAX neighbours): grid node, positions in the frontal blocks of box 1 / box 2 (-1 when
// absent) and the near flag of neighbour f.  Without the table the same values come from the
// runs.
constexpr int NB_MAX = 512;
struct NbrTab {
  const int* node;
  const short* p1;
  const short* p2;
  const unsigned char* nearf;
  bool on;
};
struct Nbr {
  int node, p1, p2;
  bool nearf;
};

__device__ __forceinline__ Nbr nbr_get(const LevelDev& d, const SegCtx& S, const NbrTab& tb, int f) {
  Nbr q;
  if (tb.on) {
    q.node = tb.node[f];
    q.p1 = tb.p1[f];
    q.p2 = tb.p2[f];
    q.nearf = tb.nearf[f] != 0;
  } else {
    int r, i;
    locate(S, f, r, i);
    const Run& R = S.run[r];
    q.node = run_node(d, R, i);
    q.p1 = R.p1 >= 0 ? R.p1 + i : -1;
    q.p2 = R.p2 >= 0 ? R.p2 + i : -1;
    q.nearf = cheb(S, q.node, d.nx) <= d.near_radius;
  }
  return q;
}

// B entry of neighbour q, half t, column c (as bval)
template <typename T>
__device__ __forceinline__ T bval_q(const LevelDev& d, const SegCtx& S, const T* F1, const T* F2, const Nbr& q,
                                    int t, int c) {
  const size_t ld = d.ldF;
  T v = T(0);
  if (q.p1 >= 0) v += t == 0 ? F1[q.p1 + ld * (S.s1 + c)] : F1[(S.s1 + c) + ld * q.p1];
  if (q.p2 >= 0) v += t == 0 ? F2[q.p2 + ld * (S.s2 + c)] : F2[(S.s2 + c) + ld * q.p2];
  return v;
}

// non-negative doubles order like their bit patterns
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// ------------------------------------------------------------ column-pivoted QR
// Businger-Golub Householder QR with column pivoting of Y (m x e, ld ldy, precision T),
// stopped at the first step i with |R_ii| <= eps |R_00|.  Squared column norms are tracked
// and downdated in FP64 — s <- s - R_ij^2, recomputed when s <= sqrt(eps_64) s_ref (the
// Drmac-Bujanovic guard written for squared norms: no division or square root per column and
// step) — and the pivot is chosen from them; the Householder products and their column sums
// run in T.  perm receives the column order; on exit the first k rows of Y hold [R_1 R_2] in
// the permuted order.  Returns k.  The factorization also stops after kstop steps (returning
// kstop): a caller that only needs to know whether k exceeds kstop - 1 skips the rest.
// sh: >= NWT*32 + 3*64 doubles of shared scratch; flags: >= e.  NWT = warps of the CTA.
template <typename T, int NWT>
__device__ int block_cpqr(T* Y, int ldy, int m, int e, double eps, int* perm, double* vn1,
                          double* vn2, double* sh, int* flags, int* shi, int kstop) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* part = reinterpret_cast<T*>(sh);                   // [NWT][32] partial dots
  T* coef = reinterpret_cast<T*>(sh + NWT * 32);         // [64]
  double* scal = sh + NWT * 32 + 64;                     // alpha, v0, c2, normx
  for (int j = threadIdx.x; j < e; j += blockDim.x) perm[j] = j;
  if (m == 0 || e == 0) { __syncthreads(); return 0; }
  // initial column norms (one warp per column)
  for (int j = warp; j < e; j += NWT) {
    T s = T(0);
    for (int r = lane; r < m; r += 32) { T v = Y[r + (size_t)ldy * j]; s += v * v; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      vn1[j] = (double)s;
      vn2[j] = (double)s;
    }
  }
  __syncthreads();
  const double tol3z = sqrt(DBL_EPSILON);
  const double tie = (1.0 - TIE_RTOL) * (1.0 - TIE_RTOL);   // on squared norms
  const int kmax = min(min(m, e), kstop);
  double ref = 0.0;
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    // the per-step scalar tasks rotate over the warps (and CTAs), so that the FP64 work of
    // co-resident CTAs does not pile up on one SM sub-partition
    const int wp = (i + blockIdx.x) % NWT, wh = (i + 1 + blockIdx.x) % NWT;
    const int wr = (i + 2 + blockIdx.x) % NWT, wd = (i + 3 + blockIdx.x) % NWT;
    if (warp == wp) {         // pivot: largest norm, near-ties -> lowest index
      long long mx = -1;
      for (int j = i + lane; j < e; j += 32) mx = max(mx, dbits(vn1[j]));
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const long long thr = dbits(__longlong_as_double(mx) * tie);
      int best = e;
      for (int j = i + lane; j < e; j += 32)
        if (dbits(vn1[j]) >= thr && j < best) best = j;
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (lane == 0) shi[0] = best;
    }
    __syncthreads();
    const int p = shi[0];
    if (p != i) {
      for (int r = threadIdx.x; r < m; r += blockDim.x) {
        T a = Y[r + (size_t)ldy * i];
        Y[r + (size_t)ldy * i] = Y[r + (size_t)ldy * p];
        Y[r + (size_t)ldy * p] = a;
      }
      if (threadIdx.x == 0) {
        int t = perm[i]; perm[i] = perm[p]; perm[p] = t;
        double a = vn1[i]; vn1[i] = vn1[p]; vn1[p] = a;
        a = vn2[i]; vn2[i] = vn2[p]; vn2[p] = a;
      }
      __syncthreads();
    }
    // Householder vector of column i (scalars by one thread)
    if (warp == wh) {
      T s = T(0);
      for (int r = i + lane; r < m; r += 32) { T v = Y[r + (size_t)ldy * i]; s += v * v; }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const T normx = sqrt(s);
        const T x0 = Y[i + (size_t)ldy * i];
        const T alpha = x0 >= T(0) ? -normx : normx;
        const T v0 = x0 - alpha;
        const T vv = v0 * v0 + (s - x0 * x0);
        scal[0] = (double)alpha;
        scal[1] = (double)v0;
        scal[2] = vv > T(0) ? (double)(T(2) / vv) : 0.0;
        scal[3] = (double)normx;
      }
    }
    __syncthreads();
    const double normx = scal[3];
    if (i == 0) ref = normx;
    if (ref == 0.0) { k = 0; break; }
    if (normx <= eps * ref || normx == 0.0) { k = i; break; }
    const T v0 = (T)scal[1];
    const T c2 = (T)scal[2];
    const int ncol = e - i - 1;
    // dots of v with the trailing columns (lanes over columns, warps over rows), then update
    for (int cg = 0; cg < ncol; cg += 32) {
      const int j = i + 1 + cg + lane;
      T acc = T(0);
      if (j < e) {
        const T* yj = Y + (size_t)ldy * j;
        const T* yi = Y + (size_t)ldy * i;
        if (warp == 0) acc = v0 * yj[i];
        for (int r = i + 1 + warp; r < m; r += NWT) acc += yi[r] * yj[r];
      }
      part[warp * 32 + lane] = acc;
      __syncthreads();
      if (warp == wr && j < e) {
        T s = T(0);
        for (int w = 0; w < NWT; ++w) s += part[w * 32 + lane];
        coef[lane] = s * c2;
      }
      __syncthreads();
      if (j < e) {
        const T cj = coef[lane];
        T* yj = Y + (size_t)ldy * j;
        const T* yi = Y + (size_t)ldy * i;
        if (warp == 0) yj[i] -= cj * v0;
        for (int r = i + 1 + warp; r < m; r += NWT) yj[r] -= cj * yi[r];
      }
      __syncthreads();
    }
    // FP64 downdates of the squared norms, one lane per column; guarded recomputations after
    if (warp == wd) {
      for (int j = i + 1 + lane; j < e; j += 32) {
        const double sq = vn1[j];
        int fl = 0;
        if (sq != 0.0) {
          const double rij = (double)Y[i + (size_t)ldy * j];
          const double sn = fmax(sq - rij * rij, 0.0);
          if (sn <= tol3z * vn2[j]) fl = 1;
          else vn1[j] = sn;
        }
        flags[j] = fl;
      }
    }
    __syncthreads();
    for (int j = i + 1 + warp; j < e; j += NWT) {
      if (!flags[j]) continue;
      double s = 0.0;
      for (int r = i + 1 + lane; r < m; r += 32) { double v = (double)Y[r + (size_t)ldy * j]; s += v * v; }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        vn1[j] = s;
        vn2[j] = s;
      }
    }
    if (threadIdx.x == 0) Y[i + (size_t)ldy * i] = (T)scal[0];
    __syncthreads();
  }
  __syncthreads();
  return k;
}

// T (k x (e-k), ld ldt) = R_1^{-1} R_2 from the R held in Y (ld ldy); rinv: >= k scratch
template <typename T>
__device__ void block_interp(const T* Y, int ldy, int k, int e, T* Tm, int ldt, T* rinv) {
  for (int a = threadIdx.x; a < k; a += blockDim.x) rinv[a] = T(1) / Y[a + (size_t)ldy * a];
  __syncthreads();
  for (int j = threadIdx.x; j < e - k; j += blockDim.x) {
    for (int a = k - 1; a >= 0; --a) {
      T s = Y[a + (size_t)ldy * (k + j)];
      for (int b = a + 1; b < k; ++b) s -= Y[a + (size_t)ldy * b] * Tm[b + (size_t)ldt * j];
      Tm[a + (size_t)ldt * j] = s * rinv[a];
    }
  }
  __syncthreads();
}

// LU with partial pivoting of the n x n block of A at (r0, r0) (ld lda), with the row
// operations carried over columns [0, ncol) outside the factored block; multipliers are
// stored below the diagonal and not interchanged afterwards (the solve interleaves
// interchanges and eliminations).  inv receives the reciprocal pivots.  Returns false on an
// exactly zero pivot.
template <typename T>
__device__ bool block_gepp(T* A, int lda, int r0, int n, int ncol, int* piv, T* inv, int* shi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    const int cj = r0 + j;
    if (warp == 0) {
      double best = -1.0;
      int bi = n;
      for (int r = j + lane; r < n; r += 32) {
        double v = fabs((double)A[(r0 + r) + (size_t)lda * cj]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { shi[0] = bi; shi[1] = best == 0.0; piv[j] = bi; }
    }
    __syncthreads();
    const int p = shi[0];
    if (shi[1]) { ok = false; if (threadIdx.x == 0) inv[j] = T(0); __syncthreads(); continue; }
    if (p != j) {
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        if (c >= r0 && c < cj) continue;
        T a = A[(r0 + j) + (size_t)lda * c];
        A[(r0 + j) + (size_t)lda * c] = A[(r0 + p) + (size_t)lda * c];
        A[(r0 + p) + (size_t)lda * c] = a;
      }
      __syncthreads();
    }
    const T ipv = T(1) / A[(r0 + j) + (size_t)lda * cj];
    if (threadIdx.x == 0) inv[j] = ipv;
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) A[(r0 + r) + (size_t)lda * cj] *= ipv;
    __syncthreads();
    const int nr = n - j - 1;
    const int nc = ncol - 1;   // every column but cj
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      int r = j + 1 + e % nr;
      int c = e / nr;
      if (c >= cj) ++c;
      if (c >= r0 && c < cj) continue;   // multipliers of earlier steps
      A[(r0 + r) + (size_t)lda * c] -= A[(r0 + r) + (size_t)lda * cj] * A[(r0 + j) + (size_t)lda * c];
    }
    __syncthreads();
  }
  return ok;
}


// ------------------------------------------------------------ block reductions (FP64)
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------ tensor-core helpers (TF32)
// mma.sync m16n8k8 with TF32 operands and FP32 accumulation.  TF32 keeps 10 mantissa bits, so
// each operand is split into a high part tf32(x) and a low part tf32(x - hi) and three products
// are accumulated (the two cross terms first, then hi*hi): the result matches an FP32 product
// to about FP32 rounding (the lo*lo term, below 2^-22 relative, is dropped).
// Fragment layouts of m16n8k8 (PTX ISA, tf32): g = lane / 4, q = lane % 4;
//   A (16 x 8, row major): a0 (g, q), a1 (g + 8, q), a2 (g, q + 4), a3 (g + 8, q + 4);
//   B (8 x 8, column major): b0 (q, g), b1 (q + 4, g);
//   C (16 x 8): c0 (g, 2q), c1 (g, 2q + 1), c2 (g + 8, 2q), c3 (g + 8, 2q + 1).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}


// ------------------------------------------------------------ far-row sketch
// Yr[rr, c] = sum over far neighbour rows f of G[rr, f] B_F[f, c] for r0 <= rr < hh (unscaled),
// neighbours taken in chunks of ch (near ones get zero weight).  Yr has leading dimension ldy.
// Rows below r0 are left alone (the one-pass sketch takes them from the probe, whose rows are
// the same rows of G).
template <typename T, class BGet>
__device__ void sketch_far(const LevelDev& d, const SegCtx& S, const NbrTab& tb, BGet bget,
                           int sid, int halves, int e, int r0, int hh, T* Yr, int ldy, T* Bc, T* Gc,
                           int ch) {
  const int nr = hh - r0;
  for (int x = threadIdx.x; x < nr * e; x += blockDim.x) Yr[(r0 + x % nr) + (size_t)ldy * (x / nr)] = T(0);
  __syncthreads();
  for (int f0 = 0; f0 < S.nb; f0 += ch) {
    const int nc = min(ch, S.nb - f0);
    const int rows = halves * nc;
    for (int x = threadIdx.x; x < rows * e; x += blockDim.x) {
      int row = x % rows, c = x / rows;
      int t = row / nc, jj = row % nc;
      Bc[row + (size_t)rows * c] = bget(t, f0 + jj, c);
    }
    // one Philox counter per group of four sketch rows (r0 is a multiple of 4)
    const int g0 = r0 >> 2, ng = ((hh + 3) >> 2) - g0;
    for (int x = threadIdx.x; x < ng * rows; x += blockDim.x) {
      const int gi = x % ng, row = x / ng;
      const int t = row / nc, jj = row % nc;
      const Nbr q = nbr_get(d, S, tb, f0 + jj);
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (!q.nearf) sketch_gauss4(d.seed, d.l, sid, g0 + gi, q.node, t, z);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = 4 * (g0 + gi) + i - r0;
        if (rr < nr) Gc[rr + (size_t)nr * row] = (T)z[i];
      }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      if (d.sketch_tc) {
        // Y_chunk (nr x e) += G_chunk (nr x rows) B_chunk (rows x e) on the tensor cores: the
        // warps take 16 x 8 output tiles in turn, k in steps of 8 rows (zero past the end)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int g = lane >> 2, q = lane & 3;
        const int mt = (nr + 15) >> 4, nt = (e + 7) >> 3;
        auto Ga = [&](int r, int k) { return (r < nr && k < rows) ? (float)Gc[r + (size_t)nr * k] : 0.f; };
        auto Bb = [&](int k, int c) { return (k < rows && c < e) ? (float)Bc[k + (size_t)rows * c] : 0.f; };
        for (int t = warp; t < mt * nt; t += nw) {
          const int m0 = 16 * (t % mt), n0 = 8 * (t / mt);
          float acc[4] = {0.f, 0.f, 0.f, 0.f};
          for (int k0 = 0; k0 < rows; k0 += 8) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            split_tf32(Ga(m0 + g, k0 + q), ah[0], al[0]);
            split_tf32(Ga(m0 + g + 8, k0 + q), ah[1], al[1]);
            split_tf32(Ga(m0 + g, k0 + q + 4), ah[2], al[2]);
            split_tf32(Ga(m0 + g + 8, k0 + q + 4), ah[3], al[3]);
            split_tf32(Bb(k0 + q, n0 + g), bh[0], bl[0]);
            split_tf32(Bb(k0 + q + 4, n0 + g), bh[1], bl[1]);
            mma_tf32(acc, al, bh);
            mma_tf32(acc, ah, bl);
            mma_tf32(acc, ah, bh);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int rr = m0 + g + 8 * (u >> 1), c = n0 + 2 * q + (u & 1);
            if (rr < nr && c < e) Yr[(r0 + rr) + (size_t)ldy * c] += (T)acc[u];
          }
        }
        __syncthreads();
        continue;
      }
    }
    // sums over blocks of SK_CHUNK far unknowns (both halves of a block, then the next block):
    // the same order of operations for every chunk size, so that the sketch does not depend on
    // the shared-memory budget the level runs with
    for (int x = threadIdx.x; x < nr * e; x += blockDim.x) {
      const int rr = x % nr, c = x / nr;
      const T* g = Gc + rr;
      const T* bc = Bc + (size_t)rows * c;
      T y = Yr[(r0 + rr) + (size_t)ldy * c];
      for (int b0 = 0; b0 < nc; b0 += SK_CHUNK) {
        const int b1 = min(nc, b0 + SK_CHUNK);
        T acc = T(0);
#pragma unroll 4
        for (int row = b0; row < b1; ++row) acc += g[(size_t)nr * row] * bc[row];
        if (halves == 2) {
#pragma unroll 4
          for (int row = nc + b0; row < nc + b1; ++row) acc += g[(size_t)nr * row] * bc[row];
        }
        y += acc;
      }
      Yr[(r0 + rr) + (size_t)ldy * c] = y;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ learned rank predictor
// (no counterpart in the paper; the definitions are those of the oracle's predictor module)
// Probe sketch Y8[r + PRED_PROBE c] = sum over the far rows of G[r, row] B[row, c], r < 8: the
// first PRED_PROBE rows of the sketch matrix of this segment, unscaled.  Warps take rows in
// turn; lanes hold columns lane + 32 q of a 64-column chunk in registers; the warps' sums meet
// in Y8 (zeroed by the caller) through shared-memory atomics.
template <typename T, class BGet>
__device__ void probe_sketch(const LevelDev& d, const SegCtx& S, const NbrTab& tb, BGet bget,
                             int sid, int halves, int e, T* Y8) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nrows = halves * S.nb;
  const int ro = lane >> 3, r8 = lane & 7;                 // lane: row ro of a group of 4, probe row r8
  for (int c0 = 0; c0 < e; c0 += 64) {
    T acc[2][PRED_PROBE];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < PRED_PROBE; ++r) acc[q][r] = T(0);
    for (int g0 = 4 * warp; g0 < nrows; g0 += 4 * nw) {
      const int row = g0 + ro;
      Nbr q{0, -1, -1, true};
      int t = 0;
      if (row < nrows) {
        t = row / S.nb;
        q = nbr_get(d, S, tb, row % S.nb);
      }
      // lanes r8 = 0 and 4 of each node row draw the two counters (rows 0-3, 4-7); the
      // others take their component by shuffle
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (!q.nearf && (r8 & 3) == 0) sketch_gauss4(d.seed, d.l, sid, r8 >> 2, q.node, t, z);
      const int srcl = lane & ~3;
      float zc = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float v = __shfl_sync(0xffffffffu, z[i], srcl);
        if ((r8 & 3) == i) zc = v;
      }
      const T g = q.nearf ? T(0) : (T)zc;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int src = 8 * rr;
        if (__shfl_sync(0xffffffffu, (int)q.nearf, src)) continue;   // near or past the end
        const int rowr = g0 + rr, tr = rowr / S.nb, fr = rowr % S.nb;
        T b[2];
#pragma unroll
        for (int qc = 0; qc < 2; ++qc) {
          const int c = c0 + 32 * qc + lane;
          b[qc] = c < e ? bget(tr, fr, c) : T(0);
        }
#pragma unroll
        for (int r = 0; r < PRED_PROBE; ++r) {
          const T gr = __shfl_sync(0xffffffffu, g, src + r);
#pragma unroll
          for (int qc = 0; qc < 2; ++qc) acc[qc][r] += gr * b[qc];
        }
      }
    }
    // the warps add their partial sums in warp order (a fixed summation order: the probe, and
    // through it the predicted sketch size, is the same in every factorization)
    for (int w = 0; w < nw; ++w) {
      if (warp == w) {
#pragma unroll
        for (int qc = 0; qc < 2; ++qc) {
          const int c = c0 + 32 * qc + lane;
          if (c < e)
#pragma unroll
            for (int r = 0; r < PRED_PROBE; ++r) Y8[r + PRED_PROBE * c] += acc[qc][r];
        }
      }
      __syncthreads();
    }
  }
}

// Features of segment sid into xf[16] (shared), needs >= 2 warps; every thread calls it.
// Arithmetic in the factor's precision T (features are inputs of a BF16 network).
// Warp 0: column-pivoted QR of the probe Y8 (PRED_PROBE x e, pitch PRED_PROBE, overwritten)
// by Gram-Schmidt with exactly recomputed column norms, lane c owning columns c + 32 q; the
// pivot is the largest norm, near-ties (relative 1e-12) to the lowest column.  Warp 1: the
// coefficient statistics of the segment's nodes from the per-node table.
template <typename T>
__device__ void probe_features(const LevelDev& d, int sid, int e, int nnear, int nfar, int nb,
                               T* Y8, float* xf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    const int nd = min(PRED_PROBE, e);
    T rd[PRED_PROBE];
#pragma unroll
    for (int i = 0; i < PRED_PROBE; ++i) rd[i] = T(0);
    unsigned used = 0;                                       // bit q: column lane + 32 q pivoted
    T sq[4];
    for (int i = 0; i < nd; ++i) {
      T mx = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        sq[q] = T(-1);
        if (c < e && !(used >> q & 1)) {
          T a = T(0);
#pragma unroll
          for (int r = 0; r < PRED_PROBE; ++r) a += Y8[r + PRED_PROBE * c] * Y8[r + PRED_PROBE * c];
          sq[q] = a;
          mx = a > mx ? a : mx;
        }
      }
      for (int o = 16; o > 0; o >>= 1) { const T w = __shfl_xor_sync(0xffffffffu, mx, o); mx = w > mx ? w : mx; }
      if (!(mx > T(0))) break;
      const T thr = mx * (T)((1.0 - TIE_RTOL) * (1.0 - TIE_RTOL));
      int best = 1 << 30;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (sq[q] >= thr) best = min(best, lane + 32 * q);
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
      T v[PRED_PROBE];
      T pn = T(0);
#pragma unroll
      for (int r = 0; r < PRED_PROBE; ++r) {
        v[r] = Y8[r + PRED_PROBE * best];
        pn += v[r] * v[r];
      }
      pn = sqrt(pn);
      rd[i] = pn;
      const T inv = T(1) / pn;
#pragma unroll
      for (int r = 0; r < PRED_PROBE; ++r) v[r] *= inv;
      if ((best & 31) == lane) used |= 1u << (best >> 5);
      __syncwarp();
      for (int q = 0, c = lane; c < e; ++q, c += 32) {
        if (used >> q & 1) continue;
        T* col = Y8 + PRED_PROBE * c;
        T dot = T(0);
#pragma unroll
        for (int r = 0; r < PRED_PROBE; ++r) dot += v[r] * col[r];
#pragma unroll
        for (int r = 0; r < PRED_PROBE; ++r) col[r] -= dot * v[r];
      }
      __syncwarp();
    }
    if (lane < 5) {                                          // one decay ratio per lane
      const int js[5] = {1, 2, 3, 5, 7};
      const int j = js[lane];
      const T le = (T)d.log10eps;
      T val;
      if (j >= nd || rd[0] == T(0)) val = T(-16) - le;
      else {
        T rj = rd[0];
#pragma unroll
        for (int q = 1; q < PRED_PROBE; ++q) if (q == j) rj = rd[q];
        const T ratio = rj / rd[0];
        val = log10(ratio > T(1e-16) ? ratio : T(1e-16)) - le;
      }
      xf[11 + lane] = (float)val;
    }
  } else if (warp == 1) {
    const int* nodes = d.nodes + (size_t)sid * d.capS;
    float lmin = 3.0e38f, lmax = -3.0e38f, lsum = 0.f, dsum = 0.f, ssum = 0.f, asum = 0.f;
    for (int t = lane; t < e; t += 32) {
      const float4 st = d.nstat[nodes[t]];
      lmin = fminf(lmin, st.x);
      lmax = fmaxf(lmax, st.x);
      lsum += st.x;
      dsum += st.y;
      ssum += st.z;
      asum += st.w;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
      asum += __shfl_xor_sync(0xffffffffu, asum, o);
    }
    const float mean = lsum / e;
    float vsum = 0.f;
    for (int t = lane; t < e; t += 32) {
      const float dv = d.nstat[nodes[t]].x - mean;
      vsum += dv * dv;
    }
    for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
    if (lane == 0) {
      xf[0] = (float)(d.L - d.l);
      xf[1] = log2f((float)e);
      xf[2] = log2f(1.0f + nb);
      xf[3] = (float)nnear;
      xf[4] = log2f(1.0f + nfar);
      xf[5] = lmin - mean;
      xf[6] = lmax - mean;
      xf[7] = sqrtf(vsum / e);
      xf[8] = dsum / e;
      xf[9] = ssum / e;
      xf[10] = asum / e;
    }
  }
  __syncthreads();
}

// Measured ID error test ||B_r - B_s T||_F <= 10 eps ||B||_F on the exact B (all neighbour
// rows, both halves of a non-symmetric B): one thread per row of B, entries read directly.
template <typename T, class BGet>
__device__ bool id_error_ok(const SegCtx& S, BGet bget, int halves, int e, int k, const int* perm,
                            const T* Tw, int ldt, double eps, double* red) {
  const int r = e - k;
  T num = T(0), den = T(0);                 // per-thread sums in T, the block sum in FP64
  for (int row = threadIdx.x; row < halves * S.nb; row += blockDim.x) {
    const int f = row % S.nb, t = row / S.nb;
    for (int c = 0; c < e; ++c) {
      const T v = bget(t, f, c);
      den += v * v;
    }
    for (int j = 0; j < r; ++j) {
      T s = bget(t, f, perm[k + j]);
      for (int a = 0; a < k; ++a) s -= bget(t, f, perm[a]) * Tw[a + (size_t)ldt * j];
      num += s * s;
    }
  }
  const double nsum = block_sum((double)num, red);
  const double dsum = block_sum((double)den, red);
  return sqrt(nsum) <= 10.0 * eps * sqrt(dsum);
}

// ------------------------------------------------------------ sparsify: one CTA per segment
// The same column-pivoted Householder QR for CTAs of NWT warps when e <= 64, with the row work
// spread over the warps and the scalar work on warp 0; three barriers per step.  Lanes own
// columns (lane l: columns l and l + 32), warps own rows (warp w: rows r = w mod NWT).  Per
// step i: warp 0 downdates the FP64 squared norms by the row of step i - 1 (recomputing below
// the guard), chooses the pivot and forms the Householder scalars from the pivot column
// (before it moves), and publishes them; then every warp swaps columns i and p on its rows and
// forms its partial dots v^T y_j over its rows; then every warp sums the partial dots in warp
// order and updates its rows.  Same arithmetic as block_cpqr up to the order of the sums.
// part: >= NWT * 64 values of T; pub: >= 4 values of T.  All threads call it.
template <typename T, int NWT>
__device__ int rows_cpqr(T* Y, int ldy, int m, int e, double eps, int* perm, T* part, T* pub, int* shi,
                         int kstop) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < e; j += blockDim.x) perm[j] = j;
  if (m == 0 || e == 0) { __syncthreads(); return 0; }
  // initial squared norms: partial sums over each warp's rows, added in warp order by warp 0
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int j = lane + 32 * t;
    T s = T(0);
    if (j < e)
      for (int r = warp; r < m; r += NWT) { const T v = Y[r + (size_t)ldy * j]; s += v * v; }
    part[warp * 64 + j] = s;
  }
  __syncthreads();
  const double tol3z = sqrt(DBL_EPSILON);
  const double tie = (1.0 - TIE_RTOL) * (1.0 - TIE_RTOL);
  const int kmax = min(min(m, e), kstop);
  double n1[2] = {0.0, 0.0}, n2[2] = {0.0, 0.0};       // warp 0: squared norms of lane's columns
  double ref = 0.0;
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      T s = T(0);
      for (int w = 0; w < NWT; ++w) s += part[w * 64 + lane + 32 * t];
      n1[t] = n2[t] = lane + 32 * t < e ? (double)s : 0.0;
    }
  }
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    // ---- warp 0: downdates by row i - 1, pivot, Householder scalars of the pivot column
    if (warp == 0) {
      if (i > 0) {
        unsigned fl = 0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int j = lane + 32 * t;
          if (j > i - 1 && j < e && n1[t] != 0.0) {
            const double rij = (double)Y[(i - 1) + (size_t)ldy * j];
            const double sn = fmax(n1[t] - rij * rij, 0.0);
            if (sn <= tol3z * n2[t]) fl |= 1u << t;
            else n1[t] = sn;
          }
        }
        unsigned f0 = __ballot_sync(0xffffffffu, fl & 1u), f1 = __ballot_sync(0xffffffffu, (fl >> 1) & 1u);
        while (f0 | f1) {          // recompute from rows i.. (rare)
          int j;
          if (f0) { j = __ffs(f0) - 1; f0 &= f0 - 1; } else { j = 32 + __ffs(f1) - 1; f1 &= f1 - 1; }
          double s2 = 0.0;
          for (int r = i + lane; r < m; r += 32) { const double v = (double)Y[r + (size_t)ldy * j]; s2 += v * v; }
          for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          if (lane == (j & 31)) { if (j >> 5) { n1[1] = s2; n2[1] = s2; } else { n1[0] = s2; n2[0] = s2; } }
        }
      }
      long long mx = -1;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = lane + 32 * t;
        if (j >= i && j < e) mx = max(mx, dbits(n1[t]));
      }
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const long long thr = dbits(__longlong_as_double(mx) * tie);
      int p = e;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = lane + 32 * t;
        if (j >= i && j < e && dbits(n1[t]) >= thr && j < p) p = j;
      }
      for (int o = 16; o > 0; o >>= 1) p = min(p, __shfl_xor_sync(0xffffffffu, p, o));
      if (p != i) {
        const int si = i >> 5, sp = p >> 5;
        const double i1 = __shfl_sync(0xffffffffu, si ? n1[1] : n1[0], i & 31);
        const double i2 = __shfl_sync(0xffffffffu, si ? n2[1] : n2[0], i & 31);
        const double p1 = __shfl_sync(0xffffffffu, sp ? n1[1] : n1[0], p & 31);
        const double p2 = __shfl_sync(0xffffffffu, sp ? n2[1] : n2[0], p & 31);
        if (lane == (i & 31)) { if (si) { n1[1] = p1; n2[1] = p2; } else { n1[0] = p1; n2[0] = p2; } }
        if (lane == (p & 31)) { if (sp) { n1[1] = i1; n2[1] = i2; } else { n1[0] = i1; n2[0] = i2; } }
        if (lane == 0) { const int t = perm[i]; perm[i] = perm[p]; perm[p] = t; }
      }
      const T* yp = Y + (size_t)ldy * p;
      T s = T(0);
      for (int r = i + lane; r < m; r += 32) { const T v = yp[r]; s += v * v; }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const T normx = sqrt(s);
        const T x0 = yp[i];
        const T alpha = x0 >= T(0) ? -normx : normx;
        const T v0 = x0 - alpha;
        const T vv = v0 * v0 + (s - x0 * x0);
        if (i == 0) ref = (double)normx;
        int stop = 0;
        if (ref == 0.0) stop = 2;
        else if ((double)normx <= eps * ref || normx == T(0)) stop = 1;
        pub[0] = alpha;
        pub[1] = v0;
        pub[2] = vv > T(0) ? T(2) / vv : T(0);
        shi[0] = p;
        shi[1] = stop;
      }
    }
    __syncthreads();
    const int p = shi[0], stop = shi[1];
    // ---- every warp, its rows (one per lane): swap columns i and p (also on the stopping step,
    //      as perm already has)
    if (p != i)
      for (int r = warp + NWT * lane; r < m; r += NWT * 32) {
        T* a = Y + r + (size_t)ldy * i;
        T* b = Y + r + (size_t)ldy * p;
        const T tmp = *a; *a = *b; *b = tmp;
      }
    if (stop) { __syncthreads(); k = stop == 2 ? 0 : i; break; }
    __syncwarp();
    const T v0 = pub[1], c2 = pub[2];
    // ---- every warp, its rows: partial dots with v (v_i = v0)
    const int r0 = i + ((warp - i % NWT) + NWT) % NWT;   // this warp's first row >= i
    T acc[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int j = lane + 32 * t;
      acc[t] = T(0);
      if (j > i && j < e) {
        const T* yj = Y + (size_t)ldy * j;
        const T* yi = Y + (size_t)ldy * i;
        for (int r = r0; r < m; r += NWT) acc[t] += (r == i ? v0 : yi[r]) * yj[r];
      }
      part[warp * 64 + j] = acc[t];
    }
    __syncthreads();
    // ---- every warp, its rows: y_j -= c2 (v^T y_j) v
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int j = lane + 32 * t;
      if (j > i && j < e) {
        T d = T(0);
        for (int w = 0; w < NWT; ++w) d += part[w * 64 + j];
        const T cj = d * c2;
        T* yj = Y + (size_t)ldy * j;
        const T* yi = Y + (size_t)ldy * i;
        for (int r = r0; r < m; r += NWT) yj[r] -= cj * (r == i ? v0 : yi[r]);
      }
    }
    if (r0 == i && lane == 0) Y[i + (size_t)ldy * i] = pub[0];   // R_ii, by the warp owning row i
    __syncthreads();
  }
  __syncthreads();
  return k;
}

// Largest-first work list of a level (scheduling, not in the paper): a counting sort of the
// segment ids by decreasing unknown count, so that the sparsify CTAs, which the hardware
// starts roughly in index order, begin with the longest segments and the last wave holds the
// shortest.  Ids of equal count land in any order: every CTA writes only its own segment's
// outputs and keys its sketch by the segment id, so the order changes no result.
constexpr int ORD_B = 256;
__global__ void __launch_bounds__(1024) seg_order_kernel(const int* cnt, int nseg, int* order) {
  __shared__ int start[ORD_B];
  auto key = [](int e) { return ORD_B - 1 - min(max(e, 0), ORD_B - 1); };
  for (int i = threadIdx.x; i < ORD_B; i += blockDim.x) start[i] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) atomicAdd(&start[key(cnt[s])], 1);
  __syncthreads();
  if (threadIdx.x < 32) {            // exclusive scan of the 256 bucket sizes by one warp
    constexpr int PER = ORD_B / 32;
    const int lane = threadIdx.x;
    int v[PER], t = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) { v[j] = start[lane * PER + j]; t += v[j]; }
    int incl = t;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    int run = incl - t;
#pragma unroll
    for (int j = 0; j < PER; ++j) { start[lane * PER + j] = run; run += v[j]; }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) order[atomicAdd(&start[key(cnt[s])], 1)] = s;
}

template <typename T, int NWT>
__global__ void __launch_bounds__(NWT * 32, NWT == NW ? 4 : 16) sparsify_kernel(LevelDev d, int smem_bytes) {
  extern __shared__ double sm[];
  __shared__ SegCtx S;
  __shared__ double shr[NWT * 64 + 3 * 64];
  __shared__ int shi[8];
  __shared__ int nearlist[NEAR_MAX];
  __shared__ int nnear_sh, nfar_sh;

  const int sid = d.use_order ? d.order[blockIdx.x] : blockIdx.x;
  if (threadIdx.x == 0) seg_context(d, sid, S);
  __syncthreads();
  const int e = S.e;
  const int capS = d.capS;
  int* perm_out = d.perm + (size_t)sid * capS;
  if (threadIdx.x == 0) atomicMax(d.lstat + LS_EMAX, e);
  if (e == 0) {
    if (threadIdx.x == 0) { d.kk[sid] = 0; d.hs[sid] = 0; }
    return;
  }
  const size_t ld = d.ldF;
  const T* F1 = static_cast<const T*>(d.F) + (size_t)S.b1 * ld * ld;
  const T* F2 = static_cast<const T*>(d.F) + (size_t)S.b2 * ld * ld;
  T* Dg = static_cast<T*>(d.Dm) + (size_t)sid * capS * capS;
  T* Tg = static_cast<T*>(d.T) + (size_t)sid * capS * capS;
  T* Ig = static_cast<T*>(d.Dinv) + (size_t)sid * capS;
  const int halves = d.symmetric ? 1 : 2;

  // eps == 0: no sparsification, the whole segment is skeleton
  if (d.eps == 0.0) {
    for (int x = threadIdx.x; x < e * e; x += blockDim.x) {
      int a = x % e, b = x / e;
      Dg[a + (size_t)capS * b] = F1[(S.s1 + a) + ld * (S.s1 + b)] + F2[(S.s2 + a) + ld * (S.s2 + b)];
    }
    for (int j = threadIdx.x; j < e; j += blockDim.x) {
      perm_out[j] = j;
      d.snodes[(size_t)sid * capS + j] = d.nodes[(size_t)sid * capS + j];
    }
    if (threadIdx.x == 0) {
      d.kk[sid] = e;
      d.hs[sid] = 0;
      atomicAdd(d.flops + 2, (unsigned long long)(e * e * sizeof(T) + 2 * e * sizeof(int)));
    }
    return;
  }

  // near / far split of the neighbours (ordered scan, warp 0)
  if (threadIdx.x < 32) {
    int lane = threadIdx.x, nn = 0;
    for (int base = 0; base < S.nb; base += 32) {
      int f = base + lane;
      bool isnear = false;
      if (f < S.nb) {
        int r, i;
        locate(S, f, r, i);
        isnear = cheb(S, run_node(d, S.run[r], i), d.nx) <= d.near_radius;
      }
      unsigned msk = __ballot_sync(0xffffffffu, isnear);
      int pos = nn + __popc(msk & ((1u << lane) - 1u));
      if (isnear && pos < NEAR_MAX) nearlist[pos] = f;
      nn += __popc(msk);
    }
    if (lane == 0) {
      if (nn > NEAR_MAX) atomicOr(d.err, ERR_CAPACITY);
      nnear_sh = min(nn, NEAR_MAX);
      nfar_sh = S.nb - nn;
    }
  }
  // neighbour table (all threads)
  __shared__ int tb_node[NB_MAX];
  __shared__ short tb_p1[NB_MAX], tb_p2[NB_MAX];
  __shared__ unsigned char tb_nf[NB_MAX];
  const NbrTab tb{tb_node, tb_p1, tb_p2, tb_nf, S.nb <= NB_MAX};
  if (tb.on) {
    const NbrTab none{nullptr, nullptr, nullptr, nullptr, false};
    for (int f = threadIdx.x; f < S.nb; f += blockDim.x) {
      const Nbr q = nbr_get(d, S, none, f);
      tb_node[f] = q.node;
      tb_p1[f] = (short)q.p1;
      tb_p2[f] = (short)q.p2;
      tb_nf[f] = q.nearf ? 1 : 0;
    }
  }
  __syncthreads();
  const int nnear = nnear_sh;
  const int nN = halves * nnear;
  const int nF = halves * nfar_sh;
  const int hcap = max(d.h0, 2 * (e + d.p_over));
  const int hmax = min(nF, hcap);
  const int mmax = nN + hmax;

  // working storage: vectors and sketch chunks in shared memory; Y, D, T too when they
  // fit, else the global scratch of this segment
  const size_t TD = sizeof(T);
  const size_t small_b = (2 * (size_t)e) * 8 + (3 * (size_t)e + 4) * 4 + (size_t)e * TD + 64;
  const size_t per_ch_b = (size_t)halves * (e + hmax) * TD;
  const size_t ydt_b = ((size_t)(mmax + 1) * e + 2 * (size_t)e * e) * TD;
  // chunk of the sketch product: the largest of 64, 32 and 16 far unknowns whose working set
  // fits the budget together with the staged B block (or without it, where B never fits):
  // fewer chunks, fewer barriers on the coarse levels' long far fields
  int ch = SK_CHUNK;
  {
    const size_t bsz = (size_t)halves * S.nb * e * TD + 48;
    const bool keep_b = small_b + SK_CHUNK * per_ch_b + ydt_b + bsz <= (size_t)smem_bytes;
    for (int c = SK_CHUNK_MAX; c > SK_CHUNK; c >>= 1)
      if (small_b + c * per_ch_b + ydt_b + (keep_b ? bsz : 0) <= (size_t)smem_bytes) { ch = c; break; }
  }
  bool in_smem = small_b + ch * per_ch_b + ydt_b <= (size_t)smem_bytes;
  if (!in_smem) {
    size_t room = (size_t)smem_bytes > small_b ? (size_t)smem_bytes - small_b : 0;
    ch = (int)min((size_t)SK_CHUNK, room / (per_ch_b > 0 ? per_ch_b : 1));
    if (ch < 1) { ch = 1; if (threadIdx.x == 0) atomicOr(d.err, ERR_CAPACITY); }
  }
  T *Y, *Dw, *Tw, *Bc, *Gc, *rinv, *Bs;
  bool bstage;
  double *vn1, *vn2;
  int *perm, *piv, *flags;
  int ldy, ldd, ldt;
  {
    char* q = reinterpret_cast<char*>(sm);
    vn1 = reinterpret_cast<double*>(q); q += (size_t)e * 8;
    vn2 = reinterpret_cast<double*>(q); q += (size_t)e * 8;
    perm = reinterpret_cast<int*>(q); q += (size_t)e * 4;
    piv = reinterpret_cast<int*>(q); q += (size_t)e * 4;
    flags = reinterpret_cast<int*>(q); q += ((size_t)e + 4) * 4;
    q = reinterpret_cast<char*>(((uintptr_t)q + 15) & ~(uintptr_t)15);
    rinv = reinterpret_cast<T*>(q); q += (size_t)e * TD;
    q = reinterpret_cast<char*>(((uintptr_t)q + 15) & ~(uintptr_t)15);
    Bc = reinterpret_cast<T*>(q); q += (size_t)halves * ch * e * TD;
    Gc = reinterpret_cast<T*>(q); q += (size_t)hmax * halves * ch * TD;
    if (in_smem) {
      Y = reinterpret_cast<T*>(q); q += (size_t)(mmax + 1) * e * TD; ldy = mmax | 1;   // odd pitch
      Dw = reinterpret_cast<T*>(q); q += (size_t)e * e * TD; ldd = e;
      Tw = reinterpret_cast<T*>(q); q += (size_t)e * e * TD; ldt = e;
    } else {
      Y = static_cast<T*>(d.Yg) + (size_t)sid * d.Ycap * capS; ldy = d.Ycap;
      Dw = Dg; ldd = capS;
      Tw = Tg; ldt = capS;
    }
    // the segment's B block (every neighbour row, e columns) in what is left, when it fits
    q = reinterpret_cast<char*>(((uintptr_t)q + 15) & ~(uintptr_t)15);
    Bs = reinterpret_cast<T*>(q);
    bstage = (size_t)(q - reinterpret_cast<char*>(sm)) + (size_t)halves * S.nb * e * TD <= (size_t)smem_bytes;
  }
  if (!in_smem && (mmax > d.Ycap || d.Yg == nullptr)) {   // no room: report, touch nothing
    if (threadIdx.x == 0) { atomicOr(d.err, ERR_CAPACITY); d.kk[sid] = 0; d.hs[sid] = 0; }
    return;
  }
  // B staged once (all loads in flight) for the near rows, every sketch pass, the probe and
  // the error test; otherwise each reads the frontal blocks through the neighbour table
  if (bstage) {
    for (int x = threadIdx.x; x < halves * S.nb * e; x += blockDim.x) {
      const int row = x / e, c = x % e;
      Bs[x] = bval_q<T>(d, S, F1, F2, nbr_get(d, S, tb, row % S.nb), row / S.nb, c);
    }
    __syncthreads();
  }
  auto bget = [&](int t, int f, int c) -> T {
    return bstage ? Bs[((size_t)t * S.nb + f) * e + c] : bval_q<T>(d, S, F1, F2, nbr_get(d, S, tb, f), t, c);
  };

  // ---- learned rank predictor (not in the paper): features from an 8-row probe of the
  //      far rows, then the network's one-pass sketch size (PRED_PREDICT) or a training
  //      record of the features and the adaptive rank (PRED_RECORD)
  __shared__ float xf[PRED_NFEAT], zs[PRED_NFEAT], hid[PRED_NHID], pout[PRED_NOUT];
  // rank bound (k <= e): a segment with e + p <= 2 h0 is sketched once with
  // h = min(2 h0, hmax) >= min(|F|, e + p), the size the adaptive schedule reaches at its
  // second pass, and that pass always stands; the predictor serves the larger segments.
  // Every h stays <= hmax, the rows the sketch buffer was sized for.
  const bool small = e + d.p_over <= 2 * d.h0;
  const bool use_pred = d.pred_mode != PRED_OFF && nF > max(d.h0, PRED_PROBE) && e <= PRED_EMAX && !small;
  int h = (nF <= d.h0) ? nF : small ? min(hmax, 2 * d.h0) : min(hmax, d.h0);
  bool predicted = false;
  if (use_pred) {
    for (int x = threadIdx.x; x < PRED_PROBE * e; x += blockDim.x) Y[x] = T(0);   // Y8, pitch 8
    __syncthreads();
    probe_sketch<T>(d, S, tb, bget, sid, halves, e, Y);
    __syncthreads();
    if (d.pred_mode == PRED_PREDICT && e >= PRED_PROBE) {
      // keep the probe (the first PRED_PROBE rows of this segment's G times B_F, unscaled) for
      // the one-pass sketch: the features' QR overwrites it, and T is free until the ID
      for (int x = threadIdx.x; x < PRED_PROBE * e; x += blockDim.x) Tw[x] = Y[x];
      __syncthreads();
    }
    probe_features<T>(d, sid, e, nnear, nfar_sh, S.nb, Y, xf);
    if (d.pred_mode == PRED_RECORD) {
      if (threadIdx.x < PRED_NFEAT) d.feat[(size_t)sid * PRED_NFEAT + threadIdx.x] = xf[threadIdx.x];
    } else {
      mlp_infer_block(*d.pred, xf, zs, hid, pout);
      h = pred_sketch_size(pout, nF, e, d.p_over, d.h0, d.pred_margin);
      predicted = true;
    }
  }

  h = min(h, hmax);          // the sketch buffer holds nN + hmax rows
  // ---- adaptive sketch + ID (Sec. 4.2.3; h = k + p with k unknown: double h until k <= h - p)
  int k = 0;
  int passes = 0;
  bool fellback = false, have_t = false;
  const bool was_predicted = predicted;
  unsigned long long work_done = 0;       // algorithmic FLOPs of this segment (thread 0)
  while (true) {
    const bool full = (h >= nF);
    const int hh = full ? nF : h;
    const int m = nN + hh;
    if (threadIdx.x == 0 && !full) work_done += work::sketch(hh, nF, e);
    // near rows
    for (int x = threadIdx.x; x < nN * e; x += blockDim.x) {
      int row = x % nN, c = x / nN;
      int t = row / nnear, a = row % nnear;
      Y[row + (size_t)ldy * c] = bget(t, nearlist[a], c);
    }
    if (full) {
      // Phi = I on the far block: far rows in the enumeration order of the neighbours;
      // position of far neighbour f = f minus the near ones before it
      for (int f = threadIdx.x; f < S.nb; f += blockDim.x) {
        int before = 0;
        bool isnear = false;
        for (int a = 0; a < nnear; ++a) {
          if (nearlist[a] < f) ++before;
          if (nearlist[a] == f) isnear = true;
        }
        if (isnear) continue;
        int j = f - before;
        for (int t = 0; t < halves; ++t)
          for (int c = 0; c < e; ++c)
            Y[(nN + t * nfar_sh + j) + (size_t)ldy * c] = bget(t, f, c);
      }
    } else {
      // Y_F = G B_F, chunks of neighbours (near ones get zero weight); the one-pass sketch of
      // a predicted segment takes its first PRED_PROBE rows from the probe
      const int r0 = (predicted && e >= PRED_PROBE) ? min(PRED_PROBE, hh) : 0;
      if (r0 < hh) sketch_far<T>(d, S, tb, bget, sid, halves, e, r0, hh, Y + nN, ldy, Bc, Gc, ch);
      const T sc = (T)(1.0 / sqrt((double)hh));
      for (int x = threadIdx.x; x < hh * e; x += blockDim.x) {
        const int rr = x % hh, c = x / hh;
        T* yv = Y + (nN + rr) + (size_t)ldy * c;
        *yv = (rr < r0 ? Tw[rr + PRED_PROBE * c] : *yv) * sc;
      }
    }
    __syncthreads();
    // a pass that can still double h only needs to know whether k > h - p: its QR stops at
    // step h - p + 1 (the same decision, the remaining steps skipped)
    const int kstop = (!full && h < nF) ? max(1, hh - d.p_over + 1) : e;
    k = (NWT == NW && e <= 64)
            ? rows_cpqr<T, NWT>(Y, ldy, m, e, d.eps, perm, reinterpret_cast<T*>(shr),
                                reinterpret_cast<T*>(shr) + NWT * 64, shi, kstop)
            : block_cpqr<T, NWT>(Y, ldy, m, e, d.eps, perm, vn1, vn2, shr, flags, shi, kstop);
    ++passes;
    if (threadIdx.x == 0) work_done += work::qr(m, e, k);
    if (predicted) {          // the one-pass ID stands if it passes the measured-error test
      predicted = false;
      if (full) break;
      bool ok = k <= h - d.p_over;
      if (ok) {
        block_interp<T>(Y, ldy, k, e, Tw, ldt, rinv);
        have_t = true;
        ok = id_error_ok<T>(S, bget, halves, e, k, perm, Tw, ldt, d.eps, shr);
      }
      if (ok) break;
      fellback = true;
      have_t = false;
      h = min(2 * h, hmax);     // hmax = min(|F|, max(h0, 2(e+p))): k <= e < hmax - p
      __syncthreads();
      continue;
    }
    if (!full && k > h - d.p_over && h < nF) {
      h = min(2 * h, hmax);     // never binds without a prediction (h < 2(k+p))
      __syncthreads();
      continue;
    }
    break;
  }
  if (threadIdx.x == 0) {
    atomicAdd(d.lstat + LS_PASSES, passes);
    if (fellback) atomicAdd(d.lstat + LS_FALLBACK, 1);
    if (was_predicted) atomicAdd(d.lstat + LS_PREDICTED, 1);
    if (use_pred && d.pred_mode == PRED_RECORD) {
      int* tg = d.tgt + (size_t)sid * 4;
      tg[0] = k; tg[1] = nF; tg[2] = 1; tg[3] = passes;
    }
  }
  const int r = e - k;
  if (!have_t) block_interp<T>(Y, ldy, k, e, Tw, ldt, rinv);

  // ---- transformed diagonal block in [skeleton | remainder] order (Eq. (UtALt))
  for (int x = threadIdx.x; x < e * e; x += blockDim.x) {
    int a = x % e, b = x / e;
    int pa = perm[a], pb = perm[b];
    Dw[a + (size_t)ldd * b] = F1[(S.s1 + pa) + ld * (S.s1 + pb)] + F2[(S.s2 + pa) + ld * (S.s2 + pb)];
  }
  __syncthreads();
  if (k > 0 && r > 0) {
    // column operation: D[:, k:] -= D[:, :k] T
    for (int x = threadIdx.x; x < e * r; x += blockDim.x) {
      int a = x % e, b = x / e;
      T s = T(0);
      for (int c = 0; c < k; ++c) s += Dw[a + (size_t)ldd * c] * Tw[c + (size_t)ldt * b];
      Dw[a + (size_t)ldd * (k + b)] -= s;
    }
    __syncthreads();
    // row operation: D[k:, :] -= T^T D[:k, :]
    for (int x = threadIdx.x; x < r * e; x += blockDim.x) {
      int a = x % r, b = x / r;
      T s = T(0);
      for (int c = 0; c < k; ++c) s += Tw[c + (size_t)ldt * a] * Dw[c + (size_t)ldd * b];
      Dw[(k + a) + (size_t)ldd * b] -= s;
    }
    __syncthreads();
  }
  // ---- eliminate the remainder: LU(A_rr) with W = L^{-1} P A_rk, Z = A_kr U^{-1},
  //      A_kk -= Z W  (Eq. (L^-1 * A * U^-1) for the segments of level l)
  if (r > 0) {
    bool ok = block_gepp<T>(Dw, ldd, k, r, e, piv, rinv, shi);
    if (!ok && threadIdx.x == 0) atomicOr(d.err, ERR_SINGULAR);
    if (k > 0) {
      for (int a = threadIdx.x; a < k; a += blockDim.x) {     // Z = A_kr U^{-1}, row by row
        for (int j = 0; j < r; ++j) {
          T s = Dw[a + (size_t)ldd * (k + j)];
          for (int i2 = 0; i2 < j; ++i2) s -= Dw[a + (size_t)ldd * (k + i2)] * Dw[(k + i2) + (size_t)ldd * (k + j)];
          Dw[a + (size_t)ldd * (k + j)] = s * rinv[j];
        }
      }
      __syncthreads();
      for (int x = threadIdx.x; x < k * k; x += blockDim.x) {
        int a = x % k, b = x / k;
        T s = T(0);
        for (int j = 0; j < r; ++j) s += Dw[a + (size_t)ldd * (k + j)] * Dw[(k + j) + (size_t)ldd * b];
        Dw[a + (size_t)ldd * b] -= s;
      }
      __syncthreads();
    }
  }
  // ---- outputs
  if (in_smem) {
    for (int x = threadIdx.x; x < e * e; x += blockDim.x) Dg[(x % e) + (size_t)capS * (x / e)] = Dw[x];
    for (int x = threadIdx.x; x < k * r; x += blockDim.x) Tg[(x % k) + (size_t)capS * (x / k)] = Tw[(x % k) + (size_t)ldt * (x / k)];
  }
  for (int j = threadIdx.x; j < e; j += blockDim.x) {
    perm_out[j] = perm[j];
    d.snodes[(size_t)sid * capS + j] = d.nodes[(size_t)sid * capS + perm[j]];
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    d.piv[(size_t)sid * capS + j] = piv[j];
    Ig[j] = rinv[j];
  }
  if (threadIdx.x == 0) {
    d.kk[sid] = k;
    d.hs[sid] = h;
    work_done += work::interp(k, e) + work::apply(e, k) + (r > 0 ? work::elim(r, k) : 0ull);
    atomicAdd(d.flops, work_done);
    atomicAdd(d.flops + 2, (unsigned long long)((k * r + e * e) * sizeof(T) + 2 * e * sizeof(int)));
  }
}

// ------------------------------------------------------------ level-L segment tables
__global__ void level_init_L_kernel(LevelDev d) {
  const int nseg = d.g.nseg();
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nseg * LEAF; x += gridDim.x * blockDim.x) {
    int sid = x / LEAF, t = x % LEAF;
    d.nodes[(size_t)sid * d.capS + t] = d.g.seg_node(sid, t, d.nx);
    if (t == 0) d.cnt[sid] = LEAF;
  }
}

// ------------------------------------------------------------ merge (Sec. 4.3, E_(l))
// Table entry per unknown of the parent's extended block [dP | p]: see MERGE_TABW.
constexpr int TABW = MERGE_TABW;

struct ParentCtx {
  int Ip, Jp, c1, c2, I1, J1, I2, J2, sep, kp;
};

__device__ void parent_ctx(const LevelDev& d, int P, ParentCtx& C) {
  C.Ip = P % d.gp.bx;
  C.Jp = P / d.gp.bx;
  if (d.vcut) { C.I1 = 2 * C.Ip; C.J1 = C.Jp; C.I2 = 2 * C.Ip + 1; C.J2 = C.Jp; }
  else { C.I1 = C.Ip; C.J1 = 2 * C.Jp; C.I2 = C.Ip; C.J2 = 2 * C.Jp + 1; }
  C.c1 = C.I1 + d.g.bx * C.J1;
  C.c2 = C.I2 + d.g.bx * C.J2;
  C.sep = d.g.box_side(C.I1, C.J1, d.vcut ? SIDE_RIGHT : SIDE_TOP);
  C.kp = d.kk[C.sep];
}

// The table is built in two passes: thread 0 lists the runs of entries (a child side's
// skeleton, a junction or corner, the separator skeleton) with their first table index and
// first position in the parent block, then all threads fill the entries.
struct TabRun {
  int kind;            // 0: side of child `child`, 1: corner / junction, 2: separator skeleton
  int n0, cnt, pos;    // first table index, entries, first position in the parent block
  int child, I, J, side;
  int I1, J1, c1, I2, J2, c2;
};
constexpr int TRUN_MAX = 16;

__global__ void merge_table_kernel(LevelDev d) {
  __shared__ TabRun runs[TRUN_MAX];
  __shared__ int nrun_sh, total_sh;
  const int P = blockIdx.x;
  ParentCtx C;
  parent_ctx(d, P, C);
  int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  const Geo gp = d.gp;
  const int Dp = gp.D();
  if (threadIdx.x == 0) {
    const bool root = gp.bx * gp.by == 1;
    int n = 0, nr = 0;
    auto side_run = [&](int pos, int child, int I, int J, int side) {
      const int sg = d.g.box_side(I, J, side);
      if (sg < 0) return 0;
      TabRun& R = runs[nr++];
      R.kind = 0; R.n0 = n; R.cnt = d.kk[sg]; R.pos = pos; R.child = child; R.I = I; R.J = J; R.side = side;
      n += R.cnt;
      return R.cnt;
    };
    auto corner_run = [&](int pos, int I1, int J1, int c1, int I2, int J2, int c2) {
      const int cid = c1 >= 0 ? d.g.box_corner(I1, J1, c1) : d.g.box_corner(I2, J2, c2);
      if (cid < 0) return 0;
      TabRun& R = runs[nr++];
      R.kind = 1; R.n0 = n; R.cnt = 1; R.pos = pos;
      R.I1 = I1; R.J1 = J1; R.c1 = c1; R.I2 = I2; R.J2 = J2; R.c2 = c2;
      n += 1;
      return 1;
    };
    // sides of P (merged or inherited), then its corners, then the separator skeleton
    for (int side = 0; side < 4 && !root; ++side) {
      if (gp.box_side(C.Ip, C.Jp, side) < 0) continue;
      const int pos = gp.side_pos(side);
      const bool split = d.vcut ? (side == SIDE_BOTTOM || side == SIDE_TOP) : (side == SIDE_LEFT || side == SIDE_RIGHT);
      if (!split) {
        const int child = d.vcut ? (side == SIDE_LEFT ? 1 : 2) : (side == SIDE_BOTTOM ? 1 : 2);
        side_run(pos, child, child == 1 ? C.I1 : C.I2, child == 1 ? C.J1 : C.J2, side);
      } else {
        const int k1 = side_run(pos, 1, C.I1, C.J1, side);
        // junction: vertical cut: bottom -> b1.BR = b2.BL, top -> b1.TR = b2.TL;
        //           horizontal cut: left -> b1.TL = b2.BL, right -> b1.TR = b2.BR
        int jc1, jc2;
        if (d.vcut) { jc1 = side == SIDE_BOTTOM ? C_BR : C_TR; jc2 = side == SIDE_BOTTOM ? C_BL : C_TL; }
        else { jc1 = side == SIDE_LEFT ? C_TL : C_TR; jc2 = side == SIDE_LEFT ? C_BL : C_BR; }
        const int kj = corner_run(pos + k1, C.I1, C.J1, jc1, C.I2, C.J2, jc2);
        side_run(pos + k1 + kj, 2, C.I2, C.J2, side);
      }
    }
    for (int c = 0; c < 4 && !root; ++c) {
      if (gp.box_corner(C.Ip, C.Jp, c) < 0) continue;
      // vertical cut: BL,TL from b1; BR,TR from b2.  horizontal: BL,BR from b1; TL,TR from b2
      const bool from1 = d.vcut ? (c == C_BL || c == C_TL) : (c == C_BL || c == C_BR);
      if (from1) corner_run(gp.corner_pos(c), C.I1, C.J1, c, 0, 0, -1);
      else corner_run(gp.corner_pos(c), 0, 0, -1, C.I2, C.J2, c);
    }
    const int ndP = n;
    {
      TabRun& R = runs[nr++];
      R.kind = 2; R.n0 = n; R.cnt = C.kp; R.pos = Dp;
      n += C.kp;
    }
    nrun_sh = nr;
    total_sh = n;
    d.pcount[2 * P] = ndP;
    d.pcount[2 * P + 1] = C.kp;
    if (C.kp > 0) {
      atomicAdd(d.flops + 1, work::elim(C.kp, ndP));
      const size_t tb = d.fp32 ? sizeof(float) : sizeof(double);
      atomicAdd(d.flops + 3, (unsigned long long)(((size_t)C.kp * C.kp + 2 * (size_t)C.kp * ndP) * tb +
                                                  (size_t)C.kp * sizeof(int)));
    }
    atomicMax(d.lstat + LS_KPMAX, C.kp);
    atomicMax(d.lstat + LS_DPMAX, ndP);
  }
  __syncthreads();
  const int nr = nrun_sh, total = total_sh;
  for (int x = threadIdx.x; x < total; x += blockDim.x) {
    int ri = 0;
    while (ri + 1 < nr && x >= runs[ri + 1].n0) ++ri;
    const TabRun& R = runs[ri];
    const int t = x - R.n0;
    int* e = tab + (size_t)x * TABW;
    if (R.kind == 0) {
      const int sg = d.g.box_side(R.I, R.J, R.side);
      const int q = d.perm[(size_t)sg * d.capS + t];
      const int pc = d.g.side_pos(R.side) + q;
      e[0] = R.pos + t;
      e[1] = e[2] = e[3] = e[4] = e[5] = e[6] = -1;
      e[R.child == 1 ? 1 : 4] = pc;
      e[R.child == 1 ? 2 : 5] = R.side;
      e[R.child == 1 ? 3 : 6] = t;
      e[7] = d.nodes[(size_t)sg * d.capS + q];
    } else if (R.kind == 1) {
      const int cid = R.c1 >= 0 ? d.g.box_corner(R.I1, R.J1, R.c1) : d.g.box_corner(R.I2, R.J2, R.c2);
      e[0] = R.pos;
      e[1] = R.c1 >= 0 ? d.g.corner_pos(R.c1) : -1;
      e[2] = R.c1 >= 0 ? 4 : -1;
      e[3] = 0;
      e[4] = R.c2 >= 0 ? d.g.corner_pos(R.c2) : -1;
      e[5] = R.c2 >= 0 ? 4 : -1;
      e[6] = 0;
      e[7] = d.g.junction_node(cid, d.nx);
    } else {
      // separator skeleton: side RIGHT/TOP of child 1 (owner) = LEFT/BOTTOM of child 2
      const int s1 = d.vcut ? SIDE_RIGHT : SIDE_TOP, s2 = d.vcut ? SIDE_LEFT : SIDE_BOTTOM;
      const int sg = C.sep;
      const int q = d.perm[(size_t)sg * d.capS + t];
      e[0] = Dp + t;
      e[1] = d.g.side_pos(s1) + q; e[2] = s1; e[3] = t;
      e[4] = d.g.side_pos(s2) + q; e[5] = s2; e[6] = t;
      e[7] = d.nodes[(size_t)sg * d.capS + q];
    }
  }
}

// M[a][b] = sum over the children holding both unknowns of the child's block, where the
// block of a segment with itself is its eliminated skeleton block A_ss' (held by the owner
// child: the segment is that child's TOP or RIGHT side) and zero in the other child.
template <typename T>
__global__ void merge_assemble_kernel(LevelDev d) {
  const int P = blockIdx.y;
  const int nM = d.pcount[2 * P] + d.pcount[2 * P + 1];
  const int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  ParentCtx C;
  parent_ctx(d, P, C);
  const size_t ld = d.ldF, ldp = d.ldFp;
  const T* F1 = static_cast<const T*>(d.F) + (size_t)C.c1 * ld * ld;
  const T* F2 = static_cast<const T*>(d.F) + (size_t)C.c2 * ld * ld;
  const T* Dm = static_cast<const T*>(d.Dm);
  T* M = static_cast<T*>(d.Fp) + (size_t)P * ldp * ldp;
  const long long tot = (long long)nM * nM;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot;
       x += (long long)gridDim.x * blockDim.x) {
    int a = (int)(x % nM), b = (int)(x / nM);
    const int* ea = tab + (size_t)a * TABW;
    const int* eb = tab + (size_t)b * TABW;
    T v = T(0);
    for (int ch = 0; ch < 2; ++ch) {
      int pa = ea[1 + 3 * ch], pb = eb[1 + 3 * ch];
      if (pa < 0 || pb < 0) continue;
      int sa = ea[2 + 3 * ch], sb = eb[2 + 3 * ch];
      if (sa == sb && sa < 4) {
        if (sa == SIDE_TOP || sa == SIDE_RIGHT) {
          int I = ch == 0 ? C.I1 : C.I2, J = ch == 0 ? C.J1 : C.J2;
          int sg = d.g.box_side(I, J, sa);
          v += Dm[(size_t)sg * d.capS * d.capS + ea[3 + 3 * ch] + (size_t)d.capS * eb[3 + 3 * ch]];
        }
      } else {
        const T* Fc = ch == 0 ? F1 : F2;
        v += Fc[pa + ld * pb];
      }
    }
    M[ea[0] + ldp * eb[0]] = v;
  }
}

// LU of the separator block with the row operations over every column (W = L^{-1} P A_pd),
// then Z = A_dp U^{-1}.  When the kp separator rows over all nM columns fit in the dynamic
// shared memory (smem_bytes), they are staged there: the elimination then runs on shared
// memory with the same operations in the same order, and the rows are written back once.
template <typename T, bool ZREG>
__global__ void __launch_bounds__(256) merge_panel_kernel(LevelDev d, int smem_bytes) {
  extern __shared__ double pm_sm[];
  __shared__ int shi[4];
  const int P = blockIdx.x;
  const int ndP = d.pcount[2 * P], kp = d.pcount[2 * P + 1];
  if (kp == 0) return;
  const int nM = ndP + kp;
  const int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  const size_t ldp = d.ldFp;
  T* M = static_cast<T*>(d.Fp) + (size_t)P * ldp * ldp;
  T* inv = static_cast<T*>(d.Pinv) + (size_t)P * d.sepcap;
  const int Dp = d.gp.D();
  int* piv = d.ppiv + (size_t)P * d.sepcap;
  bool ok = true;
  if ((size_t)kp * nM * sizeof(T) + (size_t)nM * sizeof(int) <= (size_t)smem_bytes) {
    // staged rows: Pn[r + kp c] = M[Dp + r, column of table entry c]; entries [ndP, nM) are
    // the separator itself (positions Dp + j), [0, ndP) the parent boundary
    T* Pn = reinterpret_cast<T*>(pm_sm);
    int* colp = reinterpret_cast<int*>(Pn + (size_t)kp * nM);
    for (int c = threadIdx.x; c < nM; c += blockDim.x) colp[c] = tab[(size_t)c * TABW];
    __syncthreads();
    for (int x = threadIdx.x; x < kp * nM; x += blockDim.x)
      Pn[x] = M[(Dp + x % kp) + ldp * colp[x / kp]];
    __syncthreads();
    auto at = [&](int r, int c) -> T& { return Pn[r + (size_t)kp * c]; };
    for (int j = 0; j < kp; ++j) {
      const int cs = ndP + j;                   // staged column of separator unknown j
      if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        double best = -1.0;
        int bi = kp;
        for (int r = j + lane; r < kp; r += 32) {
          double v = fabs((double)at(r, cs));
          if (v > best || (v == best && r < bi)) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { shi[0] = bi; shi[1] = best == 0.0; piv[j] = bi; }
      }
      __syncthreads();
      const int p = shi[0];
      if (shi[1]) { ok = false; if (threadIdx.x == 0) inv[j] = T(0); __syncthreads(); continue; }
      if (p != j) {
        for (int c = threadIdx.x; c < nM; c += blockDim.x) {
          if (c >= ndP && c < cs) continue;     // multipliers of earlier steps
          T a = at(j, c);
          at(j, c) = at(p, c);
          at(p, c) = a;
        }
        __syncthreads();
      }
      const T ipv = T(1) / at(j, cs);
      if (threadIdx.x == 0) inv[j] = ipv;
      for (int r = j + 1 + threadIdx.x; r < kp; r += blockDim.x) at(r, cs) *= ipv;
      __syncthreads();
      const int nr = kp - j - 1;
      const int ncols = (kp - j - 1) + ndP;
      for (int x = threadIdx.x; x < nr * ncols; x += blockDim.x) {
        int r = j + 1 + x % nr, cc = x / nr;
        int c = cc < kp - j - 1 ? (cs + 1 + cc) : (cc - (kp - j - 1));
        at(r, c) -= at(r, cs) * at(j, c);
      }
      __syncthreads();
    }
    if (!ok && threadIdx.x == 0) atomicOr(d.err, ERR_SINGULAR);
    for (int x = threadIdx.x; x < kp * nM; x += blockDim.x)
      M[(Dp + x % kp) + ldp * colp[x / kp]] = Pn[x];
    // Z = A_dp U^{-1}: each dP row solved left to right, U from the staged rows; ZREG (levels of
    // few parents, where this chain is the latency): a separator of at most 32 unknowns keeps
    // the row in registers (one load and one store per entry, the same operations in the same
    // order)
    if (ZREG && kp <= 32) {
      for (int a = threadIdx.x; a < ndP; a += blockDim.x) {
        const size_t row = colp[a];
        T z[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < kp) z[j] = M[row + ldp * (Dp + j)];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j < kp) {
            T s = z[j];
#pragma unroll
            for (int i = 0; i < j; ++i) s -= z[i] * at(i, ndP + j);
            z[j] = s * inv[j];
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < kp) M[row + ldp * (Dp + j)] = z[j];
      }
      return;
    }
    for (int a = threadIdx.x; a < ndP; a += blockDim.x) {
      size_t row = colp[a];
      for (int j = 0; j < kp; ++j) {
        T s = M[row + ldp * (Dp + j)];
        for (int i = 0; i < j; ++i) s -= M[row + ldp * (Dp + i)] * at(i, ndP + j);
        M[row + ldp * (Dp + j)] = s * inv[j];
      }
    }
    return;
  }
  for (int j = 0; j < kp; ++j) {
    const int cj = Dp + j;
    if (threadIdx.x < 32) {
      int lane = threadIdx.x;
      double best = -1.0;
      int bi = kp;
      for (int r = j + lane; r < kp; r += 32) {
        double v = fabs((double)M[(Dp + r) + ldp * cj]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { shi[0] = bi; shi[1] = best == 0.0; piv[j] = bi; }
    }
    __syncthreads();
    const int p = shi[0];
    if (shi[1]) { ok = false; if (threadIdx.x == 0) inv[j] = T(0); __syncthreads(); continue; }
    if (p != j) {
      for (int c = threadIdx.x; c < nM; c += blockDim.x) {
        const int pc = tab[(size_t)c * TABW];
        if (pc >= Dp && pc < cj) continue;
        size_t col = ldp * pc;
        T a = M[(Dp + j) + col];
        M[(Dp + j) + col] = M[(Dp + p) + col];
        M[(Dp + p) + col] = a;
      }
      __syncthreads();
    }
    const T ipv = T(1) / M[(Dp + j) + ldp * cj];
    if (threadIdx.x == 0) inv[j] = ipv;
    for (int r = j + 1 + threadIdx.x; r < kp; r += blockDim.x) M[(Dp + r) + ldp * cj] *= ipv;
    __syncthreads();
    const int nr = kp - j - 1;
    // update rows j+1.. over columns: the separator columns j+1..kp-1 and every dP column
    const int ncols = (kp - j - 1) + ndP;
    for (int x = threadIdx.x; x < nr * ncols; x += blockDim.x) {
      int r = j + 1 + x % nr, cc = x / nr;
      int col = cc < kp - j - 1 ? (Dp + j + 1 + cc) : tab[(size_t)(cc - (kp - j - 1)) * TABW];
      M[(Dp + r) + ldp * col] -= M[(Dp + r) + ldp * cj] * M[(Dp + j) + ldp * col];
    }
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) atomicOr(d.err, ERR_SINGULAR);
  // Z = A_dp U^{-1}: each dP row solved left to right
  for (int a = threadIdx.x; a < ndP; a += blockDim.x) {
    size_t row = tab[(size_t)a * TABW];
    for (int j = 0; j < kp; ++j) {
      T s = M[row + ldp * (Dp + j)];
      for (int i = 0; i < j; ++i) s -= M[row + ldp * (Dp + i)] * M[(Dp + i) + ldp * (Dp + j)];
      M[row + ldp * (Dp + j)] = s * inv[j];
    }
  }
}

// Schur update of the parent's boundary block: M[dP, dP] -= Z W (64 x 64 tiles)
template <typename T>
__global__ void __launch_bounds__(256) merge_schur_kernel(LevelDev d) {
  __shared__ T Zs[64][17];
  __shared__ T Ws[16][65];
  __shared__ int ra[64], cb[64];
  const int P = blockIdx.z;
  const int ndP = d.pcount[2 * P], kp = d.pcount[2 * P + 1];
  if (kp == 0 || ndP == 0) return;
  const int tiles = (ndP + 63) / 64;
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (ti >= tiles || tj >= tiles) return;
  const int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  const size_t ldp = d.ldFp;
  T* M = static_cast<T*>(d.Fp) + (size_t)P * ldp * ldp;
  const int Dp = d.gp.D();
  for (int x = threadIdx.x; x < 64; x += blockDim.x) {
    int a = ti * 64 + x, b = tj * 64 + x;
    ra[x] = a < ndP ? tab[(size_t)a * TABW] : -1;
    cb[x] = b < ndP ? tab[(size_t)b * TABW] : -1;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 4 x 4 each
  T acc[4][4] = {};
  for (int j0 = 0; j0 < kp; j0 += 16) {
    for (int x = threadIdx.x; x < 64 * 16; x += blockDim.x) {
      int i = x % 64, j = x / 64;
      Zs[i][j] = (ra[i] >= 0 && j0 + j < kp) ? M[ra[i] + ldp * (Dp + j0 + j)] : T(0);
      int c = x % 64, jj = x / 64;
      Ws[jj][c] = (cb[c] >= 0 && j0 + jj < kp) ? M[(Dp + j0 + jj) + ldp * cb[c]] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      T z[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { z[u] = Zs[ty * 4 + u][j]; w[u] = Ws[j][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += z[u] * w[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = ty * 4 + u, c = tx * 4 + v;
      if (ra[i] >= 0 && cb[c] >= 0) M[ra[i] + ldp * cb[c]] -= acc[u][v];
    }
}

// The same update on the tensor cores (mixed path, schur_tc): 3xTF32 mma.sync (helpers above).
// 64 x 64 tile per CTA: warp w owns rows 16 (w % 4) .. +16 and columns 32 (w / 4) .. +32
// (four 16 x 8 accumulator tiles).
__global__ void __launch_bounds__(256) merge_schur_tc_kernel(LevelDev d) {
  __shared__ float Zs[64][17];
  __shared__ float Ws[16][65];
  __shared__ int ra[64], cb[64];
  const int P = blockIdx.z;
  const int ndP = d.pcount[2 * P], kp = d.pcount[2 * P + 1];
  if (kp == 0 || ndP == 0) return;
  const int tiles = (ndP + 63) / 64;
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (ti >= tiles || tj >= tiles) return;
  const int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  const size_t ldp = d.ldFp;
  float* M = static_cast<float*>(d.Fp) + (size_t)P * ldp * ldp;
  const int Dp = d.gp.D();
  for (int x = threadIdx.x; x < 64; x += blockDim.x) {
    int a = ti * 64 + x, b = tj * 64 + x;
    ra[x] = a < ndP ? tab[(size_t)a * TABW] : -1;
    cb[x] = b < ndP ? tab[(size_t)b * TABW] : -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int r0 = 16 * (warp & 3), c0 = 32 * (warp >> 2);
  float acc[4][4] = {};
  for (int j0 = 0; j0 < kp; j0 += 16) {
    for (int x = threadIdx.x; x < 64 * 16; x += blockDim.x) {
      int i = x % 64, j = x / 64;
      Zs[i][j] = (ra[i] >= 0 && j0 + j < kp) ? M[ra[i] + ldp * (Dp + j0 + j)] : 0.f;
      Ws[j][i] = (cb[i] >= 0 && j0 + j < kp) ? M[(Dp + j0 + j) + ldp * cb[i]] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t ah[4], al[4];
      split_tf32(Zs[r0 + g][8 * ks + q], ah[0], al[0]);
      split_tf32(Zs[r0 + g + 8][8 * ks + q], ah[1], al[1]);
      split_tf32(Zs[r0 + g][8 * ks + q + 4], ah[2], al[2]);
      split_tf32(Zs[r0 + g + 8][8 * ks + q + 4], ah[3], al[3]);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        uint32_t bh[2], bl[2];
        split_tf32(Ws[8 * ks + q][c0 + 8 * t + g], bh[0], bl[0]);
        split_tf32(Ws[8 * ks + q + 4][c0 + 8 * t + g], bh[1], bl[1]);
        mma_tf32(acc[t], al, bh);
        mma_tf32(acc[t], ah, bl);
        mma_tf32(acc[t], ah, bh);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = r0 + g + 8 * (u >> 1), c = c0 + 8 * t + 2 * q + (u & 1);
      if (ra[i] >= 0 && cb[c] >= 0) M[ra[i] + ldp * cb[c]] -= acc[t][u];
    }
}

// Level-(l-1) segment tables: counts and grid nodes (merged sides: [skel 1, junction, skel 2]).
__global__ void seg_merge_kernel(LevelDev d) {
  const Geo gp = d.gp, g = d.g;
  const int sidp = blockIdx.x;
  const bool horiz = sidp < gp.nh();
  int Ip, Jp;
  if (horiz) { Ip = sidp % gp.bx; Jp = sidp / gp.bx + 1; }
  else { int t = sidp - gp.nh(); Ip = t % (gp.bx - 1) + 1; Jp = t / (gp.bx - 1); }
  int* out = d.nodes_up + (size_t)sidp * d.capS_up;
  bool split = d.vcut ? horiz : !horiz;
  int cs1, cs2 = -1, jn = -1;
  if (!split) {
    // horizontal cut at level l: hs_p(Ip,Jp) -> hs(Ip, 2Jp); vertical cut: vs_p(Ip,Jp) -> vs(2Ip, Jp)
    if (horiz) cs1 = Ip + g.bx * (2 * Jp - 1);
    else cs1 = g.nh() + (2 * Ip - 1) + (g.bx - 1) * Jp;
  } else if (horiz) {   // vertical cut: hs_p(Ip,Jp) -> hs(2Ip,Jp), c(2Ip+1,Jp), hs(2Ip+1,Jp)
    cs1 = 2 * Ip + g.bx * (Jp - 1);
    cs2 = 2 * Ip + 1 + g.bx * (Jp - 1);
    jn = g.junction_node((2 * Ip + 1 - 1) + (g.bx - 1) * (Jp - 1), d.nx);
  } else {              // horizontal cut: vs_p(Ip,Jp) -> vs(Ip,2Jp), c(Ip,2Jp+1), vs(Ip,2Jp+1)
    cs1 = g.nh() + (Ip - 1) + (g.bx - 1) * (2 * Jp);
    cs2 = g.nh() + (Ip - 1) + (g.bx - 1) * (2 * Jp + 1);
    jn = g.junction_node((Ip - 1) + (g.bx - 1) * (2 * Jp + 1 - 1), d.nx);
  }
  const int k1 = d.kk[cs1];
  for (int t = threadIdx.x; t < k1; t += blockDim.x)
    out[t] = d.nodes[(size_t)cs1 * d.capS + d.perm[(size_t)cs1 * d.capS + t]];
  int n = k1;
  if (cs2 >= 0) {
    if (threadIdx.x == 0) out[n] = jn;
    ++n;
    const int k2 = d.kk[cs2];
    for (int t = threadIdx.x; t < k2; t += blockDim.x)
      out[n + t] = d.nodes[(size_t)cs2 * d.capS + d.perm[(size_t)cs2 * d.capS + t]];
    n += k2;
  }
  if (threadIdx.x == 0) d.cnt_up[sidp] = n;
}

// ------------------------------------------------------------ solve
constexpr int SC = 16;      // right-hand sides per solve pass (register accumulators per thread)
constexpr int DCAP = 512;   // parent boundaries up to this size are staged in shared memory

// out(a, c, acc) for a < nout, c < nc with acc = sum_j A(a, j) v[j + ldv c]: one thread per
// (row, right-hand side) pair, so that short products (a few rows, as in the finest levels)
// still spread over the CTA; v is read from shared memory, A from shared or global memory.
template <typename T, class Row, class Out>
__device__ __forceinline__ void gemv_pairs(int nout, int nin, Row row, size_t sj, const T* v, int ldv, int nc,
                                           Out out) {
  for (int x = threadIdx.x; x < nout * nc; x += blockDim.x) {
    const int a = x % nout, c = x / nout;
    const T* Aa = row(a);   // global or shared memory: plain (generic) loads
    const T* vc = v + (size_t)ldv * c;
    T acc = T(0);
#pragma unroll 4
    for (int j = 0; j < nin; ++j) acc += Aa[j * sj] * vc[j];
    out(a, c, acc);
  }
}

// Triangular sweeps on the SC columns held in shared memory (one warp per column).
template <typename T>
__device__ __forceinline__ void lower_sweep(T* y, int ldy, int n, const T* LU, size_t ldl, const int* pv, int nc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nw) {
    T* yy = y + (size_t)ldy * c;
    for (int j = 0; j < n; ++j) {
      const int p = pv[j];
      __syncwarp();
      if (p != j && lane == 0) { T t = yy[j]; yy[j] = yy[p]; yy[p] = t; }
      __syncwarp();
      const T yj = yy[j];
      for (int i = j + 1 + lane; i < n; i += 32) yy[i] -= LU[i + ldl * j] * yj;
    }
    __syncwarp();
  }
}

template <typename T>
__device__ __forceinline__ void upper_sweep(T* y, int ldy, int n, const T* LU, size_t ldl, const T* iv, int nc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < nc; c += nw) {
    T* yy = y + (size_t)ldy * c;
    for (int j = n - 1; j >= 0; --j) {
      __syncwarp();
      const T yj = yy[j] * iv[j];
      __syncwarp();
      if (lane == 0) yy[j] = yj;
      for (int i = lane; i < j; i += 32) yy[i] -= LU[i + ldl * j] * yj;
    }
    __syncwarp();
  }
}


// Triangular blocks of order up to INV_MAX are inverted after the factorization (factor
// kernels below), so that the solve applies them as one product per right-hand side instead of
// a sequential sweep: [L\U] becomes [L~^{-1}\U^{-1}] with L~ the multipliers after all later
// interchanges, and the pivot sequence becomes the permutation q, (P b)_i = b_{q_i}.
constexpr int INV_MAX = 64;

// v[:, c] = L~^{-1} v[q, c] (lower) or U^{-1} v[:, c] (upper) for c < nc, n <= INV_MAX, A the
// inverted block (ld lda) in shared or global memory.  NT threads (the CTA), each holding at
// most INV_MAX x 16 / NT outputs.
template <typename T, bool LOWER, int NT = 256>
__device__ __forceinline__ void tri_apply(T* v, int ldv, int n, const T* A, size_t lda, const int* q, int nc) {
  constexpr int PER = (INV_MAX * 16 + NT - 1) / NT;   // outputs per thread (nc <= 16)
  T acc[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int x = threadIdx.x + NT * t;
    acc[t] = T(0);
    if (x < n * nc) {
      const int i = x % n, c = x / n;
      const T* vc = v + (size_t)ldv * c;
      T s;
      if constexpr (LOWER) {
        s = vc[q[i]];
        for (int k = 0; k < i; ++k) s += A[i + lda * k] * vc[q[k]];
      } else {
        s = T(0);
        for (int k = i; k < n; ++k) s += A[i + lda * k] * vc[k];
      }
      acc[t] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int x = threadIdx.x + NT * t;
    if (x < n * nc) v[(x % n) + (size_t)ldv * (x / n)] = acc[t];
  }
  __syncthreads();
}

// In place on one GEPP block (n <= INV_MAX, column-major, ld lda; interchanges not applied to
// earlier multipliers; rinv the reciprocal pivots): thread j moves column j's multipliers
// through the later interchanges, then forms column j of L~^{-1} (below the diagonal) and of
// U^{-1} (on and above it) from a shared-memory copy.  S and X: n * n each; q: n.
template <typename T>
__device__ void invert_lu_block(T* A, size_t lda, int n, const T* rinv, int* piv, T* S, T* X, int* q) {
  for (int x = threadIdx.x; x < n * n; x += blockDim.x) S[x] = A[(x % n) + lda * (x / n)];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) q[i] = i;
    for (int j = 0; j < n; ++j) { const int p = piv[j], t = q[j]; q[j] = q[p]; q[p] = t; }
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    T* sc = S + (size_t)n * j;
    for (int t = j + 1; t < n; ++t) {
      const int p = piv[t];
      if (p != t) { const T a = sc[t]; sc[t] = sc[p]; sc[p] = a; }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    T* xc = X + (size_t)n * j;
    for (int i = j + 1; i < n; ++i) {          // L~ x = e_j (unit diagonal)
      T s = S[i + (size_t)n * j];
      for (int m = j + 1; m < i; ++m) s += S[i + (size_t)n * m] * xc[m];
      xc[i] = -s;
    }
    xc[j] = rinv[j];                           // U x = e_j
    for (int i = j - 1; i >= 0; --i) {
      T s = T(0);
      for (int m = i + 1; m <= j; ++m) s += S[i + (size_t)n * m] * xc[m];
      xc[i] = -s * rinv[i];
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n * n; x += blockDim.x) A[(x % n) + lda * (x / n)] = X[x];
  for (int i = threadIdx.x; i < n; i += blockDim.x) piv[i] = q[i];
}

template <typename T>
__device__ __forceinline__ void gather_panel(T* dst, int nr, int ncl, const T* src, size_t ldsrc,
                                             const int* rowidx, size_t colbase) {
  // dst[i + nr * j] = src[rowidx(i) + ldsrc * (colbase + j)]; independent loads, coalesced per column
  for (int x = threadIdx.x; x < nr * ncl; x += blockDim.x) {
    const int i = x % nr, j = x / nr;
    dst[x] = src[(size_t)rowidx[i] + ldsrc * (colbase + j)];
  }
}

// Inverse of each segment's remainder block (after the level's sparsification).
template <typename T>
__global__ void __launch_bounds__(64) seg_invert_kernel(LevelDev d) {
  extern __shared__ double ism[];
  const int sid = blockIdx.x;
  const int e = d.cnt[sid], k = d.kk[sid], r = e - k;
  if (r <= 0 || r > INV_MAX) return;
  const size_t capS = d.capS;
  T* S = reinterpret_cast<T*>(ism);
  T* X = S + (size_t)r * r;
  int* q = reinterpret_cast<int*>(X + (size_t)r * r);
  T* Dg = static_cast<T*>(d.Dm) + (size_t)sid * capS * capS;
  invert_lu_block<T>(Dg + k + capS * k, capS, r, static_cast<const T*>(d.Dinv) + (size_t)sid * capS,
                     d.piv + (size_t)sid * capS, S, X, q);
}

// Inverse of each parent's separator block (after its elimination in the merge).
template <typename T>
__global__ void __launch_bounds__(64) sep_invert_kernel(LevelDev d) {
  extern __shared__ double ism[];
  const int P = blockIdx.x;
  const int kp = d.pcount[2 * P + 1];
  if (kp <= 0 || kp > INV_MAX) return;
  const size_t ldp = d.ldFp;
  const int Dp = d.gp.D();
  T* S = reinterpret_cast<T*>(ism);
  T* X = S + (size_t)kp * kp;
  int* q = reinterpret_cast<int*>(X + (size_t)kp * kp);
  T* M = static_cast<T*>(d.Fp) + (size_t)P * ldp * ldp;
  invert_lu_block<T>(M + Dp + ldp * Dp, ldp, kp, static_cast<const T*>(d.Pinv) + (size_t)P * d.sepcap,
                     d.ppiv + (size_t)P * d.sepcap, S, X, q);
}

template <typename T>
size_t invert_smem() { return 2 * sizeof(T) * INV_MAX * INV_MAX + sizeof(int) * INV_MAX; }

// The right-hand sides of a launch are split into gridDim.y groups (one CTA per group and
// segment or separator: more CTAs where a level has few segments); this CTA's group becomes
// columns 0 .. nc-1 of X.  False when the group is empty.
template <typename T>
__device__ __forceinline__ bool rhs_group(T*& X, int& nc, const VecLayout& lay) {
  const int per = (nc + (int)gridDim.y - 1) / (int)gridDim.y, c0 = (int)blockIdx.y * per;
  if (c0 >= nc) return false;
  X += (size_t)c0 * (size_t)lay.cs;
  nc = nc - c0 < per ? nc - c0 : per;
  return true;
}

// Forward, per segment: b_r -= T^T b_s; y_r = L^{-1} P b_r; b_s -= Z y_r.
// Backward, per segment: x_r = U^{-1} (y_r - W x_s); x_s -= T x_r.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 16) seg_solve_kernel(LevelDev d, SolveCaps cap, T* X, int nc, VecLayout lay, int bwd) {
  pdl_trigger();
  extern __shared__ double smd[];
  if (!rhs_group(X, nc, lay)) return;
  const int sid = blockIdx.x;
  const int e = d.cnt[sid], k = d.kk[sid], r = e - k;
  if (r == 0 || e == 0) return;
  if (e > cap.vrows) { if (threadIdx.x == 0) atomicOr(d.err, ERR_CAPACITY); return; }
  const int capS = d.capS;
  T* v = reinterpret_cast<T*>(smd);                      // e x SC, [skeleton | remainder]
  T* LUsm = v + (size_t)cap.vrows * SC;                  // r x r LU (when r <= lucap)
  T* Psm = LUsm + (size_t)cap.lucap * cap.lucap;         // two k x r panels (when k r <= pcap)
  T* invs = Psm + 2 * (size_t)cap.pcap;
  int* pivs = reinterpret_cast<int*>(invs + cap.lucap);
  int* nds = pivs + cap.lucap;                           // the segment's nodes (vrows)
  const bool staged = r <= cap.lucap;
  const bool pstaged = (size_t)k * r <= (size_t)cap.pcap;
  const int* snodes = d.snodes + (size_t)sid * capS;     // nodes in [skeleton | remainder] order
  const int* piv = d.piv + (size_t)sid * capS;
  const T* Tm = static_cast<const T*>(d.T) + (size_t)sid * capS * capS;
  const T* Dg = static_cast<const T*>(d.Dm) + (size_t)sid * capS * capS;
  const T* inv = static_cast<const T*>(d.Dinv) + (size_t)sid * capS;
  // factor data first (it overlaps the preceding kernel), the right-hand side after the wait
  if (staged) {
    for (int x = threadIdx.x; x < r * r; x += blockDim.x)
      LUsm[x] = Dg[(k + x % r) + (size_t)capS * (k + x / r)];
    for (int x = threadIdx.x; x < r; x += blockDim.x) { invs[x] = inv[x]; pivs[x] = piv[x]; }
  }
  // panels: T (k x r, ld capS) and Z = D[0:k, k:e] (forward) or W = D[k:e, 0:k] (backward)
  T* Ts = Psm;              // k x r, ld k
  T* Ps = Psm + cap.pcap;   // forward: Z as k x r (ld k); backward: W as r x k (ld r)
  if (pstaged && k > 0) {
    for (int x = threadIdx.x; x < k * r; x += blockDim.x) {
      const int i = x % k, j = x / k;
      Ts[x] = Tm[i + (size_t)capS * j];
      if (!bwd) Ps[x] = Dg[i + (size_t)capS * (k + j)];
    }
    if (bwd)
      for (int x = threadIdx.x; x < r * k; x += blockDim.x) Ps[x] = Dg[(k + x % r) + (size_t)capS * (x / r)];
  }
  for (int a = threadIdx.x; a < e; a += blockDim.x) nds[a] = snodes[a];
  __syncthreads();
  pdl_wait();
  for (int x = threadIdx.x; x < e * nc; x += blockDim.x) {
    int a = x % e, c = x / e;
    v[x] = X[lay.at(nds[a], c)];
  }
  __syncthreads();
  const T* LUs = staged ? LUsm : Dg + k + (size_t)capS * k;
  const size_t ldl = staged ? (size_t)r : (size_t)capS;
  const T* ivs = staged ? invs : inv;
  const int* pvs = staged ? pivs : piv;
  const T* Tp = pstaged ? Ts : Tm;
  const size_t ldt = pstaged ? (size_t)k : (size_t)capS;
  T* vs = v;          // skeleton part
  T* vr = v + k;      // remainder part
  if (!bwd) {
    if (k > 0) {      // b_r -= T^T b_s: row a of T^T is column a of T
      gemv_pairs<T>(r, k, [&](int a) { return Tp + ldt * a; }, 1, vs, e, nc,
                    [&](int a, int c, T acc) { vr[a + e * c] -= acc; });
      __syncthreads();
    }
    if (r <= INV_MAX) tri_apply<T, true, NT>(vr, e, r, LUs, ldl, pvs, nc);
    else lower_sweep<T>(vr, e, r, LUs, ldl, pvs, nc);
    __syncthreads();
    if (k > 0) {      // b_s -= Z y_r
      const T* Zp = pstaged ? Ps : Dg + (size_t)capS * k;
      const size_t ldz = pstaged ? (size_t)k : (size_t)capS;
      gemv_pairs<T>(k, r, [&](int a) { return Zp + a; }, ldz, vr, e, nc,
                    [&](int a, int c, T acc) { vs[a + e * c] -= acc; });
    }
  } else {
    if (k > 0) {      // y_r -= W x_s
      const T* Wp = pstaged ? Ps : Dg + k;
      const size_t ldw = pstaged ? (size_t)r : (size_t)capS;
      gemv_pairs<T>(r, k, [&](int a) { return Wp + a; }, ldw, vs, e, nc,
                    [&](int a, int c, T acc) { vr[a + e * c] -= acc; });
      __syncthreads();
    }
    if (r <= INV_MAX) tri_apply<T, false, NT>(vr, e, r, LUs, ldl, pvs, nc);
    else upper_sweep<T>(vr, e, r, LUs, ldl, ivs, nc);
    __syncthreads();
    if (k > 0) {      // x_s -= T x_r
      gemv_pairs<T>(k, r, [&](int a) { return Tp + a; }, ldt, vr, e, nc,
                    [&](int a, int c, T acc) { vs[a + e * c] -= acc; });
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < e * nc; x += blockDim.x) {
    int a = x % e, c = x / e;
    X[lay.at(nds[a], c)] = v[x];
  }
}

// Separator of each parent: forward y_p = L^{-1} P b_p, then b_dP -= Z y_p added atomically
// (a boundary unknown is shared by up to four parents; the order of their contributions is
// not fixed); backward x_p = U^{-1} (y_p - W x_dP).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 16) sep_solve_kernel(LevelDev d, SolveCaps cap, T* X, int nc, VecLayout lay, int bwd) {
  pdl_trigger();
  extern __shared__ double smd[];
  if (!rhs_group(X, nc, lay)) return;
  const int P = blockIdx.x;
  const int ndP = d.pcount[2 * P], kp = d.pcount[2 * P + 1];
  if (kp == 0) return;
  if (kp > cap.yrows) { if (threadIdx.x == 0) atomicOr(d.err, ERR_CAPACITY); return; }
  const int* tab = d.ptab + (size_t)P * d.ldFp * TABW;
  const size_t ldp = d.ldFp;
  const T* M = static_cast<const T*>(d.Fp) + (size_t)P * ldp * ldp;
  const T* inv = static_cast<const T*>(d.Pinv) + (size_t)P * d.sepcap;
  const int Dp = d.gp.D();
  const int* piv = d.ppiv + (size_t)P * d.sepcap;
  const int ub = cap.lucap * cap.lucap > cap.qcap ? cap.lucap * cap.lucap : cap.qcap;
  T* y = reinterpret_cast<T*>(smd);                     // kp x SC
  T* U = y + (size_t)cap.yrows * SC;                    // union: LU block / panel
  T* xd = U + ub;                                       // drows x SC (backward)
  T* invs = xd + (size_t)cap.drows * SC;
  int* pivs = reinterpret_cast<int*>(invs + cap.lucap);
  int* rows_sm = pivs + cap.lucap;                      // 2 * drows
  int* ynode = rows_sm + 2 * cap.drows;                 // the separator skeleton's nodes (yrows)
  const bool staged = kp <= cap.lucap;
  const bool dstage = ndP <= cap.drows;
  const int ldw = ndP | 1;                              // odd pitch of the staged W^T panel
  const bool pstaged = dstage && (size_t)ldw * kp <= (size_t)cap.qcap;
  if (dstage) {
    for (int x = threadIdx.x; x < ndP; x += blockDim.x) {
      rows_sm[x] = tab[(size_t)x * TABW];
      rows_sm[cap.drows + x] = tab[(size_t)x * TABW + 7];
    }
  }
  auto rowpos = [&](int a) { return dstage ? rows_sm[a] : tab[(size_t)a * TABW]; };
  auto rownode = [&](int a) { return dstage ? rows_sm[cap.drows + a] : tab[(size_t)a * TABW + 7]; };
  if (staged) for (int x = threadIdx.x; x < kp; x += blockDim.x) { invs[x] = inv[x]; pivs[x] = piv[x]; }
  for (int a = threadIdx.x; a < kp; a += blockDim.x) ynode[a] = tab[(size_t)(ndP + a) * TABW + 7];
  const size_t ldl = staged ? (size_t)kp : ldp;
  const T* ivs = staged ? invs : inv;
  const int* pvs = staged ? pivs : piv;
  auto stage_lu = [&]() {
    if (staged)
      for (int x = threadIdx.x; x < kp * kp; x += blockDim.x) U[x] = M[(Dp + x % kp) + ldp * (Dp + x / kp)];
  };
  // factor data first (it overlaps the preceding kernel): the LU block (forward) or the W^T
  // panel (backward); the solve vector after the wait
  T* Wt = U;                                            // W^T panel, pitch ldw
  if (!bwd) stage_lu();
  else if (pstaged) {
    __syncthreads();                                    // rows_sm
    for (int x = threadIdx.x; x < ndP * kp; x += blockDim.x) {
      const int j = x % kp, b = x / kp;
      Wt[b + (size_t)ldw * j] = M[(Dp + j) + ldp * rows_sm[b]];
    }
  }
  __syncthreads();          // ynode, rows_sm
  pdl_wait();
  for (int x = threadIdx.x; x < kp * nc; x += blockDim.x) {
    int a = x % kp, c = x / kp;
    y[x] = X[lay.at(ynode[a], c)];
  }
  __syncthreads();          // y (and the LU block) are read by other threads below
  if (!bwd) {
    if (kp <= INV_MAX) tri_apply<T, true, NT>(y, kp, kp, staged ? U : M + Dp + ldp * Dp, ldl, pvs, nc);
    else lower_sweep<T>(y, kp, kp, staged ? U : M + Dp + ldp * Dp, ldl, pvs, nc);
    __syncthreads();
    // b_dP -= Z y_p, Z = M[dP rows, separator columns]
    if (pstaged) {
      gather_panel<T>(U, ndP, kp, M, ldp, rows_sm, Dp);
      __syncthreads();
    }
    gemv_pairs<T>(ndP, kp,
                  [&](int a) { return pstaged ? U + a : M + rowpos(a) + ldp * Dp; },
                  pstaged ? (size_t)ndP : ldp, y, kp, nc,
                  [&](int a, int c, T acc) { atomicAdd(X + lay.at(rownode(a), c), -acc); });
  } else {
    if (dstage) {
      for (int x = threadIdx.x; x < ndP * nc; x += blockDim.x) {
        int b = x % ndP, c = x / ndP;
        xd[x] = X[lay.at(rows_sm[cap.drows + b], c)];
      }
    }
    __syncthreads();
    // y_p -= W x_dP, one thread per (row a, right-hand side c)
    for (int x = threadIdx.x; x < kp * nc; x += blockDim.x) {
      const int a = x % kp, c = x / kp;
      T acc = T(0);
      if (pstaged) {
        const T* wa = Wt + (size_t)ldw * a;
        const T* xc = xd + (size_t)ndP * c;
#pragma unroll 4
        for (int b = 0; b < ndP; ++b) acc += wa[b] * xc[b];
      } else if (dstage) {
        const T* xc = xd + (size_t)ndP * c;
        for (int b = 0; b < ndP; ++b) acc += M[(Dp + a) + ldp * rows_sm[b]] * xc[b];
      } else {
        for (int b = 0; b < ndP; ++b) acc += M[(Dp + a) + ldp * rowpos(b)] * X[lay.at(rownode(b), c)];
      }
      y[a + kp * c] -= acc;
    }
    __syncthreads();
    stage_lu();             // the panel is consumed: U takes the LU block
    __syncthreads();
    if (kp <= INV_MAX) tri_apply<T, false, NT>(y, kp, kp, staged ? U : M + Dp + ldp * Dp, ldl, pvs, nc);
    else upper_sweep<T>(y, kp, kp, staged ? U : M + Dp + ldp * Dp, ldl, ivs, nc);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < kp * nc; x += blockDim.x) {
    int a = x % kp, c = x / kp;
    X[lay.at(ynode[a], c)] = y[x];
  }
}


}  // namespace

size_t sparsify_smem_need(int e, int symmetric, int h0, int p_over, int tbytes, int chunk) {
  const size_t halves = symmetric ? 1 : 2;
  const size_t hcap = (size_t)(h0 > 2 * (e + p_over) ? h0 : 2 * (e + p_over));
  const size_t mmax = halves * NEAR_MAX + hcap;
  const size_t small_b = 2 * (size_t)e * 8 + (3 * (size_t)e + 4) * 4 + (size_t)e * tbytes + 64;
  // segments of at most 32 unknowns also stage their B block (<= 6 sides of e + 8 corners)
  const size_t bs = e <= 32 ? halves * (6 * (size_t)e + 8) * e + 4 : 0;
  return small_b + ((size_t)chunk * halves * (e + hcap) + (mmax + 1) * e + 2 * (size_t)e * e + bs) * tbytes;
}

size_t sparsify_smem_min(int e, int symmetric, int h0, int p_over, int tbytes) {
  const size_t halves = symmetric ? 1 : 2;
  const size_t hcap = (size_t)(h0 > 2 * (e + p_over) ? h0 : 2 * (e + p_over));
  return 2 * (size_t)e * 8 + (3 * (size_t)e + 4) * 4 + (size_t)e * tbytes + 64 + halves * (e + hcap) * tbytes;
}

int sm_count() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

size_t sparsify_smem_budget(int fp32, int capS, int ctas) {
  if (ctas < 1) return 0;
  int dev = 0, per_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaFuncAttributes fa{};
  cudaError_t e;
  const int threads = (capS <= 16 ? NW_SMALL : NW) * 32;
  if (capS <= 16)
    e = fp32 ? cudaFuncGetAttributes(&fa, sparsify_kernel<float, NW_SMALL>)
             : cudaFuncGetAttributes(&fa, sparsify_kernel<double, NW_SMALL>);
  else
    e = fp32 ? cudaFuncGetAttributes(&fa, sparsify_kernel<float, NW>)
             : cudaFuncGetAttributes(&fa, sparsify_kernel<double, NW>);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  // no more CTAs than the register file holds: shared memory beyond that buys nothing
  const int regs = fa.numRegs > 0 ? fa.numRegs : 64;
  const int by_regs = 65536 / (regs * threads);
  if (by_regs >= 1 && ctas > by_regs) ctas = by_regs;
  const long long share = ((long long)per_sm / ctas) & ~255LL;   // allocation granularity
  const long long dyn = share - reserved - (long long)fa.sharedSizeBytes;
  return dyn > 0 ? (size_t)(dyn & ~255LL) : 0;
}

void launch_level_init_L(const LevelDev& d, cudaStream_t s) {
  int n = d.g.nseg() * LEAF;
  if (n == 0) return;
  note_launch();
  level_init_L_kernel<<<(n + 255) / 256, 256, 0, s>>>(d);
}

template <typename T>
static void sparsify_launch(const LevelDev& d, const LevelPlan& p, cudaStream_t s) {
  int smem = (int)p.spars_smem;
  if (d.use_order && d.g.nseg() > 0) {
    note_launch();
    seg_order_kernel<<<1, 1024, 0, s>>>(d.cnt, d.g.nseg(), d.order);
  }
  note_launch();
  if (d.capS <= 16) {       // finest segments: two warps each, many segments per SM
    cudaFuncSetAttribute(sparsify_kernel<T, NW_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sparsify_kernel<T, NW_SMALL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    sparsify_kernel<T, NW_SMALL><<<d.g.nseg(), NW_SMALL * 32, smem, s>>>(d, smem);
  } else {
    cudaFuncSetAttribute(sparsify_kernel<T, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sparsify_kernel<T, NW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    sparsify_kernel<T, NW><<<d.g.nseg(), NW * 32, smem, s>>>(d, smem);
  }
  const int ism = (int)invert_smem<T>();
  cudaFuncSetAttribute(seg_invert_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, ism);
  note_launch();
  seg_invert_kernel<T><<<d.g.nseg(), 64, ism, s>>>(d);
}

void launch_sparsify(const LevelDev& d, const LevelPlan& p, cudaStream_t s) {
  if (d.g.nseg() == 0) return;
  if (d.fp32) sparsify_launch<float>(d, p, s);
  else sparsify_launch<double>(d, p, s);
}

template <typename T>
static void merge_launch(const LevelDev& d, const LevelPlan& p, cudaStream_t s) {
  const int np = d.gp.nbox();
  note_launch();
  merge_table_kernel<<<np, 128, 0, s>>>(d);
  {
    long long nmax = (long long)p.ldFp;
    int gx = (int)((nmax * nmax + 255) / 256);
    if (gx > 256) gx = 256;
    dim3 grid(gx, np);
    note_launch();
    merge_assemble_kernel<T><<<grid, 256, 0, s>>>(d);
  }
  {
    // shared memory for the staged separator rows: the geometric bound, at most 96 KB (larger
    // parents take the global-memory path inside the kernel)
    const size_t geo = (size_t)p.sepcap * p.ldFp * sizeof(T) + (size_t)p.ldFp * sizeof(int);
    const int pm = (int)(geo < 96 * 1024 ? geo : 96 * 1024);
    note_launch();
    if (np <= 2 * sm_count()) {      // at most two parents per SM: latency-bound, rows in registers
      if (pm > 48 * 1024) cudaFuncSetAttribute(merge_panel_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pm);
      merge_panel_kernel<T, true><<<np, 256, pm, s>>>(d, pm);
    } else {
      if (pm > 48 * 1024) cudaFuncSetAttribute(merge_panel_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, pm);
      merge_panel_kernel<T, false><<<np, 256, pm, s>>>(d, pm);
    }
  }
  {
    const int ism = (int)invert_smem<T>();
    cudaFuncSetAttribute(sep_invert_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, ism);
    note_launch();
    sep_invert_kernel<T><<<np, 64, ism, s>>>(d);
  }
  {
    int tiles = (p.ldFp + 63) / 64;
    dim3 grid(tiles, tiles, np);
    note_launch();
    if (d.schur_tc && d.fp32) merge_schur_tc_kernel<<<grid, 256, 0, s>>>(d);
    else merge_schur_kernel<T><<<grid, 256, 0, s>>>(d);
  }
  if (d.l > 1 && d.gp.nseg() > 0) {
    note_launch();
    seg_merge_kernel<<<d.gp.nseg(), 128, 0, s>>>(d);
  }
}

void launch_merge(const LevelDev& d, const LevelPlan& p, cudaStream_t s) {
  if (d.fp32) merge_launch<float>(d, p, s);
  else merge_launch<double>(d, p, s);
}

bool level_solve_caps(const LevelDev& d, const int* lmax, SolveCaps* out) {
  // lmax: the level counters, LS_EMAX / LS_KPMAX / LS_DPMAX first
  auto mn = [](long long a, long long b) { return a < b ? a : b; };
  auto mx = [](long long a, long long b) { return a > b ? a : b; };
  const long long TB = d.fp32 ? 4 : 8, budget = 200 * 1024;
  SolveCaps sc{};
  sc.vrows = (int)mx(lmax[0], 1);
  sc.yrows = (int)mx(lmax[1], 1);
  sc.drows = (int)mn(lmax[2], DCAP);
  sc.lucap = (int)mn(mx(lmax[0], lmax[1]), RSTAGE);
  long long seg_fixed = 0, sep_fixed = 0;
  for (;;) {
    // segment: v, LU block, reciprocal pivots, pivots (panels come on top)
    seg_fixed = TB * ((long long)sc.vrows * SC + (long long)sc.lucap * sc.lucap + sc.lucap) +
                4LL * (sc.lucap + sc.vrows) + 16;
    // separator: y, xd, reciprocal pivots, pivots, boundary rows (the LU block / panel union on top)
    sep_fixed = TB * ((long long)sc.yrows * SC + (long long)sc.drows * SC + sc.lucap) +
                4LL * (sc.lucap + 2 * sc.drows + sc.yrows) + 16;
    const long long lu = TB * (long long)sc.lucap * sc.lucap;
    if (seg_fixed <= budget && sep_fixed + lu <= budget) break;
    if (sc.lucap > 8) sc.lucap /= 2;
    else if (sc.lucap > 0) sc.lucap = 0;
    else if (sc.drows > 0) sc.drows /= 2;
    else return false;              // the right-hand-side blocks alone exceed the budget
  }
  // a segment panel is k x r <= (e/2)^2; a separator panel |dP| x kp
  sc.pcap = (int)mx(0, mn((long long)(sc.vrows / 2 + 1) * (sc.vrows / 2 + 1), (budget - seg_fixed) / (2 * TB)));
  sc.qcap = (int)mx(0, mn((long long)(sc.drows | 1) * sc.yrows, (budget - sep_fixed) / TB));
  sc.seg_smem = (size_t)(seg_fixed + 2 * TB * sc.pcap);
  // CTA widths before any tuning: 2-warp segment CTAs where segments have at most 32 unknowns
  sc.seg_nt = d.capS <= 32 ? 64 : 256;
  sc.sep_nt = 256;
  sc.seg_split = sc.sep_split = 1;
  sc.sep_smem = (size_t)(sep_fixed + TB * mx((long long)sc.lucap * sc.lucap, sc.qcap));
  *out = sc;
  return true;
}

template <typename T>
static void level_solve(const LevelDev& d, const SolveCaps& sc, T* X, int nrhs, VecLayout lay, int bwd, cudaStream_t s) {
  cudaFuncSetAttribute(seg_solve_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.seg_smem);
  cudaFuncSetAttribute(seg_solve_kernel<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.seg_smem);
  cudaFuncSetAttribute(sep_solve_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.sep_smem);
  cudaFuncSetAttribute(sep_solve_kernel<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.sep_smem);
  for (int c0 = 0; c0 < nrhs; c0 += SC) {
    const int nc = nrhs - c0 < SC ? nrhs - c0 : SC;
    T* Xc = X + (size_t)(c0 / SC) * lay.chunk;
    auto seg_go = [&](int dir) {
      note_launch();
      const dim3 grid(d.g.nseg(), sc.seg_split < nc ? sc.seg_split : nc);
      if (sc.seg_nt == 64)  // 2-warp CTAs: four times as many resident per SM
        launch_pdl(seg_solve_kernel<T, 64>, grid, dim3(64), sc.seg_smem, s, d, sc, Xc, nc, lay, dir);
      else
        launch_pdl(seg_solve_kernel<T, 256>, grid, dim3(256), sc.seg_smem, s, d, sc, Xc, nc, lay, dir);
    };
    auto sep_go = [&](int dir) {
      note_launch();
      const dim3 grid(d.gp.nbox(), sc.sep_split < nc ? sc.sep_split : nc);
      if (sc.sep_nt == 64)
        launch_pdl(sep_solve_kernel<T, 64>, grid, dim3(64), sc.sep_smem, s, d, sc, Xc, nc, lay, dir);
      else
        launch_pdl(sep_solve_kernel<T, 256>, grid, dim3(256), sc.sep_smem, s, d, sc, Xc, nc, lay, dir);
    };
    if (!bwd) {
      if (d.g.nseg() > 0) seg_go(0);
      sep_go(0);
    } else {
      sep_go(1);
      if (d.g.nseg() > 0) seg_go(1);
    }
  }
}

void launch_level_solve_fwd(const LevelDev& d, const SolveCaps& c, void* X, int nrhs, VecLayout lay, cudaStream_t s) {
  if (d.fp32) level_solve<float>(d, c, static_cast<float*>(X), nrhs, lay, 0, s);
  else level_solve<double>(d, c, static_cast<double*>(X), nrhs, lay, 0, s);
}

void launch_level_solve_bwd(const LevelDev& d, const SolveCaps& c, void* X, int nrhs, VecLayout lay, cudaStream_t s) {
  if (d.fp32) level_solve<float>(d, c, static_cast<float*>(X), nrhs, lay, 1, s);
  else level_solve<double>(d, c, static_cast<double*>(X), nrhs, lay, 1, s);
}

}  // namespace spalu
