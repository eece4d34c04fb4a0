// Leaf-interior elimination (Sec. 4.3, first step: L_(L+1)^{-1} A U_(L+1)^{-1} = diag(I, A^(L)))
// and the leaf part of the tree-ordered solve (Eq. (WV)).
//
// The 225 x 225 interior block A_II of a 15 x 15 leaf is banded in the natural in-leaf order
// (x fastest, lower and upper bandwidth 15).  Gaussian elimination with partial pivoting
// (pivot = largest |a_ij| in the column, ties -> lowest row) runs in LAPACK band storage
// (kl = ku = 15, 46 rows incl. the fill of the row interchanges) in FP64: it performs exactly
// the operations of dense partial-pivoting LU on the nonzeros.  The Schur complement
// S_b = A_dI A_II^{-1} A_Id onto the 60 side unknowns needs A_II^{-1} only at the ring of
// interior nodes next to the sides (every side unknown couples to one interior node), so it
// comes from 60 solves with unit right-hand sides.
//
// GB300 mapping: FP64 runs at 2 FMA per clock per SM, so every FP64 warp instruction must
// carry 32 useful lanes.  The solves therefore give one thread to one (leaf, right-hand side)
// column and sweep the band with a register window (the interchanges stay inside it); the
// reciprocal pivots are stored once, and the upper sweep runs at the bandwidth the
// interchanges actually produced (15 when there were none).
#include <cstdio>

#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int KV = KL + KU;   // row of the diagonal in band storage
constexpr int NQ = 4 * LEAF;  // side unknowns of a leaf
constexpr int LPC = 2;        // leaves per CTA of the factor kernel
constexpr int FTH = 128;      // threads of the factor kernel (64 per leaf)
constexpr int QL = 64;        // column slots per leaf in the sweep buffer (60 used by the factor)

__device__ __forceinline__ int leaf_frontal_pos(int vx, int vy, int x0, int y0) {
  const int w = LEAF;
  if (vy == y0 - 1 && vx >= x0 && vx < x0 + w) return vx - x0;                  // bottom
  if (vy == y0 + w && vx >= x0 && vx < x0 + w) return w + vx - x0;              // top
  if (vx == x0 - 1 && vy >= y0 && vy < y0 + w) return 2 * w + vy - y0;          // left
  if (vx == x0 + w && vy >= y0 && vy < y0 + w) return 3 * w + vy - y0;          // right
  if (vx == x0 - 1 && vy == y0 - 1) return 4 * w + C_BL;
  if (vx == x0 + w && vy == y0 - 1) return 4 * w + C_BR;
  if (vx == x0 - 1 && vy == y0 + w) return 4 * w + C_TL;
  if (vx == x0 + w && vy == y0 + w) return 4 * w + C_TR;
  return -1;
}

// side unknown q (0..59: BOTTOM, TOP, LEFT, RIGHT, 15 each): grid node and the local index of
// its interior neighbour
__device__ __forceinline__ void side_unknown(int q, int x0, int y0, int* vx, int* vy, int* m) {
  int s = q / LEAF, t = q % LEAF;
  switch (s) {
    case SIDE_BOTTOM: *vx = x0 + t; *vy = y0 - 1; *m = t; break;
    case SIDE_TOP: *vx = x0 + t; *vy = y0 + LEAF; *m = t + LEAF * (LEAF - 1); break;
    case SIDE_LEFT: *vx = x0 - 1; *vy = y0 + t; *m = LEAF * t; break;
    default: *vx = x0 + LEAF; *vy = y0 + t; *m = LEAF * t + LEAF - 1; break;
  }
}

__device__ __forceinline__ double csr_entry(const int* rowptr, const int* colind, const double* val, int r, int c) {
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p)
    if (colind[p] == c) return val[p];
  return 0.0;
}

// side unknowns ordered by the position of their interior neighbour (so that the solves of
// one warp can start late: L^{-1} P e_m vanishes above row m - 15)
__constant__ int c_qorder[NQ];
__constant__ int c_qstart[2];   // first sweep step of the two solve warps of a leaf

// Read-only view of one leaf's factors in precision T: RO = true reads global memory through
// the read-only path (factors written by an earlier kernel); false reads plain (shared) memory.
template <typename T, bool RO>
struct Band {
  const T* __restrict__ ab;     // LDAB x NI
  const int* __restrict__ piv;
  const T* __restrict__ invd;
  __device__ __forceinline__ T ld(const T* q) const { if constexpr (RO) return __ldg(q); else return *q; }
  __device__ __forceinline__ T l(int r, int j) const { return ld(ab + (KV + r) + LDAB * j); }   // L(j+r, j)
  __device__ __forceinline__ T u(int r, int j) const { return ld(ab + (KV - r) + LDAB * j); }   // U(j-r, j)
  __device__ __forceinline__ int p(int j) const { if constexpr (RO) return __ldg(piv + j); else return piv[j]; }
  __device__ __forceinline__ T dinv(int j) const { return ld(invd + j); }
};

// Forward sweep y = L^{-1} P x for one column held by this thread.  in(j) gives x_j,
// out(j, y) receives y_j for j = j0..NI-1 (x_j = 0 for j < j0 is assumed).
template <typename T, class BandT, class In, class Out>
__device__ __forceinline__ void sweep_L(const BandT& B, int j0, In in, Out out) {
  T W[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) W[r] = (j0 + r < NI) ? in(j0 + r) : T(0);
  for (int t0 = 0; j0 + t0 < NI; t0 += 16) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int j = j0 + t0 + u;
      if (j < NI) {
        const int dsw = B.p(j) - j;     // 0..15: the interchange stays in the window
        T a = W[u], b = a;
        if (__any_sync(__activemask(), dsw != 0)) {   // skipped when no lane interchanges
#pragma unroll
          for (int r = 1; r < 16; ++r)
            if (r == dsw) { b = W[(u + r) & 15]; W[(u + r) & 15] = a; }
          W[u] = b;
        }
#pragma unroll
        for (int r = 1; r < 16; ++r) W[(u + r) & 15] -= B.l(r, j) * b;
        out(j, b);
        W[u] = (j + 16 < NI) ? in(j + 16) : T(0);
      }
    }
  }
}

// Backward sweep x = U^{-1} y (upper bandwidth < KUW) for one column: in(j) gives y_j,
// out(j, x) receives x_j for j = NI-1 .. 0.
template <typename T, int KUW, class BandT, class In, class Out>
__device__ __forceinline__ void sweep_U(const BandT& B, In in, Out out) {
  T V[KUW];
#pragma unroll
  for (int r = 0; r < KUW; ++r) V[r] = (NI - 1 - r >= 0) ? in(NI - 1 - r) : T(0);
  constexpr int RMAX = KUW - 1 < KV ? KUW - 1 : KV;
  for (int t0 = 0; t0 < NI; t0 += KUW) {
#pragma unroll
    for (int u = 0; u < KUW; ++u) {
      const int t = t0 + u;
      if (t < NI) {
        const int j = NI - 1 - t;
        const T x = V[u] * B.dinv(j);
        out(j, x);
#pragma unroll
        for (int r = 1; r <= RMAX; ++r) V[(u + r) & (KUW - 1)] -= B.u(r, j) * x;
        V[u] = (j - KUW >= 0) ? in(j - KUW) : T(0);
      }
    }
  }
}

// ---- leaf factorization, kernel A: band LU (the dgbtf2 sequence: pivot = largest |entry| of
// the column inside the band, ties -> lowest row; interchanges applied to the columns the U
// factor can reach; multipliers scaled by the reciprocal pivot) of one leaf per 64-thread
// CTA, in FP64, on a sliding window of WS band columns in shared memory: column c sits in
// slot c mod WS; after step j column j is final, goes to global memory in precision T and its
// slot is refilled with column j + WS assembled from the CSR (first touched at step j + 2).
// Also zeroes the leaf's frontal block and records the upper bandwidth reached.
constexpr int WS = 32;       // window columns (> KV)
constexpr int LUT = 64;      // threads per leaf LU

template <typename T>
__global__ void __launch_bounds__(LUT) leaf_lu_kernel(LeafDev d) {
  __shared__ double W[LDAB * WS];
  __shared__ int sh[2];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const Geo g = d.g;
  const int I = b % g.bx, J = b / g.bx;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  {
    T* F = reinterpret_cast<T*>(d.F) + (size_t)b * d.ldF * d.ldF;
    const int D = g.D();
    for (int e = tid; e < D * D; e += LUT) F[(e % D) + (size_t)d.ldF * (e / D)] = T(0);
  }
  T* bandg = reinterpret_cast<T*>(d.band) + (size_t)b * LDAB * NI;
  T* invg = reinterpret_cast<T*>(d.invd) + (size_t)b * NI;
  int* pivg = d.piv + (size_t)b * NI;
  auto node_of = [&](int j) { return (x0 + j % LEAF) + nx * (y0 + j / LEAF); };
  // band row r of column c of A_II from the CSR: A(i, c), i = c + r - KV (5-point stencil)
  auto assemble = [&](int r, int c) -> double {
    const int i = c + r - KV;
    if (c >= NI || i < 0 || i >= NI) return 0.0;
    const int di = i - c;
    const bool adj = di == 0 || di == LEAF || di == -LEAF || ((di == 1 || di == -1) && i / LEAF == c / LEAF);
    if (!adj) return 0.0;
    return csr_entry(d.rowptr, d.colind, d.val, node_of(i), node_of(c));
  };
  auto w = [&](int i, int c) -> double& { return W[(KV + i - c) + LDAB * (c & (WS - 1))]; };
  for (int x = tid; x < LDAB * WS; x += LUT) W[x] = assemble(x % LDAB, x / LDAB);
  __syncthreads();
  int ju = 0, kureach = KU;
  bool ok = true;
  const int ur = 1 + (tid & 15), ucg = tid >> 4;       // rank-1 update: row, column group
  for (int j = 0; j < NI; ++j) {
    const int km = min(KL, NI - 1 - j);
    if (tid < 32) {           // pivot: |entries| compared as bit patterns (no FP64 arithmetic)
      long long best = -1;
      int bi = 0;
      if (lane <= km) { best = __double_as_longlong(w(j + lane, j)) & 0x7fffffffffffffffll; bi = lane; }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        sh[0] = bi;
        sh[1] = best == 0 ? 1 : 0;
        pivg[j] = j + bi;
      }
    }
    __syncthreads();
    const int jp = sh[0];
    const bool zero = sh[1] != 0;
    if (zero) ok = false;
    ju = max(ju, min(j + KU + jp, NI - 1));
    kureach = max(kureach, ju - j);
    if (!zero && jp != 0)
      for (int c = j + tid; c <= ju; c += LUT) {
        const double a = w(j, c);
        w(j, c) = w(j + jp, c);
        w(j + jp, c) = a;
      }
    __syncthreads();
    if (tid < 32) {           // one reciprocal per pivot; multipliers scaled by it
      const double rp = zero ? 0.0 : 1.0 / w(j, j);
      if (!zero && tid < km) w(j + 1 + tid, j) *= rp;
      if (tid == 0) invg[j] = (T)rp;
    }
    __syncthreads();
    if (!zero && ur <= km) {
      const double m = w(j + ur, j);
      for (int c = j + 1 + ucg; c <= ju; c += LUT / 16) w(j + ur, c) -= m * w(j, c);
    }
    __syncthreads();
    if (tid < LDAB) {         // column j is final: store it, refill its slot with column j + WS
      double& slot = W[tid + LDAB * (j & (WS - 1))];
      bandg[tid + LDAB * j] = (T)slot;
      slot = assemble(tid, j + WS);
    }
  }
  if (!ok && tid == 0) atomicOr(d.err, ERR_SINGULAR);
  if (tid == 0) {
    const int ku = min(kureach, KV);
    d.kur[b] = ku;
    atomicMax(d.kumax, ku);
  }
}

// ---- leaf factorization, kernel B: the Schur complement onto the sides from the ring of
// A_II^{-1} (one thread per side unknown q: a band solve with the unit vector of its interior
// neighbour, the factor read from global memory), then the original couplings this box owns.
// Two leaves per 128-thread CTA.
template <typename T>
__global__ void __launch_bounds__(FTH) leaf_schur_kernel(LeafDev d) {
  __shared__ double qa[LPC][NQ], qc[LPC][NQ];
  __shared__ int qm[LPC][NQ], qex[LPC][NQ];
  const int sub = threadIdx.x / 64;
  const int tid = threadIdx.x % 64;
  const int b = blockIdx.x * LPC + sub;
  const int nbox = d.g.nbox();
  const bool live = b < nbox;
  const Geo g = d.g;
  const int I = live ? b % g.bx : 0, J = live ? b / g.bx : 0;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  T* F = reinterpret_cast<T*>(d.F) + (size_t)(live ? b : 0) * d.ldF * d.ldF;
  if (live) {
    for (int q = tid; q < NQ; q += 64) {
      int vx, vy, m;
      side_unknown(q, x0, y0, &vx, &vy, &m);
      const bool exists = vx >= 0 && vx < nx && vy >= 0 && vy < d.ny;
      qm[sub][q] = m;
      qex[sub][q] = exists ? 1 : 0;
      double a = 0.0, c = 0.0;
      if (exists) {
        const int node = vx + nx * vy;
        const int mnode = (x0 + m % LEAF) + nx * (y0 + m / LEAF);
        a = csr_entry(d.rowptr, d.colind, d.val, node, mnode);
        c = csr_entry(d.rowptr, d.colind, d.val, mnode, node);
      }
      qa[sub][q] = a;
      qc[sub][q] = c;
    }
  }
  __syncthreads();
  if (live && tid < NQ) {
    const int q = c_qorder[tid];
    const int j0 = c_qstart[tid >> 5];
    Band<T, true> Bd{reinterpret_cast<const T*>(d.band) + (size_t)b * LDAB * NI, d.piv + (size_t)b * NI,
                     reinterpret_cast<const T*>(d.invd) + (size_t)b * NI};
    T* yb = reinterpret_cast<T*>(d.ybuf) + (size_t)b * NI * QL;
    const int mq = qm[sub][q];
    const T cq = qex[sub][q] ? (T)qc[sub][q] : T(0);
    sweep_L<T>(Bd, j0, [&](int j) { return j == mq ? cq : T(0); },
               [&](int j, T y) { yb[(size_t)j * QL + tid] = y; });
    const size_t ldF = d.ldF;
    auto yin = [&](int j) { return j < j0 ? T(0) : yb[(size_t)j * QL + tid]; };
    auto ring_out = [&](int j, T x) {
      const int lx = j % LEAF, ly = j / LEAF;
      if (ly == 0 && qex[sub][lx]) F[lx + ldF * q] = -(T)qa[sub][lx] * x;
      if (ly == LEAF - 1 && qex[sub][LEAF + lx]) F[(LEAF + lx) + ldF * q] = -(T)qa[sub][LEAF + lx] * x;
      if (lx == 0 && qex[sub][2 * LEAF + ly]) F[(2 * LEAF + ly) + ldF * q] = -(T)qa[sub][2 * LEAF + ly] * x;
      if (lx == LEAF - 1 && qex[sub][3 * LEAF + ly]) F[(3 * LEAF + ly) + ldF * q] = -(T)qa[sub][3 * LEAF + ly] * x;
    };
    if (d.kur[b] <= 15) sweep_U<T, 16>(Bd, yin, ring_out);   // no interchange widened U
    else sweep_U<T, 32>(Bd, yin, ring_out);
  }
  __syncthreads();
  const bool active = live;
  // original couplings owned by this box: its TOP and RIGHT sides (it is their lower /
  // left box) with their end junctions, and the diagonal of its BL junction.
  //   task 0..14 TOP row -> TOP, TL, TR   15..29 RIGHT row -> RIGHT, BR, TR
  //   30 TL row -> TOP   31 TR row -> TOP, RIGHT   32 BR row -> RIGHT   33 BL row -> BL
  if (active && tid < 2 * LEAF + 4) {
    int vx, vy;
    if (tid < LEAF) { vx = x0 + tid; vy = y0 + LEAF; }
    else if (tid < 2 * LEAF) { vx = x0 + LEAF; vy = y0 + tid - LEAF; }
    else if (tid == 30) { vx = x0 - 1; vy = y0 + LEAF; }
    else if (tid == 31) { vx = x0 + LEAF; vy = y0 + LEAF; }
    else if (tid == 32) { vx = x0 + LEAF; vy = y0 - 1; }
    else { vx = x0 - 1; vy = y0 - 1; }
    if (vx >= 0 && vx < nx && vy >= 0 && vy < d.ny) {
      const int row = vx + nx * vy;
      const int pi = leaf_frontal_pos(vx, vy, x0, y0);
      for (int p = d.rowptr[row]; p < d.rowptr[row + 1]; ++p) {
        int c = d.colind[p];
        int pj = leaf_frontal_pos(c % nx, c / nx, x0, y0);
        if (pj < 0) continue;
        const bool on_top = pj >= LEAF && pj < 2 * LEAF;
        const bool on_right = pj >= 3 * LEAF && pj < 4 * LEAF;
        bool take;
        if (tid < LEAF) take = on_top || pj == 4 * LEAF + C_TL || pj == 4 * LEAF + C_TR;
        else if (tid < 2 * LEAF) take = on_right || pj == 4 * LEAF + C_BR || pj == 4 * LEAF + C_TR;
        else if (tid == 30) take = on_top;
        else if (tid == 31) take = on_top || on_right;
        else if (tid == 32) take = on_right;
        else take = (pj == pi);
        if (take) F[pi + (size_t)d.ldF * pj] += (T)d.val[p];
      }
    }
  }
}

// ---------------------------------------------------------------- solve
// One thread per (leaf, right-hand side).  Forward (leaf part of W~): X[I] <- A_II^{-1} X[I];
// the side unknowns are updated afterwards by sep_update_fwd_kernel.  Backward (leaf part of
// V~): X[I] <- X[I] - A_II^{-1} (A_Id x_d).  The intermediate L^{-1} P b goes through ybuf.
// One thread per (leaf, right-hand side slot), LPB leaves x 16 slots per CTA.  The band
// columns of the next block of steps (16 for L, KUW for U) are copied into a double-buffered
// shared-memory stage with cp.async while the current block is swept, so the sequential
// sweeps read their factor entries from shared memory without waiting on L2.
constexpr int SLOT = 16;   // right-hand-side slots per leaf and launch

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
template <typename T>
__device__ __forceinline__ void cp_async_t(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8) cp_async8(smem, gmem); else cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T, int KUW, int LPB>
__global__ void __launch_bounds__(LPB * SLOT) leaf_solve_kernel(LeafDev d, double* X, int nrhs, int ld, int bwd) {
  extern __shared__ double lsm[];
  constexpr int LST = SLOT * SLOT;                    // L stage per leaf: 16 columns x 16 (r = 1..15)
  constexpr int UST = KUW * KUW;                      // U stage per leaf: KUW columns x KUW (r = 0 -> 1/U_jj)
  constexpr int RMAX = KUW - 1 < KV ? KUW - 1 : KV;
  T* stg = reinterpret_cast<T*>(lsm);                 // 2 buffers
  const int nbox = d.g.nbox();
  const int sub = threadIdx.x / SLOT, c = threadIdx.x % SLOT;
  const int b0 = blockIdx.x * LPB;
  const int b = b0 + sub;
  const bool active = b < nbox && c < nrhs;
  const int bb = b < nbox ? b : nbox - 1;
  const T* gband = reinterpret_cast<const T*>(d.band);
  const T* ginv = reinterpret_cast<const T*>(d.invd);
  const size_t bufL = (size_t)LPB * (LST + SLOT);     // values + pivots (pivots stored as T slots)
  const size_t bufU = (size_t)LPB * UST;
  const size_t bufsz = bufL > bufU ? bufL : bufU;
  const int I = bb % d.g.bx, J = bb / d.g.bx;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  T* yb = reinterpret_cast<T*>(d.ybuf) + (size_t)bb * NI * QL;
  double* Xc = X + (size_t)ld * c;
  auto node_of = [&](int j) { return (x0 + j % LEAF) + nx * (y0 + j / LEAF); };

  // ---- L sweep: y = L^{-1} P x, blocks of 16 steps
  auto issue_L = [&](int blk, int buf) {
    T* S = stg + (size_t)buf * bufsz;
    const int j0 = blk * SLOT;
    for (int x = threadIdx.x; x < LPB * SLOT * (SLOT - 1); x += blockDim.x) {
      const int sl = x / (SLOT * (SLOT - 1)), rem = x % (SLOT * (SLOT - 1));
      const int u = rem / (SLOT - 1), r = rem % (SLOT - 1) + 1;
      const int lb = b0 + sl < nbox ? b0 + sl : nbox - 1;
      if (j0 + u < NI) cp_async_t(S + (size_t)sl * LST + u * SLOT + r, gband + (size_t)lb * LDAB * NI + (KV + r) + LDAB * (j0 + u));
    }
    int* P = reinterpret_cast<int*>(S + (size_t)LPB * LST);
    for (int x = threadIdx.x; x < LPB * SLOT; x += blockDim.x) {
      const int sl = x / SLOT, u = x % SLOT;
      const int lb = b0 + sl < nbox ? b0 + sl : nbox - 1;
      if (j0 + u < NI) cp_async4(P + x, d.piv + (size_t)lb * NI + j0 + u);
    }
    cp_async_commit();
  };
  const int nbl = (NI + SLOT - 1) / SLOT;
  T W[16];
  if (active) {
    if (!bwd) {
#pragma unroll
      for (int r = 0; r < 16; ++r) W[r] = (T)Xc[node_of(r)];
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) W[r] = T(0);
    }
  }
  auto coupling = [&](int j) {            // (A_Id x_d)_j for the backward sweep
    T v = T(0);
    const int lx = j % LEAF, ly = j / LEAF;
    if (lx == 0 || ly == 0 || lx == LEAF - 1 || ly == LEAF - 1) {
      const int node = node_of(j);
      for (int p = d.rowptr[node]; p < d.rowptr[node + 1]; ++p) {
        const int cc = d.colind[p];
        const int cx = cc % nx - x0, cy = cc / nx - y0;
        if (!(cx >= 0 && cx < LEAF && cy >= 0 && cy < LEAF)) v += (T)(d.val[p] * Xc[cc]);
      }
    }
    return v;
  };
  if (active && bwd) {
#pragma unroll
    for (int r = 0; r < 16; ++r) W[r] = coupling(r);
  }
  issue_L(0, 0);
  for (int blk = 0; blk < nbl; ++blk) {
    if (blk + 1 < nbl) { issue_L(blk + 1, (blk + 1) & 1); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncthreads();
    const T* S = stg + (size_t)(blk & 1) * bufsz + (size_t)sub * LST;
    const int* P = reinterpret_cast<const int*>(stg + (size_t)(blk & 1) * bufsz + (size_t)LPB * LST) + sub * SLOT;
    if (active) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = blk * SLOT + u;
        if (j < NI) {
          const int dsw = P[u] - j;
          T a = W[u], bv = a;
          if (__any_sync(__activemask(), dsw != 0)) {
#pragma unroll
            for (int r = 1; r < 16; ++r)
              if (r == dsw) { bv = W[(u + r) & 15]; W[(u + r) & 15] = a; }
            W[u] = bv;
          }
#pragma unroll
          for (int r = 1; r < 16; ++r) W[(u + r) & 15] -= S[u * SLOT + r] * bv;
          yb[(size_t)j * QL + c] = bv;
          W[u] = (j + 16 < NI) ? (!bwd ? (T)Xc[node_of(j + 16)] : coupling(j + 16)) : T(0);
        }
      }
    }
    __syncthreads();
  }

  // ---- U sweep: x = U^{-1} y, blocks of KUW steps from the bottom
  auto issue_U = [&](int blk, int buf) {
    T* S = stg + (size_t)buf * bufsz;
    const int t0 = blk * KUW;
    for (int x = threadIdx.x; x < LPB * KUW * KUW; x += blockDim.x) {
      const int sl = x / (KUW * KUW), rem = x % (KUW * KUW);
      const int u = rem / KUW, r = rem % KUW;
      const int lb = b0 + sl < nbox ? b0 + sl : nbox - 1;
      const int j = NI - 1 - (t0 + u);
      if (j >= 0 && r <= RMAX) {
        if (r == 0) cp_async_t(S + x, ginv + (size_t)lb * NI + j);
        else cp_async_t(S + x, gband + (size_t)lb * LDAB * NI + (KV - r) + LDAB * j);
      }
    }
    cp_async_commit();
  };
  const int nbu = (NI + KUW - 1) / KUW;
  T V[KUW];
  if (active) {
#pragma unroll
    for (int r = 0; r < KUW; ++r) V[r] = (NI - 1 - r >= 0) ? yb[(size_t)(NI - 1 - r) * QL + c] : T(0);
  }
  issue_U(0, 0);
  for (int blk = 0; blk < nbu; ++blk) {
    if (blk + 1 < nbu) { issue_U(blk + 1, (blk + 1) & 1); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncthreads();
    const T* S = stg + (size_t)(blk & 1) * bufsz + (size_t)sub * UST;
    if (active) {
#pragma unroll
      for (int u = 0; u < KUW; ++u) {
        const int t = blk * KUW + u;
        if (t < NI) {
          const int j = NI - 1 - t;
          const T x = V[u] * S[u * KUW];
          if (!bwd) Xc[node_of(j)] = (double)x;
          else Xc[node_of(j)] -= (double)x;
#pragma unroll
          for (int r = 1; r <= RMAX; ++r) V[(u + r) & (KUW - 1)] -= S[u * KUW + r] * x;
          V[u] = (j - KUW >= 0) ? yb[(size_t)(j - KUW) * QL + c] : T(0);
        }
      }
    }
    __syncthreads();
  }
}

// b_u -= sum over interior neighbours j of A_uj t_j, for every separator node u.  One thread
// per (separator node, right-hand side); separator nodes are enumerated in closed form: the
// R full separator rows (y = 16 r + 15) first, then the C separator columns (x = 16 q + 15) of
// the remaining rows.
__global__ void sep_update_fwd_kernel(LeafDev d, double* X, int nrhs, int ld) {
  const int nx = d.nx, ny = d.ny;
  const int R = (ny + 1) / (LEAF + 1) - 1, C = (nx + 1) / (LEAF + 1) - 1;
  const long long nrow = (long long)R * nx;
  const long long nsep = nrow + (long long)(ny - R) * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nsep * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    const long long sidx = e % nsep;
    const int c = (int)(e / nsep);
    int ux, uy;
    if (sidx < nrow) {
      uy = (int)(sidx / nx) * (LEAF + 1) + LEAF;
      ux = (int)(sidx % nx);
    } else {
      const long long t = sidx - nrow;
      const int yy = (int)(t / C);
      ux = (int)(t % C) * (LEAF + 1) + LEAF;
      uy = (yy / LEAF) * (LEAF + 1) + yy % LEAF;
    }
    const int u = ux + nx * uy;
    double acc = 0.0;
    for (int p = d.rowptr[u]; p < d.rowptr[u + 1]; ++p) {
      const int v = d.colind[p];
      const int vx = v % nx, vy = v / nx;
      const bool vsep = ((vx + 1) % (LEAF + 1) == 0) || ((vy + 1) % (LEAF + 1) == 0);
      if (!vsep) acc += d.val[p] * X[v + (size_t)ld * c];
    }
    X[u + (size_t)ld * c] -= acc;
  }
}

// side unknowns sorted by the in-leaf index of their interior neighbour, and the first
// sweep step of each of the two warps that solve for them
void qorder_tables(int* ord, int* start) {
  int m[NQ];
  for (int q = 0; q < NQ; ++q) {
    int s = q / LEAF, t = q % LEAF;
    m[q] = s == SIDE_BOTTOM ? t : s == SIDE_TOP ? t + LEAF * (LEAF - 1) : s == SIDE_LEFT ? LEAF * t : LEAF * t + LEAF - 1;
    ord[q] = q;
  }
  for (int a = 1; a < NQ; ++a)
    for (int b2 = a; b2 > 0 && (m[ord[b2]] < m[ord[b2 - 1]] || (m[ord[b2]] == m[ord[b2 - 1]] && ord[b2] < ord[b2 - 1])); --b2) {
      int t = ord[b2]; ord[b2] = ord[b2 - 1]; ord[b2 - 1] = t;
    }
  for (int w = 0; w < 2; ++w) {
    int mn = NI;
    for (int l = 32 * w; l < 32 * w + 32 && l < NQ; ++l) mn = m[ord[l]] < mn ? m[ord[l]] : mn;
    start[w] = mn - KL > 0 ? mn - KL : 0;
  }
}

}  // namespace


cudaError_t leaf_init_tables() {
  int ord[NQ], start[2];
  qorder_tables(ord, start);
  cudaError_t e = cudaMemcpyToSymbol(c_qorder, ord, sizeof(ord));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_qstart, start, sizeof(start));
  return e;
}

void launch_leaf_factor(const LeafDev& d, cudaStream_t s) {
  const int nbox = d.g.nbox();
  note_launch();
  if (d.fp32) leaf_lu_kernel<float><<<nbox, LUT, 0, s>>>(d);
  else leaf_lu_kernel<double><<<nbox, LUT, 0, s>>>(d);
  note_launch();
  if (d.fp32) leaf_schur_kernel<float><<<(nbox + LPC - 1) / LPC, FTH, 0, s>>>(d);
  else leaf_schur_kernel<double><<<(nbox + LPC - 1) / LPC, FTH, 0, s>>>(d);
}

template <typename T, int KUW, int LPB>
static void leaf_solve_go(const LeafDev& d, double* X, int nrhs, int ld, int bwd, cudaStream_t s) {
  const size_t bufL = (size_t)LPB * (SLOT * SLOT + SLOT), bufU = (size_t)LPB * KUW * KUW;
  const size_t smem = 2 * sizeof(T) * (bufL > bufU ? bufL : bufU);
  cudaFuncSetAttribute(leaf_solve_kernel<T, KUW, LPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  leaf_solve_kernel<T, KUW, LPB><<<(d.g.nbox() + LPB - 1) / LPB, LPB * SLOT, smem, s>>>(d, X, nrhs, ld, bwd);
}

void launch_leaf_solve(const LeafDev& d, double* X, int nrhs, int ld, int bwd, int kumax, cudaStream_t s) {
  for (int c0 = 0; c0 < nrhs; c0 += SLOT) {
    const int nc = nrhs - c0 < SLOT ? nrhs - c0 : SLOT;
    double* Xc = X + (size_t)ld * c0;
    if (d.fp32) {
      if (kumax <= 15) leaf_solve_go<float, 16, 8>(d, Xc, nc, ld, bwd, s);
      else leaf_solve_go<float, 32, 8>(d, Xc, nc, ld, bwd, s);
    } else {
      if (kumax <= 15) leaf_solve_go<double, 16, 4>(d, Xc, nc, ld, bwd, s);
      else leaf_solve_go<double, 32, 4>(d, Xc, nc, ld, bwd, s);
    }
  }
}

void launch_sep_update_fwd(const LeafDev& d, double* X, int nrhs, int ld, cudaStream_t s) {
  const int R = (d.ny + 1) / (LEAF + 1) - 1, C = (d.nx + 1) / (LEAF + 1) - 1;
  long long n = ((long long)R * d.nx + (long long)(d.ny - R) * C) * nrhs;
  if (n <= 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  note_launch();
  sep_update_fwd_kernel<<<blocks, 256, 0, s>>>(d, X, nrhs, ld);
}

}  // namespace spalu
