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
// The LU works on a window of band columns in shared memory (LAPACK band layout); each final
// column leaves it as three 16-value records (L multipliers and pivot offset; reciprocal
// pivot and U above the diagonal; U entries 16..30 that interchanges create), which the sweeps
// stage 16 columns at a time as contiguous runs.
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

// Read-only view of one leaf's factor records in precision T (written by an earlier kernel,
// read through the read-only path).
template <typename T>
struct Band {
  const T* __restrict__ lr;     // NI x 16: L(j+1+r, j) at r, pivot offset at 15
  const T* __restrict__ ur;     // NI x 16: 1/U_jj at 0, U(j-r, j) at r <= 15
  const T* __restrict__ ux;     // NI x 16: U(j-r, j) at r - 16 for r >= 16
  __device__ __forceinline__ T l(int r, int j) const { return __ldg(lr + 16 * j + r - 1); }   // L(j+r, j)
  __device__ __forceinline__ T u(int r, int j) const {                                        // U(j-r, j)
    return r < 16 ? __ldg(ur + 16 * j + r) : __ldg(ux + 16 * j + r - 16);
  }
  __device__ __forceinline__ int p(int j) const { return j + (int)__ldg(lr + 16 * j + 15); }
  __device__ __forceinline__ T dinv(int j) const { return __ldg(ur + 16 * j); }
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
// L2 policy for data read once per pass (the factor records of the sweeps): first to be evicted,
// so that the solve vector, written and read back within the pass, stays in L2
__device__ __forceinline__ unsigned long long evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_ef(void* smem, const void* gmem, unsigned long long pol) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "l"(pol));
}

// 16 consecutive values of shared memory (16-byte aligned) into registers, 128-bit loads
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T* p, T (&v)[N]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 q = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 q = reinterpret_cast<const double2*>(p)[i];
      v[2 * i] = q.x; v[2 * i + 1] = q.y;
    }
  }
}

// Warp-staged variants of the two sweeps for the leaf Schur kernel: every lane of the warp
// takes part (act = this lane owns a column), the warp starts its forward sweep at the same
// column j0, and the records of the next 16 columns are copied into a double-buffered per-warp
// stage with 16-byte cp.async while the current 16 columns are swept.  A stage holds 16
// records of 16 values: the L records of columns jb..jb+15, or the U records of columns
// NI-1-t0 down to NI-16-t0.  Upper bandwidth <= 15 (no interchange widened U).
template <typename T>
struct WarpStage {
  T* v;      // 2 x 16 x 16, 16-byte aligned
};

template <typename T>
__device__ __forceinline__ void stage_L(const WarpStage<T>& w, int buf, const T* lr, int jb, int lane) {
  constexpr int EPC = 16 / sizeof(T), CPR = 16 / EPC;   // values per chunk, chunks per record
  T* v = w.v + buf * 256;
  for (int x = lane; x < 16 * CPR; x += 32) {
    const int u = x / CPR, k = x % CPR, j = jb + u;
    if (j < NI) cp_async16(v + u * 16 + k * EPC, lr + (size_t)16 * j + k * EPC);
  }
  cp_async_commit();
}

template <typename T>
__device__ __forceinline__ void stage_U(const WarpStage<T>& w, int buf, const T* ur, int t0, int lane) {
  constexpr int EPC = 16 / sizeof(T), CPR = 16 / EPC;
  T* v = w.v + buf * 256;
  for (int x = lane; x < 16 * CPR; x += 32) {
    const int u = x / CPR, k = x % CPR, j = NI - 1 - (t0 + u);
    if (j >= 0) cp_async16(v + u * 16 + k * EPC, ur + (size_t)16 * j + k * EPC);
  }
  cp_async_commit();
}

template <typename T, class In, class Out>
__device__ __forceinline__ void sweep_L_staged(const WarpStage<T>& w, const T* lr, int j0, bool act, In in,
                                               Out out) {
  const int lane = threadIdx.x & 31;
  T W[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) W[r] = (act && j0 + r < NI) ? in(j0 + r) : T(0);
  const int nb = (NI - j0 + 15) / 16;
  stage_L(w, 0, lr, j0, lane);
  for (int blk = 0; blk < nb; ++blk) {
    if (blk + 1 < nb) { stage_L(w, (blk + 1) & 1, lr, j0 + 16 * (blk + 1), lane); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncwarp();
    const T* S = w.v + (blk & 1) * 256;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int j = j0 + 16 * blk + u;
      if (j < NI) {
        T lv[16];
        lds_vec(S + u * 16, lv);
        const int dsw = (int)lv[15];   // the same for the whole warp (one leaf)
        T a = W[u], b = a;
        if (dsw != 0) {
#pragma unroll
          for (int r = 1; r < 16; ++r)
            if (r == dsw) { b = W[(u + r) & 15]; W[(u + r) & 15] = a; }
          W[u] = b;
        }
#pragma unroll
        for (int r = 1; r < 16; ++r) W[(u + r) & 15] -= lv[r - 1] * b;
        if (act) out(j, b);
        W[u] = (act && j + 16 < NI) ? in(j + 16) : T(0);
      }
    }
    __syncwarp();
  }
}

template <typename T, class In, class Out>
__device__ __forceinline__ void sweep_U_staged(const WarpStage<T>& w, const T* ur, bool act, In in, Out out) {
  const int lane = threadIdx.x & 31;
  T V[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) V[r] = act ? in(NI - 1 - r) : T(0);
  const int nb = (NI + 15) / 16;
  stage_U(w, 0, ur, 0, lane);
  for (int blk = 0; blk < nb; ++blk) {
    if (blk + 1 < nb) { stage_U(w, (blk + 1) & 1, ur, 16 * (blk + 1), lane); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncwarp();
    const T* S = w.v + (blk & 1) * 256;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = 16 * blk + u;
      if (t < NI) {
        const int j = NI - 1 - t;
        T uv[16];
        lds_vec(S + u * 16, uv);
        const T x = V[u] * uv[0];
        if (act) out(j, x);
#pragma unroll
        for (int r = 1; r < 16; ++r) V[(u + r) & 15] -= uv[r] * x;
        V[u] = (act && j - 16 >= 0) ? in(j - 16) : T(0);
      }
    }
    __syncwarp();
  }
}

// The backward sweep of the leaf Schur kernel in FP32 with the y rows of the next block staged
// too: row j of the warp's 32 columns is one 128-byte run of the sweep buffer (ybw + j QL),
// written by this warp's forward sweep; the refill of step u of block blk reads row j - 16 from
// the stage of block blk + 1 instead of a global load outstanding at the warp barriers.
// Rows below j0 (where this warp's forward sweep started) are zero.
template <typename T, class Out>
__device__ __forceinline__ void sweep_U_staged_y(const WarpStage<T>& w, T* ys, const T* ur, const T* ybw, int j0,
                                                 bool act, Out out) {
  const int lane = threadIdx.x & 31;
  T V[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) V[r] = (act && NI - 1 - r >= j0) ? ybw[(size_t)(NI - 1 - r) * QL + lane] : T(0);
  auto stage_y = [&](int buf, int blk) {   // rows of block blk (no commit: stage_U commits)
    T* Y = ys + buf * 512;
    for (int x = lane; x < 16 * 8; x += 32) {
      const int u = x >> 3, k = x & 7, j = NI - 1 - 16 * blk - u;
      if (j >= j0) cp_async16(Y + u * 32 + 4 * k, ybw + (size_t)j * QL + 4 * k);
    }
  };
  const int nb = (NI + 15) / 16;
  stage_y(0, 1);
  stage_U(w, 0, ur, 0, lane);
  for (int blk = 0; blk < nb; ++blk) {
    if (blk + 1 < nb) {
      stage_y((blk + 1) & 1, blk + 2);
      stage_U(w, (blk + 1) & 1, ur, 16 * (blk + 1), lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const T* S = w.v + (blk & 1) * 256;
    const T* Ys = ys + (blk & 1) * 512 + lane;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int t = 16 * blk + u;
      if (t < NI) {
        const int j = NI - 1 - t;
        T uv[16];
        lds_vec(S + u * 16, uv);
        const T x = V[u] * uv[0];
        if (act) out(j, x);
#pragma unroll
        for (int r = 1; r < 16; ++r) V[(u + r) & 15] -= uv[r] * x;
        V[u] = (act && j - 16 >= j0) ? Ys[u * 32] : T(0);
      }
    }
    __syncwarp();
  }
}

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
// slot is refilled with column j + WS (first touched at step j + 2) from the gathered nonzeros
// (leaf_band5_kernel) by cp.async, waited for two steps later.
// Also zeroes the leaf's frontal block and records the upper bandwidth reached.
constexpr int WS = 32;       // window columns (> KV)
constexpr int LUT = 64;      // threads per leaf LU

// The leaf matrices' nonzeros by column, gathered from the CSR once for all leaves (one thread
// per leaf, column and stencil offset, every lookup independent), so that the LU's window
// refills read them with plain loads issued a step ahead instead of searching the CSR on the
// critical path of every step.
__global__ void leaf_band5_kernel(LeafDev d) {
  const int nbox = d.g.nbox();
  const long long n = (long long)nbox * NI * 5;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(x % 5), c = (int)((x / 5) % NI), b = (int)(x / (5 * NI));
    const int o = k == 0 ? -LEAF : k == 1 ? -1 : k == 2 ? 0 : k == 3 ? 1 : LEAF;
    const int i = c + o;
    double v = 0.0;
    if (i >= 0 && i < NI && (o == 0 || o == LEAF || o == -LEAF || i / LEAF == c / LEAF)) {
      const int x0 = (b % d.g.bx) * (LEAF + 1), y0 = (b / d.g.bx) * (LEAF + 1);
      v = csr_entry(d.rowptr, d.colind, d.val, (x0 + i % LEAF) + d.nx * (y0 + i / LEAF),
                    (x0 + c % LEAF) + d.nx * (y0 + c / LEAF));
    }
    d.band5[x] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(LUT) leaf_lu_kernel(LeafDev d) {
  __shared__ double W[LDAB * WS];
  __shared__ int sh[2];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const Geo g = d.g;
  {
    T* F = reinterpret_cast<T*>(d.F) + (size_t)b * d.ldF * d.ldF;
    const int D = g.D();
    for (int e = tid; e < D * D; e += LUT) F[(e % D) + (size_t)d.ldF * (e / D)] = T(0);
  }
  T* lrg = reinterpret_cast<T*>(d.lrec) + (size_t)b * NI * 16;
  T* urg = reinterpret_cast<T*>(d.urec) + (size_t)b * NI * 16;
  T* uxg = reinterpret_cast<T*>(d.uext) + (size_t)b * NI * 16;
  // band row r of column c of A_II: A(c + r - KV, c), nonzero for the five stencil offsets only
  const double* b5 = d.band5 + (size_t)b * NI * 5;
  auto assemble = [&](int r, int c) -> double {
    const int o = r - KV;
    const int k = o == -LEAF ? 0 : o == -1 ? 1 : o == 0 ? 2 : o == 1 ? 3 : o == LEAF ? 4 : -1;
    return (c < NI && k >= 0) ? b5[5 * c + k] : 0.0;
  };
  auto w = [&](int i, int c) -> double& { return W[(KV + i - c) + LDAB * (c & (WS - 1))]; };
  for (int x = tid; x < LDAB * WS; x += LUT) W[x] = assemble(x % LDAB, x / LDAB);
  // band row tid of a refilled column: stencil offset k of the gathered nonzeros, or none
  const int ko = tid - KV;
  const int kst = ko == -LEAF ? 0 : ko == -1 ? 1 : ko == 0 ? 2 : ko == 1 ? 3 : ko == LEAF ? 4 : -1;
  __syncthreads();
  int ju = 0, kureach = KU;
  bool ok = true, swapped = false;
  const int ur = 1 + (tid & 15), ucg = tid >> 4;       // rank-1 update: row, column group
  for (int j = 0; j < NI; ++j) {
    const int km = min(KL, NI - 1 - j);
    cp_async_wait<1>();       // the refills issued up to step j - 2 (column j + 30 at the latest)
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
        lrg[16 * j + 15] = (T)bi;      // pivot offset 0..15, exact in T
      }
    }
    __syncthreads();
    const int jp = sh[0];
    const bool zero = sh[1] != 0;
    if (zero) ok = false;
    swapped |= jp != 0;
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
      if (tid == 0) urg[16 * j] = (T)rp;
    }
    __syncthreads();
    if (!zero && ur <= km) {
      const double m = w(j + ur, j);
      for (int c = j + 1 + ucg; c <= ju; c += LUT / 16) w(j + ur, c) -= m * w(j, c);
    }
    __syncthreads();
    if (tid < LDAB) {         // column j is final: store its records, refill its slot with column j + WS
      double& slot = W[tid + LDAB * (j & (WS - 1))];
      const T v = (T)slot;
      if (tid > KV) lrg[16 * j + (tid - KV - 1)] = v;              // L(j+1+r, j), r = tid - KV - 1
      else if (tid > KV - 16) { if (tid < KV) urg[16 * j + (KV - tid)] = v; }   // U(j-r, j), r = KV - tid <= 15
      else uxg[16 * j + (KV - 16 - tid)] = v;                      // U(j-r, j), r = 16..30
      if (tid == KV) uxg[16 * j + 15] = T(0);
      // column j + WS (first touched at step j + 2): its stencil rows copied asynchronously, the
      // rest zero, so that no global load is outstanding at the next barriers
      if (j + WS < NI && kst >= 0) cp_async8(&slot, b5 + 5 * (j + WS) + kst);
      else slot = 0.0;
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  if (!ok && tid == 0) atomicOr(d.err, ERR_SINGULAR);
  if (tid == 0) {
    const int ku = min(kureach, KV);
    d.kur[b] = ku;
    atomicMax(d.kumax, swapped && ku < 16 ? 16 : ku);   // <= 15: no leaf made an interchange
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
      reinterpret_cast<T*>(d.cpl)[(size_t)b * NQ + q] = (T)c;   // A(m, side unknown q), 0 outside the grid
    }
  }
  __syncthreads();
  __shared__ __align__(16) T stv[FTH / 32][512];
  __shared__ __align__(16) T sty[FTH / 32][sizeof(T) == 4 ? 1024 : 4];   // FP32: y rows of the U sweep
  if (live && d.kur[b] <= 15) {     // warp-staged sweeps (all lanes; lanes >= NQ only stage)
    const bool act = tid < NQ;
    const int q = act ? c_qorder[tid] : 0;
    const int j0 = c_qstart[tid >> 5];
    const WarpStage<T> ws{stv[threadIdx.x >> 5]};
    const T* lr = reinterpret_cast<const T*>(d.lrec) + (size_t)b * NI * 16;
    const T* ur = reinterpret_cast<const T*>(d.urec) + (size_t)b * NI * 16;
    T* yb = reinterpret_cast<T*>(d.ybuf) + (size_t)b * NI * QL;
    T* Gb = d.G ? reinterpret_cast<T*>(d.G) + (size_t)b * NI * NQ : nullptr;
    const int mq = act ? qm[sub][q] : -1;
    const T cq = (act && qex[sub][q]) ? (T)qc[sub][q] : T(0);
    sweep_L_staged<T>(ws, lr, j0, act, [&](int j) { return j == mq ? cq : T(0); },
                      [&](int j, T y) { yb[(size_t)j * QL + tid] = y; });
    const size_t ldF = d.ldF;
    auto yin = [&](int j) { return j < j0 ? T(0) : yb[(size_t)j * QL + tid]; };
    auto ring_out = [&](int j, T x) {
      if (Gb) Gb[(size_t)j * NQ + q] = x;                   // column q of A_II^{-1} A_Id
      const int lx = j % LEAF, ly = j / LEAF;
      if (ly == 0 && qex[sub][lx]) F[lx + ldF * q] = -(T)qa[sub][lx] * x;
      if (ly == LEAF - 1 && qex[sub][LEAF + lx]) F[(LEAF + lx) + ldF * q] = -(T)qa[sub][LEAF + lx] * x;
      if (lx == 0 && qex[sub][2 * LEAF + ly]) F[(2 * LEAF + ly) + ldF * q] = -(T)qa[sub][2 * LEAF + ly] * x;
      if (lx == LEAF - 1 && qex[sub][3 * LEAF + ly]) F[(3 * LEAF + ly) + ldF * q] = -(T)qa[sub][3 * LEAF + ly] * x;
    };
    if constexpr (sizeof(T) == 4)
      sweep_U_staged_y<T>(ws, sty[threadIdx.x >> 5], ur, yb + 32 * (tid >> 5), j0, act, ring_out);
    else
      sweep_U_staged<T>(ws, ur, act, yin, ring_out);
  } else if (live && tid < NQ) {    // widened U: sweeps reading the band from global memory
    const int q = c_qorder[tid];
    const int j0 = c_qstart[tid >> 5];
    Band<T> Bd{reinterpret_cast<const T*>(d.lrec) + (size_t)b * NI * 16,
               reinterpret_cast<const T*>(d.urec) + (size_t)b * NI * 16,
               reinterpret_cast<const T*>(d.uext) + (size_t)b * NI * 16};
    T* yb = reinterpret_cast<T*>(d.ybuf) + (size_t)b * NI * QL;
    T* Gb = d.G ? reinterpret_cast<T*>(d.G) + (size_t)b * NI * NQ : nullptr;
    const int mq = qm[sub][q];
    const T cq = qex[sub][q] ? (T)qc[sub][q] : T(0);
    sweep_L<T>(Bd, j0, [&](int j) { return j == mq ? cq : T(0); },
               [&](int j, T y) { yb[(size_t)j * QL + tid] = y; });
    const size_t ldF = d.ldF;
    auto yin = [&](int j) { return j < j0 ? T(0) : yb[(size_t)j * QL + tid]; };
    auto ring_out = [&](int j, T x) {
      if (Gb) Gb[(size_t)j * NQ + q] = x;                   // column q of A_II^{-1} A_Id
      const int lx = j % LEAF, ly = j / LEAF;
      if (ly == 0 && qex[sub][lx]) F[lx + ldF * q] = -(T)qa[sub][lx] * x;
      if (ly == LEAF - 1 && qex[sub][LEAF + lx]) F[(LEAF + lx) + ldF * q] = -(T)qa[sub][LEAF + lx] * x;
      if (lx == 0 && qex[sub][2 * LEAF + ly]) F[(2 * LEAF + ly) + ldF * q] = -(T)qa[sub][2 * LEAF + ly] * x;
      if (lx == LEAF - 1 && qex[sub][3 * LEAF + ly]) F[(3 * LEAF + ly) + ldF * q] = -(T)qa[sub][3 * LEAF + ly] * x;
    };
    sweep_U<T, 32>(Bd, yin, ring_out);
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
// V~): X[I] <- X[I] - A_II^{-1} (A_Id x_d).
constexpr int SLOT = 16;   // right-hand-side slots per leaf and launch
constexpr int SWPB = 4;    // warps per CTA of the solve sweeps (two leaves per warp)

// Per-warp shared-memory stage of leaf_solve_kernel (values of T).  L phase, two buffers of:
// for each of the warp's two leaves 16 L records and (FP32 forward) the right-hand-side rows
// of the next block; backward also the leaves' 60 side values x_d and coupling coefficients.
// U phase, two buffers of: KUW columns of KUW values (the U record, and for KUW = 32 its
// extension) and (FP32) the KUW rows y of the next block and (FP32 backward) the KUW rows of x
// this block updates.  Rows hold 16 values (the right-hand sides); the pads put the two
// leaves of a warp on different banks.
template <typename T, int KUW, bool bwd>
struct SolveStage {
  static constexpr int EPC = 16 / (int)sizeof(T);      // values per 16-byte chunk
  static constexpr int CPR = SLOT / EPC;                // chunks per 16-value record
  static constexpr bool CHKV = sizeof(T) == 4;          // FP32: the chunked solve vector
  static constexpr bool XPF = !bwd && CHKV;
  static constexpr bool YPF = CHKV;
  static constexpr bool XOPF = bwd && CHKV;
  static constexpr int LSTP = SLOT * SLOT + EPC;
  static constexpr int USTP = KUW * KUW + EPC;
  static constexpr int XSTP = SLOT * SLOT + 16;
  static constexpr int YSTP = KUW * SLOT + 16;
  static constexpr int XDSTP = NQ * SLOT + 16;
  static constexpr int bufL = 2 * (LSTP + (XPF ? XSTP : 0));
  static constexpr int bufU = 2 * (USTP + (YPF ? YSTP : 0) + (XOPF ? YSTP : 0));
  static constexpr int xdsz = bwd ? 2 * XDSTP + 2 * 64 : 0;
  static constexpr int warpsz = 2 * bufL + xdsz > 2 * bufU ? 2 * bufL + xdsz : 2 * bufU;
  static constexpr size_t bytes = (size_t)SWPB * warpsz * sizeof(T);
};

// Band sweeps, one warp per two leaves x 16 right-hand sides, thread (leaf, rhs): forward
// x_I = U^{-1} L^{-1} P b_I; backward x_I -= U^{-1} L^{-1} P (A_Id x_d).
// - Warp-synchronous: a warp stages the factor records of its own two leaves for the next
//   block of 16 (L) or KUW (U) steps with 16-byte cp.async (L2 evict-first: read once per
//   pass) into its double-buffered stage while it sweeps the current block; no CTA barrier.
// - Forward: y = L^{-1} P b overwrites b in the solve vector (row j is written at step j,
//   after the last read of b_j) and the U sweep reads it back from there, so the intermediate
//   costs no scratch traffic and stays in L2 between the sweeps.  Backward: x_I is needed
//   until the last step, so y goes through the sweep buffer.
// - Backward input: (A_Id x_d)_j is nonzero on the leaf's boundary rows only, one term per
//   side the node touches: the coupling coefficient (stored by the factorization) times the
//   side value, both staged once per warp.
// - FP32: the solve vector is chunked (a node's 16 right-hand sides are one 64-byte run); the
//   right-hand-side rows of the next L block, the y rows of the next U block and (backward)
//   the rows a U block updates are staged with the records, so no global load is
//   outstanding at a warp barrier.  FP64 reads them directly.
// - KUW = 16 is launched only when no leaf made an interchange (the step has no swap).
// All lanes run the sweep arithmetic (lanes without a right-hand side or leaf on values that
// are never stored), so the warp votes and barriers are full-warp.
template <typename T, int KUW, bool bwd>
__global__ void __launch_bounds__(SWPB * 32) leaf_solve_kernel(LeafDev d, T* X, int nrhs, VecLayout lay) {
  pdl_trigger();
  extern __shared__ float4 lsm4[];
  using St = SolveStage<T, KUW, bwd>;
  constexpr int EPC = St::EPC, CPR = St::CPR;
  constexpr int LSTP = St::LSTP, USTP = St::USTP, XSTP = St::XSTP, YSTP = St::YSTP, XDSTP = St::XDSTP;
  constexpr int bufL = St::bufL, bufU = St::bufU;
  constexpr int RMAX = KUW - 1 < KV ? KUW - 1 : KV;
  constexpr bool CHK = St::CHKV, XPF = St::XPF, YPF = St::YPF, XOPF = St::XOPF;
  constexpr bool PIV = KUW > 16;
  constexpr int RPC = SLOT * CPR;                     // chunks of one leaf's 16 records
  constexpr int CPC = (KUW / SLOT) * CPR;             // chunks of one U column
  static_assert(RPC % 32 == 0 && (KUW * CPC) % 32 == 0, "a leaf's stage is a whole number of warp copies");
  const int lane = threadIdx.x & 31;
  const int sub = lane >> 4, c = lane & 15;
  const int nbox = d.g.nbox();
  const int b0 = (blockIdx.x * SWPB + (threadIdx.x >> 5)) * 2;   // the warp's first leaf
  if (b0 >= nbox) return;                             // whole warp: no leaf
  const int b = b0 + sub;
  const bool act = b < nbox && c < nrhs;
  T* stg = reinterpret_cast<T*>(lsm4) + (size_t)(threadIdx.x >> 5) * St::warpsz;
  const T* lrec = reinterpret_cast<const T*>(d.lrec);
  const T* urec = reinterpret_cast<const T*>(d.urec);
  const T* uext = reinterpret_cast<const T*>(d.uext);
  const unsigned long long pol = evict_first_policy();
  const int bx = d.g.bx, nx = d.nx;
  const int bb = b < nbox ? b : nbox - 1;
  // the warp's two leaves (the second clamped) and the grid nodes of their interiors' (0, 0)
  const int bl0 = b0, bl1 = b0 + 1 < nbox ? b0 + 1 : b0;
  const int og0 = (bl0 % bx) * (LEAF + 1) + nx * ((bl0 / bx) * (LEAF + 1));
  const int og1 = (bl1 % bx) * (LEAF + 1) + nx * ((bl1 / bx) * (LEAF + 1));
  auto bl = [&](int s) { return s ? bl1 : bl0; };
  auto og = [&](int s) { return s ? og1 : og0; };
  const int o0 = og(sub);                             // this lane's leaf
  auto node_of = [&](int j) { return o0 + j % LEAF + nx * (j / LEAF); };
  T* yb = reinterpret_cast<T*>(d.ybuf) + (size_t)bb * NI * QL;   // backward only, rows of 16
  T* Xc = X + (size_t)c * lay.cs;
  const long long rs = lay.rs;
  auto xat = [&](int node) -> T& {
    if constexpr (CHK) return X[(size_t)node * SLOT + c];
    else return Xc[(size_t)(node * rs)];
  };
  // chunk k (4 values) of the 16-value row of grid node `node` (FP32 chunked vector)
  auto node_chunk = [&](T* dst, int node, int k) { cp_async16(dst, X + (size_t)node * SLOT + 4 * k); };

  // ---- backward input: side values x_d (60 per leaf: BOTTOM, TOP, LEFT, RIGHT, 15 each, the
  //      grid neighbours of the boundary rows) and their coupling coefficients
  T* xd = stg + 2 * bufL;                             // [leaf][q][16], pitch XDSTP
  T* cf = xd + 2 * XDSTP;                             // [leaf][q], pitch 64
  auto side_node = [&](int s, int q) {
    const int t = q % LEAF, o = og(s);
    switch (q / LEAF) {
      case SIDE_BOTTOM: return o - nx + t;
      case SIDE_TOP: return o + LEAF * nx + t;
      case SIDE_LEFT: return o - 1 + nx * t;
      default: return o + LEAF + nx * t;
    }
  };
  if constexpr (bwd) {
    // a side exists unless the leaf touches the grid boundary there (coefficient 0)
    for (int x = lane; x < 2 * NQ; x += 32) {
      const int s = x / NQ, q = x % NQ;
      cf[s * 64 + q] = reinterpret_cast<const T*>(d.cpl)[(size_t)bl(s) * NQ + q];
    }
    __syncwarp();
  }
  // (A_Id x_d)_j of row j = (lx, ly), terms in the order of the CSR columns
  auto cplin = [&](int lx, int ly) -> T {
    const T* xs = xd + sub * XDSTP + c;
    const T* cs = cf + sub * 64;
    T v = T(0);
    if (ly == 0) v += cs[lx] * xs[lx * SLOT];
    if (lx == 0) v += cs[2 * LEAF + ly] * xs[(2 * LEAF + ly) * SLOT];
    if (lx == LEAF - 1) v += cs[3 * LEAF + ly] * xs[(3 * LEAF + ly) * SLOT];
    if (ly == LEAF - 1) v += cs[LEAF + lx] * xs[(LEAF + lx) * SLOT];
    return v;
  };

  // ---- L sweep: y = L^{-1} P x, blocks of 16 steps.  Stage of block blk: its records and
  //      (FP32 forward) right-hand-side rows blk * 16 + 16 .. + 31, the refills of its steps.
  auto issue_L_rec = [&](int blk, int buf) {
    T* S = stg + (size_t)buf * bufL;
    const int j0 = blk * SLOT;
    const int nch = (NI - j0 < SLOT ? NI - j0 : SLOT) * CPR;
#pragma unroll
    for (int i = 0; i < 2 * RPC / 32; ++i) {
      const int s = i / (RPC / 32), k = lane + 32 * (i % (RPC / 32));
      if (k < nch) cp_async16_ef(S + s * LSTP + k * EPC, lrec + ((size_t)bl(s) * NI + j0) * SLOT + k * EPC, pol);
    }
  };
  auto issue_L_x = [&](int blk, int buf) {
    if constexpr (XPF) {
      T* S = stg + (size_t)buf * bufL + 2 * LSTP;
#pragma unroll
      for (int i = 0; i < 2 * SLOT * 4 / 32; ++i) {
        const int s = i / (SLOT * 4 / 32), u = (lane + 32 * (i % (SLOT * 4 / 32))) / 4, k = lane % 4;
        const int r = blk * SLOT + SLOT + u;
        if (r < NI) node_chunk(S + s * XSTP + u * SLOT + 4 * k, og(s) + r % LEAF + nx * (r / LEAF), k);
      }
    }
    cp_async_commit();
  };
  const int nbl = (NI + SLOT - 1) / SLOT;
  issue_L_rec(0, 0);
  pdl_wait();                             // the solve vector is written by the preceding kernel
  if constexpr (bwd) {
    if constexpr (CHK) {
      for (int x = lane; x < 2 * NQ * 4; x += 32) {
        const int s = x / (NQ * 4), q = (x / 4) % NQ, k = x % 4;
        T* dst = xd + s * XDSTP + q * SLOT + 4 * k;
        if (cf[s * 64 + q] != T(0)) node_chunk(dst, side_node(s, q), k);
        else *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      for (int q = 0; q < NQ; ++q) {
        const T a = cf[sub * 64 + q];
        xd[sub * XDSTP + q * SLOT + c] = (act && a != T(0)) ? xat(side_node(sub, q)) : T(0);
      }
    }
  }
  issue_L_x(0, 0);
  T W[16];
  if constexpr (bwd) {
    cp_async_wait<0>();
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) W[r] = cplin(r % LEAF, r / LEAF);
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) W[r] = act ? xat(node_of(r)) : T(0);
  }
  for (int blk = 0; blk < nbl; ++blk) {
    if (blk + 1 < nbl) {
      issue_L_rec(blk + 1, (blk + 1) & 1);
      issue_L_x(blk + 1, (blk + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const T* S = stg + (size_t)(blk & 1) * bufL + sub * LSTP;
    const T* xs = stg + (size_t)(blk & 1) * bufL + 2 * LSTP + sub * XSTP + c;
    int lx = (blk * SLOT) % LEAF, node = node_of(blk * SLOT);   // grid node of step j
    int rx = (blk * SLOT + SLOT) % LEAF, ry = (blk * SLOT + SLOT) / LEAF;   // row j + 16 (backward)
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int j = blk * SLOT + u;
      if (j < NI) {
        T lv[16];
        lds_vec(S + u * SLOT, lv);
        T bv = W[u];
        if constexpr (PIV) {
          const int dsw = (int)lv[15];     // 0..15: the interchange stays in the window
          if (__any_sync(0xffffffffu, dsw != 0)) {
            const T a = bv;
#pragma unroll
            for (int r = 1; r < 16; ++r)
              if (r == dsw) { bv = W[(u + r) & 15]; W[(u + r) & 15] = a; }
          }
        }
#pragma unroll
        for (int r = 1; r < 16; ++r) W[(u + r) & 15] -= lv[r - 1] * bv;
        if (act) {
          if constexpr (!bwd) xat(node) = bv;    // y_j over b_j
          else yb[(size_t)j * SLOT + c] = bv;
        }
        T nv = T(0);
        if (j + 16 < NI) {
          if constexpr (bwd) nv = cplin(rx, ry);
          else if constexpr (XPF) nv = xs[u * SLOT];
          else nv = act ? xat(node_of(j + 16)) : T(0);
        }
        W[u] = nv;
        const bool wrap = lx == LEAF - 1;
        lx = wrap ? 0 : lx + 1;
        node += wrap ? nx - (LEAF - 1) : 1;
        if constexpr (bwd) {
          const bool rw = rx == LEAF - 1;
          rx = rw ? 0 : rx + 1;
          ry += rw ? 1 : 0;
        }
      }
    }
    __syncwarp();
  }

  // ---- U sweep: x = U^{-1} y, blocks of KUW steps from the bottom.  Stage of block blk: its
  //      U columns, (FP32) the y rows of block blk + 1 (the refills of its steps) and
  //      (FP32 backward) the x rows of block blk.
  auto issue_U = [&](int blk, int buf) {
    T* S = stg + (size_t)buf * bufU;
    const int t0 = blk * KUW;
#pragma unroll
    for (int i = 0; i < 2 * KUW * CPC / 32; ++i) {
      const int s = i / (KUW * CPC / 32), rem = lane + 32 * (i % (KUW * CPC / 32)), u = rem / CPC, k = rem % CPC;
      const int j = NI - 1 - (t0 + u);
      if (j >= 0) {
        const size_t rec = ((size_t)bl(s) * NI + j) * SLOT;
        const T* src = k < CPR ? urec + rec + k * EPC : uext + rec + (k - CPR) * EPC;
        cp_async16_ef(S + s * USTP + u * KUW + k * EPC, src, pol);
      }
    }
    if constexpr (YPF) {
      T* Y = S + 2 * USTP;
#pragma unroll
      for (int i = 0; i < 2 * KUW * 4 / 32; ++i) {
        const int s = i / (KUW * 4 / 32), u = (lane + 32 * (i % (KUW * 4 / 32))) / 4, k = lane % 4;
        const int r = NI - 1 - (t0 + KUW + u);
        if (r >= 0) {
          if constexpr (bwd)
            cp_async16(Y + s * YSTP + u * SLOT + 4 * k,
                       reinterpret_cast<const T*>(d.ybuf) + ((size_t)bl(s) * NI * QL + (size_t)r * SLOT) + 4 * k);
          else
            node_chunk(Y + s * YSTP + u * SLOT + 4 * k, og(s) + r % LEAF + nx * (r / LEAF), k);
        }
      }
    }
    if constexpr (XOPF) {
      T* XO = S + 2 * USTP + 2 * YSTP;
#pragma unroll
      for (int i = 0; i < 2 * KUW * 4 / 32; ++i) {
        const int s = i / (KUW * 4 / 32), u = (lane + 32 * (i % (KUW * 4 / 32))) / 4, k = lane % 4;
        const int r = NI - 1 - (t0 + u);
        if (r >= 0) node_chunk(XO + s * YSTP + u * SLOT + 4 * k, og(s) + r % LEAF + nx * (r / LEAF), k);
      }
    }
    cp_async_commit();
  };
  // (FP64 forward) row j - KUW from row j: KUW = 15 q + m, so q leaf rows down and m nodes
  // left, one more row down (and LEAF nodes right) when fewer than m nodes are left of j
  constexpr int QD = KUW / LEAF, MD = KUW % LEAF;
  const int nbu = (NI + KUW - 1) / KUW;
  T V[KUW];
#pragma unroll
  for (int r = 0; r < KUW; ++r)
    V[r] = (act && NI - 1 - r >= 0) ? (bwd ? yb[(size_t)(NI - 1 - r) * SLOT + c] : xat(node_of(NI - 1 - r))) : T(0);
  issue_U(0, 0);
  for (int blk = 0; blk < nbu; ++blk) {
    if (blk + 1 < nbu) { issue_U(blk + 1, (blk + 1) & 1); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncwarp();
    const T* S = stg + (size_t)(blk & 1) * bufU + sub * USTP;
    const T* ys = stg + (size_t)(blk & 1) * bufU + 2 * USTP + sub * YSTP + c;
    const T* xo = stg + (size_t)(blk & 1) * bufU + 2 * USTP + 2 * YSTP + sub * YSTP + c;
    const int jt = NI - 1 - blk * KUW;
    int lx = jt % LEAF, node = node_of(jt);      // grid node of step j (descending)
#pragma unroll
    for (int u = 0; u < KUW; ++u) {
      const int t = blk * KUW + u;
      if (t < NI) {
        const int j = NI - 1 - t;
        T uv[KUW];
        lds_vec(S + u * KUW, uv);
        const T x = V[u] * uv[0];
        if (act) {
          if constexpr (!bwd) xat(node) = x;
          else if constexpr (XOPF) xat(node) = xo[u * SLOT] - x;
          else xat(node) -= x;
        }
#pragma unroll
        for (int r = 1; r <= RMAX; ++r) V[(u + r) & (KUW - 1)] -= uv[r] * x;
        T nv = T(0);
        if (j - KUW >= 0) {
          if constexpr (YPF) nv = ys[u * SLOT];
          else if constexpr (bwd) nv = act ? yb[(size_t)(j - KUW) * SLOT + c] : T(0);
          else nv = act ? xat(node - QD * nx - MD + (lx < MD ? LEAF - nx : 0)) : T(0);
        }
        V[u] = nv;
        const bool wrap = lx == 0;
        lx = wrap ? LEAF - 1 : lx - 1;
        node -= wrap ? nx - (LEAF - 1) : 1;
      }
    }
    __syncwarp();
  }
}

// Backward leaf step of the mixed path on grids of few leaves: x_I -= G x_d with
// G = A_II^{-1} A_Id (FP32, stored by the factorization) and x_d the 60 side unknowns of the
// leaf.  One leaf per CTA: G is staged in shared memory by cp.async while x_d is gathered,
// then thread j forms row j of G x_d for all right-hand sides of the chunk (up to 16) and
// updates the interior unknown j.  225 independent rows per leaf instead of one sequential
// sweep pair: on a grid of few leaves the sweeps' step latency, not traffic, bounds the time.
constexpr int GTH = 256;
constexpr int GRC = 16;                          // right-hand sides per launch
__global__ void __launch_bounds__(GTH, 3) leaf_bwd_g_kernel(LeafDev d, float* X, int nrhs, VecLayout lay) {
  pdl_trigger();
  extern __shared__ float4 gsm4[];
  float* Gs = reinterpret_cast<float*>(gsm4);    // NI x NQ
  float* xd = Gs + NI * NQ;                      // NQ x GRC
  const int b = blockIdx.x;
  const float* Gg = reinterpret_cast<const float*>(d.G) + (size_t)b * NI * NQ;
  for (int i = threadIdx.x; i < NI * NQ / 4; i += GTH) cp_async16(Gs + 4 * i, Gg + 4 * i);
  cp_async_commit();
  pdl_wait();              // G is the factorization's; the solve vector is the preceding kernel's
  const int I = b % d.g.bx, J = b / d.g.bx;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  for (int i = threadIdx.x; i < NQ * GRC; i += GTH) {
    const int q = i / GRC, c = i % GRC;
    int vx, vy, m;
    side_unknown(q, x0, y0, &vx, &vy, &m);
    const bool ex = c < nrhs && vx >= 0 && vx < nx && vy >= 0 && vy < d.ny;
    xd[i] = ex ? X[lay.at(vx + nx * vy, c)] : 0.f;
  }
  cp_async_wait<0>();
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= NI) return;
  float acc[GRC];
#pragma unroll
  for (int c = 0; c < GRC; ++c) acc[c] = 0.f;
  const float4* gr = reinterpret_cast<const float4*>(Gs + j * NQ);
  const float4* x4 = reinterpret_cast<const float4*>(xd);
#pragma unroll 3
  for (int k = 0; k < NQ / 4; ++k) {
    const float4 g = gr[k];
    const float gq[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
      for (int c4 = 0; c4 < GRC / 4; ++c4) {
        const float4 v = x4[(4 * k + t) * (GRC / 4) + c4];
        acc[4 * c4 + 0] += gq[t] * v.x;
        acc[4 * c4 + 1] += gq[t] * v.y;
        acc[4 * c4 + 2] += gq[t] * v.z;
        acc[4 * c4 + 3] += gq[t] * v.w;
      }
    }
  }
  const int node = (x0 + j % LEAF) + nx * (y0 + j / LEAF);
#pragma unroll
  for (int c = 0; c < GRC; ++c)
    if (c < nrhs) X[lay.at(node, c)] -= acc[c];
}

// b_u -= sum over interior neighbours j of A_uj t_j, for every separator node u.  One thread
// per (separator node, right-hand side); separator nodes are enumerated in closed form: the
// R full separator rows (y = 16 r + 15) first, then the C separator columns (x = 16 q + 15) of
// the remaining rows.
template <typename T>
__global__ void sep_update_fwd_kernel(LeafDev d, T* X, int nrhs, VecLayout lay) {
  pdl_enter();
  const int nx = d.nx, ny = d.ny;
  const int R = (ny + 1) / (LEAF + 1) - 1, C = (nx + 1) / (LEAF + 1) - 1;
  const long long nrow = (long long)R * nx;
  const long long nsep = nrow + (long long)(ny - R) * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nsep * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    // consecutive threads: consecutive nodes (column-major vectors) or right-hand sides
    const bool cin = lay.cs == 1;
    const long long sidx = cin ? e / nrhs : e % nsep;
    const int c = (int)(cin ? e % nrhs : e / nsep);
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
    T acc = T(0);
    for (int p = d.rowptr[u]; p < d.rowptr[u + 1]; ++p) {
      const int v = d.colind[p];
      const int vx = v % nx, vy = v / nx;
      const bool vsep = ((vx + 1) % (LEAF + 1) == 0) || ((vy + 1) % (LEAF + 1) == 0);
      if (!vsep) {
        T a;
        if constexpr (sizeof(T) == 4) a = d.fval[p]; else a = d.val[p];
        acc += a * X[lay.atc(v, c)];
      }
    }
    X[lay.atc(u, c)] -= acc;
  }
}

// The same update for the chunked FP32 vector (a node's 16 right-hand sides contiguous): one
// thread per separator node and all 16 right-hand sides, so that the row's CSR entries are
// read and classified once instead of once per right-hand side, and the neighbour values move
// as four 16-byte loads.  Same operations in the same order for every right-hand side.
__global__ void sep_update_fwd16_kernel(LeafDev d, float* X) {
  pdl_enter();
  const int nx = d.nx, ny = d.ny;
  const int R = (ny + 1) / (LEAF + 1) - 1, C = (nx + 1) / (LEAF + 1) - 1;
  const long long nrow = (long long)R * nx;
  const long long nsep = nrow + (long long)(ny - R) * C;
  for (long long sidx = blockIdx.x * (long long)blockDim.x + threadIdx.x; sidx < nsep;
       sidx += (long long)gridDim.x * blockDim.x) {
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
    float4 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = d.rowptr[u]; p < d.rowptr[u + 1]; ++p) {
      const int v = d.colind[p];
      const int vx = v % nx, vy = v / nx;
      const bool vsep = ((vx + 1) % (LEAF + 1) == 0) || ((vy + 1) % (LEAF + 1) == 0);
      if (!vsep) {
        const float a = d.fval[p];
        const float4* xv = reinterpret_cast<const float4*>(X + (size_t)v * 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 t = xv[q];
          acc[q].x += a * t.x; acc[q].y += a * t.y; acc[q].z += a * t.z; acc[q].w += a * t.w;
        }
      }
    }
    float4* xu = reinterpret_cast<float4*>(X + (size_t)u * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4 t = xu[q];
      t.x -= acc[q].x; t.y -= acc[q].y; t.z -= acc[q].z; t.w -= acc[q].w;
      xu[q] = t;
    }
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
  {
    const long long n = (long long)nbox * NI * 5;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    leaf_band5_kernel<<<(int)blocks, 256, 0, s>>>(d);
  }
  note_launch();
  if (d.fp32) leaf_lu_kernel<float><<<nbox, LUT, 0, s>>>(d);
  else leaf_lu_kernel<double><<<nbox, LUT, 0, s>>>(d);
  note_launch();
  if (d.fp32) leaf_schur_kernel<float><<<(nbox + LPC - 1) / LPC, FTH, 0, s>>>(d);
  else leaf_schur_kernel<double><<<(nbox + LPC - 1) / LPC, FTH, 0, s>>>(d);
}

template <typename T, int KUW>
static void leaf_solve_go(const LeafDev& d, T* X, int nrhs, VecLayout lay, int bwd, cudaStream_t s) {
  const int grid = (d.g.nbox() + 2 * SWPB - 1) / (2 * SWPB);
  note_launch();
  if (!bwd) {
    const int smem = (int)SolveStage<T, KUW, false>::bytes;
    cudaFuncSetAttribute(leaf_solve_kernel<T, KUW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    launch_pdl(leaf_solve_kernel<T, KUW, false>, dim3(grid), dim3(SWPB * 32), smem, s, d, X, nrhs, lay);
  } else {
    const int smem = (int)SolveStage<T, KUW, true>::bytes;
    cudaFuncSetAttribute(leaf_solve_kernel<T, KUW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    launch_pdl(leaf_solve_kernel<T, KUW, true>, dim3(grid), dim3(SWPB * 32), smem, s, d, X, nrhs, lay);
  }
}

// The FP32 solve vector is always chunked (VecLayout{16, 1, 16 N}: a node's 16 right-hand
// sides contiguous, every chunk 64-byte aligned); the FP32 forward sweep stages its rows as such.
void launch_leaf_solve(const LeafDev& d, void* Xv, int nrhs, VecLayout lay, int bwd, int kumax, cudaStream_t s) {
  if (bwd && d.fp32 && d.G) {
    const int smem = (int)(sizeof(float) * (NI * NQ + NQ * GRC));
    cudaFuncSetAttribute(leaf_bwd_g_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    for (int c0 = 0; c0 < nrhs; c0 += GRC) {
      const int nc = nrhs - c0 < GRC ? nrhs - c0 : GRC;
      note_launch();
      launch_pdl(leaf_bwd_g_kernel, dim3(d.g.nbox()), dim3(GTH), smem, s, d,
                 static_cast<float*>(Xv) + (size_t)(c0 / GRC) * lay.chunk, nc, lay);
    }
    return;
  }
  for (int c0 = 0; c0 < nrhs; c0 += SLOT) {
    const int nc = nrhs - c0 < SLOT ? nrhs - c0 : SLOT;
    if (d.fp32) {
      float* Xc = static_cast<float*>(Xv) + (size_t)(c0 / SLOT) * lay.chunk;
      if (kumax <= 15) leaf_solve_go<float, 16>(d, Xc, nc, lay, bwd, s);
      else leaf_solve_go<float, 32>(d, Xc, nc, lay, bwd, s);
    } else {
      double* Xc = static_cast<double*>(Xv) + (size_t)(c0 / SLOT) * lay.chunk;
      if (kumax <= 15) leaf_solve_go<double, 16>(d, Xc, nc, lay, bwd, s);
      else leaf_solve_go<double, 32>(d, Xc, nc, lay, bwd, s);
    }
  }
}

void launch_sep_update_fwd(const LeafDev& d, void* X, int nrhs, VecLayout lay, cudaStream_t s) {
  const int R = (d.ny + 1) / (LEAF + 1) - 1, C = (d.nx + 1) / (LEAF + 1) - 1;
  long long n = ((long long)R * d.nx + (long long)(d.ny - R) * C) * nrhs;
  if (n <= 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  note_launch();
  if (d.fp32 && lay.cs == 1 && lay.rs == 16) {   // the chunked FP32 vector: a thread per node
    const long long nsep = n / nrhs;
    int b16 = (int)((nsep + 255) / 256);
    if (b16 > 152 * 32) b16 = 152 * 32;
    if (b16 < 1) b16 = 1;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {       // one launch per chunk of 16 right-hand sides
      if (c0 > 0) note_launch();
      launch_pdl(sep_update_fwd16_kernel, dim3(b16), dim3(256), 0, s, d,
                 static_cast<float*>(X) + (size_t)(c0 / 16) * lay.chunk);
    }
  } else if (d.fp32) {
    launch_pdl(sep_update_fwd_kernel<float>, dim3(blocks), dim3(256), 0, s, d, static_cast<float*>(X), nrhs, lay);
  } else {
    launch_pdl(sep_update_fwd_kernel<double>, dim3(blocks), dim3(256), 0, s, d, static_cast<double*>(X), nrhs, lay);
  }
}

}  // namespace spalu
