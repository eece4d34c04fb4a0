// Leaf-interior elimination (Sec. 4.3, first step: L_(L+1)^{-1} A U_(L+1)^{-1} = diag(I, A^(L)))
// and the leaf part of the tree-ordered solve (Eq. (WV)).
//
// One CTA per leaf box.  The 225 x 225 interior block A_II is banded in the natural
// in-leaf order (x fastest): lower and upper bandwidth 15.  Gaussian elimination with
// partial pivoting (pivot = largest |a_ij| in the column, ties -> lowest row) is done in
// LAPACK band storage (kl = ku = 15, 46 rows incl. the fill of the row interchanges),
// which performs exactly the operations of dense partial-pivoting LU on the nonzeros.
// The Schur complement S_b = A_dI A_II^{-1} A_Id onto the 60 side unknowns needs
// A_II^{-1} only at the ring of interior nodes next to the sides, because every side
// unknown couples to exactly one interior node; it is formed from 60 band solves.
#include <cstdio>

#include "spalu_internal.h"

namespace spalu {
namespace {

constexpr int KV = KL + KU;   // row of the diagonal in band storage
constexpr int NQ = 4 * LEAF;  // side unknowns of a leaf
constexpr int RHS_CHUNK = 16; // right-hand sides per pass of the Schur solves

__device__ __forceinline__ double& ab(double* AB, int i, int j) { return AB[(KV + i - j) + LDAB * j]; }

// Position of grid node (vx, vy) in the frontal layout of the leaf box at (x0, y0), or -1.
__device__ int leaf_frontal_pos(int vx, int vy, int x0, int y0) {
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

// side unknown q (0..59, sides BOTTOM, TOP, LEFT, RIGHT of 15 each): its grid node and
// the local index of its single interior neighbour.
__device__ void side_unknown(int q, int x0, int y0, int* vx, int* vy, int* m) {
  int s = q / LEAF, t = q % LEAF;
  switch (s) {
    case SIDE_BOTTOM: *vx = x0 + t; *vy = y0 - 1; *m = t; break;
    case SIDE_TOP: *vx = x0 + t; *vy = y0 + LEAF; *m = t + LEAF * (LEAF - 1); break;
    case SIDE_LEFT: *vx = x0 - 1; *vy = y0 + t; *m = LEAF * t; break;
    default: *vx = x0 + LEAF; *vy = y0 + t; *m = LEAF * t + LEAF - 1; break;
  }
}

__device__ double csr_entry(const int* rowptr, const int* colind, const double* val, int r, int c) {
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p)
    if (colind[p] == c) return val[p];
  return 0.0;
}

// Band GEPP (the dgbtf2 sequence) by the whole CTA; multipliers stay in their column.
__device__ bool band_gepp(double* AB, int* piv, int* sh_int) {
  int ju = 0;
  bool ok = true;
  for (int j = 0; j < NI; ++j) {
    const int km = min(KL, NI - 1 - j);
    if (threadIdx.x < 32) {                       // pivot search: warp 0
      double best = -1.0;
      int bi = 0;
      for (int r = threadIdx.x; r <= km; r += 32) {
        double v = fabs(ab(AB, j + r, j));
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        sh_int[0] = bi;
        piv[j] = j + bi;
        sh_int[1] = (best == 0.0) ? 1 : 0;
      }
    }
    __syncthreads();
    const int jp = sh_int[0];
    if (sh_int[1]) { ok = false; __syncthreads(); continue; }
    ju = max(ju, min(j + KU + jp, NI - 1));
    if (jp != 0) {
      for (int c = j + threadIdx.x; c <= ju; c += blockDim.x) {
        double a = ab(AB, j, c), b = ab(AB, j + jp, c);
        ab(AB, j, c) = b;
        ab(AB, j + jp, c) = a;
      }
      __syncthreads();
    }
    const double piv_v = ab(AB, j, j);
    for (int r = 1 + threadIdx.x; r <= km; r += blockDim.x) ab(AB, j + r, j) /= piv_v;
    __syncthreads();
    // rank-1 update of rows j+1..j+km, columns j+1..ju
    const int ncol = ju - j;
    for (int e = threadIdx.x; e < km * ncol; e += blockDim.x) {
      int r = 1 + e % km, c = j + 1 + e / km;
      ab(AB, j + r, c) -= ab(AB, j + r, j) * ab(AB, j, c);
    }
    __syncthreads();
  }
  return ok;
}

// Solve with the band LU for ncol columns X (ld NI), one warp per column.
__device__ void band_solve_cols(const double* AB, const int* piv, double* X, int ncol) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < ncol; q += nw) {
    double* x = X + (size_t)q * NI;
    for (int j = 0; j < NI; ++j) {                 // L: interchanges then unit lower
      int p = piv[j];
      if (p != j) {
        __syncwarp();
        if (lane == 0) { double t = x[j]; x[j] = x[p]; x[p] = t; }
      }
      __syncwarp();
      double xj = x[j];
      int km = min(KL, NI - 1 - j);
      if (lane < km) x[j + 1 + lane] -= ab(const_cast<double*>(AB), j + 1 + lane, j) * xj;
    }
    __syncwarp();
    for (int j = NI - 1; j >= 0; --j) {            // U: upper bandwidth KL+KU
      __syncwarp();
      double xj = x[j] / ab(const_cast<double*>(AB), j, j);
      __syncwarp();
      if (lane == 0) x[j] = xj;
      int i0 = max(0, j - KV);
      for (int i = i0 + lane; i < j; i += 32) x[i] -= ab(const_cast<double*>(AB), i, j) * xj;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) leaf_factor_kernel(LeafDev d) {
  extern __shared__ double sm[];
  double* AB = sm;                                   // LDAB * NI
  double* X = AB + LDAB * NI;                        // NI * RHS_CHUNK
  double* qa = X + NI * RHS_CHUNK;                   // NQ: A[q, m_q]
  double* qc = qa + NQ;                              // NQ: A[m_q, q]
  int* piv = reinterpret_cast<int*>(qc + NQ);        // NI
  int* qm = piv + NI;                                // NQ: interior neighbour (local index)
  int* qex = qm + NQ;                                // NQ: side exists
  int* sh_int = qex + NQ;                            // scratch

  const int b = blockIdx.x;
  const Geo g = d.g;
  const int I = b % g.bx, J = b / g.bx;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  double* F = d.F + (size_t)b * d.ldF * d.ldF;
  const int D = g.D();

  for (int i = threadIdx.x; i < LDAB * NI; i += blockDim.x) AB[i] = 0.0;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) F[(e % D) + (size_t)d.ldF * (e / D)] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < NI; i += blockDim.x) {
    int row = (x0 + i % LEAF) + nx * (y0 + i / LEAF);
    for (int p = d.rowptr[row]; p < d.rowptr[row + 1]; ++p) {
      int c = d.colind[p];
      int cx = c % nx - x0, cy = c / nx - y0;
      if (cx >= 0 && cx < LEAF && cy >= 0 && cy < LEAF) ab(AB, i, cx + LEAF * cy) += d.val[p];
    }
  }
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
    int vx, vy, m;
    side_unknown(q, x0, y0, &vx, &vy, &m);
    bool exists = vx >= 0 && vx < nx && vy >= 0 && vy < d.ny;
    qm[q] = m;
    qex[q] = exists ? 1 : 0;
    double a = 0.0, c = 0.0;
    if (exists) {
      int node = vx + nx * vy;
      int mnode = (x0 + m % LEAF) + nx * (y0 + m / LEAF);
      a = csr_entry(d.rowptr, d.colind, d.val, node, mnode);
      c = csr_entry(d.rowptr, d.colind, d.val, mnode, node);
    }
    qa[q] = a;
    qc[q] = c;
  }
  __syncthreads();

  const bool ok = band_gepp(AB, piv, sh_int);
  if (!ok && threadIdx.x == 0) atomicOr(d.err, ERR_SINGULAR);

  // F[i][q] = -A[i, m_i] (A_II^{-1})[m_i, m_q] A[m_q, q]: the Schur complement S_b
  for (int q0 = 0; q0 < NQ; q0 += RHS_CHUNK) {
    const int nc = min(RHS_CHUNK, NQ - q0);
    for (int e = threadIdx.x; e < NI * nc; e += blockDim.x) X[e] = 0.0;
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
      if (qex[q0 + c]) X[(size_t)c * NI + qm[q0 + c]] = qc[q0 + c];
    __syncthreads();
    if (ok) band_solve_cols(AB, piv, X, nc);
    __syncthreads();
    for (int e = threadIdx.x; e < NQ * nc; e += blockDim.x) {
      int i = e % NQ, c = e / NQ;
      if (qex[i] && qex[q0 + c]) F[i + (size_t)d.ldF * (q0 + c)] = -qa[i] * X[(size_t)c * NI + qm[i]];
    }
    __syncthreads();
  }

  // original couplings owned by this box: its TOP and RIGHT sides (it is their lower /
  // left box) with their end junctions, and the diagonal of its BL junction.
  //   task 0..14  : TOP side row      -> TOP, TL, TR
  //   task 15..29 : RIGHT side row    -> RIGHT, BR, TR
  //   task 30     : TL junction row   -> TOP
  //   task 31     : TR junction row   -> TOP, RIGHT
  //   task 32     : BR junction row   -> RIGHT
  //   task 33     : BL junction row   -> BL
  const int tk = threadIdx.x;
  if (tk < 2 * LEAF + 4) {
    int vx, vy;
    if (tk < LEAF) { vx = x0 + tk; vy = y0 + LEAF; }
    else if (tk < 2 * LEAF) { vx = x0 + LEAF; vy = y0 + tk - LEAF; }
    else if (tk == 30) { vx = x0 - 1; vy = y0 + LEAF; }
    else if (tk == 31) { vx = x0 + LEAF; vy = y0 + LEAF; }
    else if (tk == 32) { vx = x0 + LEAF; vy = y0 - 1; }
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
        if (tk < LEAF) take = on_top || pj == 4 * LEAF + C_TL || pj == 4 * LEAF + C_TR;
        else if (tk < 2 * LEAF) take = on_right || pj == 4 * LEAF + C_BR || pj == 4 * LEAF + C_TR;
        else if (tk == 30) take = on_top;
        else if (tk == 31) take = on_top || on_right;
        else if (tk == 32) take = on_right;
        else take = (pj == pi);
        if (take) F[pi + (size_t)d.ldF * pj] += d.val[p];
      }
    }
  }
  // keep the band LU and pivots for the solve
  double* band = d.band + (size_t)b * LDAB * NI;
  for (int i = threadIdx.x; i < LDAB * NI; i += blockDim.x) band[i] = AB[i];
  for (int i = threadIdx.x; i < NI; i += blockDim.x) d.piv[(size_t)b * NI + i] = piv[i];
}

// ---------------------------------------------------------------- solve
// Forward (leaf part of W~): t = A_II^{-1} b_I stored in X[I]; the side unknowns are
// updated afterwards by sep_update_fwd_kernel (b_d -= A_dI t).
__global__ void leaf_solve_kernel(LeafDev d, double* X, int nrhs, int ld, int bwd, const double* tmp) {
  extern __shared__ double sm[];
  double* AB = sm;
  double* x = AB + LDAB * NI;         // NI * nrhs
  int* piv = reinterpret_cast<int*>(x + (size_t)NI * nrhs);
  const int b = blockIdx.x;
  const int I = b % d.g.bx, J = b / d.g.bx;
  const int x0 = I * (LEAF + 1), y0 = J * (LEAF + 1);
  const int nx = d.nx;
  const double* band = d.band + (size_t)b * LDAB * NI;
  for (int i = threadIdx.x; i < LDAB * NI; i += blockDim.x) AB[i] = band[i];
  for (int i = threadIdx.x; i < NI; i += blockDim.x) piv[i] = d.piv[(size_t)b * NI + i];
  for (int e = threadIdx.x; e < NI * nrhs; e += blockDim.x) {
    int i = e % NI, c = e / NI;
    int node = (x0 + i % LEAF) + nx * (y0 + i / LEAF);
    double v;
    if (!bwd) {
      v = X[node + (size_t)ld * c];
    } else {
      // b_I <- A_Id x_d  (couplings to side unknowns)
      v = 0.0;
      for (int p = d.rowptr[node]; p < d.rowptr[node + 1]; ++p) {
        int cc = d.colind[p];
        int cx = cc % nx - x0, cy = cc / nx - y0;
        if (!(cx >= 0 && cx < LEAF && cy >= 0 && cy < LEAF)) v += d.val[p] * X[cc + (size_t)ld * c];
      }
    }
    x[e] = v;
  }
  __syncthreads();
  band_solve_cols(AB, piv, x, nrhs);
  __syncthreads();
  for (int e = threadIdx.x; e < NI * nrhs; e += blockDim.x) {
    int i = e % NI, c = e / NI;
    int node = (x0 + i % LEAF) + nx * (y0 + i / LEAF);
    if (!bwd) X[node + (size_t)ld * c] = x[e];
    else X[node + (size_t)ld * c] -= x[e];         // x_I = t - A_II^{-1} A_Id x_d
  }
}

// b_u -= sum over interior neighbours j of A_uj t_j, for every separator node u.
__global__ void sep_update_fwd_kernel(LeafDev d, double* X, int nrhs, int ld) {
  const int nx = d.nx, ny = d.ny;
  const long long n = (long long)nx * ny;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    int u = (int)(e % n), c = (int)(e / n);
    int ux = u % nx, uy = u / nx;
    bool sep = ((ux + 1) % (LEAF + 1) == 0) || ((uy + 1) % (LEAF + 1) == 0);
    if (!sep) continue;
    double acc = 0.0;
    for (int p = d.rowptr[u]; p < d.rowptr[u + 1]; ++p) {
      int v = d.colind[p];
      int vx = v % nx, vy = v / nx;
      bool vsep = ((vx + 1) % (LEAF + 1) == 0) || ((vy + 1) % (LEAF + 1) == 0);
      if (!vsep) acc += d.val[p] * X[v + (size_t)ld * c];
    }
    X[u + (size_t)ld * c] -= acc;
  }
}

}  // namespace

static size_t leaf_factor_smem() {
  return sizeof(double) * (LDAB * NI + NI * RHS_CHUNK + 2 * NQ) + sizeof(int) * (NI + 2 * NQ + 8);
}

void launch_leaf_factor(const LeafDev& d, cudaStream_t s) {
  size_t smem = leaf_factor_smem();
  cudaFuncSetAttribute(leaf_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  leaf_factor_kernel<<<d.g.nbox(), 256, smem, s>>>(d);
}

static size_t leaf_solve_smem(int nrhs) {
  return sizeof(double) * (LDAB * NI + (size_t)NI * nrhs) + sizeof(int) * NI;
}

void launch_leaf_solve_fwd(const LeafDev& d, double* X, int nrhs, int ld, cudaStream_t s) {
  size_t smem = leaf_solve_smem(nrhs);
  cudaFuncSetAttribute(leaf_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  leaf_solve_kernel<<<d.g.nbox(), 256, smem, s>>>(d, X, nrhs, ld, 0, nullptr);
}

void launch_sep_update_fwd(const LeafDev& d, double* X, int nrhs, int ld, cudaStream_t s) {
  long long n = (long long)d.nx * d.ny * nrhs;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  note_launch();
  sep_update_fwd_kernel<<<blocks, 256, 0, s>>>(d, X, nrhs, ld);
}

void launch_leaf_solve_bwd(const LeafDev& d, double* X, int nrhs, int ld, double* tmp, cudaStream_t s) {
  size_t smem = leaf_solve_smem(nrhs);
  cudaFuncSetAttribute(leaf_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  leaf_solve_kernel<<<d.g.nbox(), 256, smem, s>>>(d, X, nrhs, ld, 1, tmp);
}

}  // namespace spalu
