// Internal declarations of the spaLU CUDA library (not part of the C ABI).
//
// Geometry of the nested dissection on an nx x ny grid (Sec. 2.2, Alg. 1 on a regular
// grid): the boxes of depth d tile the grid in bx x by boxes of w x h interior nodes,
// separated by 1-wide lines.  Box (I, J) covers x in [I(w+1), I(w+1)+w-1] and y in
// [J(h+1), J(h+1)+h-1].  The level-l separators split every depth-(l-1) box into its two
// depth-l children (vertical cut when the parent is at least as wide as tall).
//
// Level-l objects (Sec. 2.3.1, Sec. 3.2), all derived from the depth-l tiling:
//   horizontal segment hs(I,J), 0<=I<bx, 1<=J<by:  sid = I + bx (J-1);
//       line y = J(h+1)-1, below it box (I,J-1) (its owner, the side is that box's TOP),
//       above it box (I,J) (its BOTTOM);
//   vertical segment vs(I,J), 1<=I<bx, 0<=J<by:    sid = nh + (I-1) + (bx-1) J;
//       line x = I(w+1)-1, left box (I-1,J) (owner, its RIGHT side), right box (I,J) (LEFT);
//   junction c(I,J), 1<=I<bx, 1<=J<by: node (I(w+1)-1, J(h+1)-1), id (I-1)+(bx-1)(J-1).
//
// Frontal layout of a depth-d box (position of each boundary unknown in its dense block):
//   BOTTOM [0,w)  TOP [w,2w)  LEFT [2w,2w+h)  RIGHT [2w+h,2w+2h)  corners BL,BR,TL,TR at
//   2w+2h+{0,1,2,3}.  The root (depth 0) has no boundary unknowns (D = 0).  A side holds
//   cnt <= its length unknowns at the start of its range.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spalu.h"

namespace spalu {

enum { SIDE_BOTTOM = 0, SIDE_TOP = 1, SIDE_LEFT = 2, SIDE_RIGHT = 3 };
enum { C_BL = 0, C_BR = 1, C_TL = 2, C_TR = 3 };

// device error word bits
enum { ERR_SINGULAR = 1, ERR_NONFINITE = 2, ERR_CAPACITY = 4, ERR_TIMEOUT = 8 };

// ---- learned rank predictor (no counterpart in the paper): 16 features -> 64 ReLU -> 2
constexpr int PRED_NFEAT = 16;
constexpr int PRED_NHID = 64;
constexpr int PRED_NOUT = 2;
constexpr int PRED_NPARAM = PRED_NHID * PRED_NFEAT + PRED_NHID + PRED_NOUT * PRED_NHID + PRED_NOUT;
constexpr int PRED_PROBE = 8;          // rows of the probe sketch behind features 11-15
constexpr int PRED_MAXBLK = 256;       // blocks of the training gradient kernel
constexpr int PRED_EMAX = 128;         // largest segment the predictor serves
constexpr int PRED_OFF_B1 = PRED_NHID * PRED_NFEAT;
constexpr int PRED_OFF_W2 = PRED_OFF_B1 + PRED_NHID;
constexpr int PRED_OFF_B2 = PRED_OFF_W2 + PRED_NOUT * PRED_NHID;
// predictor modes of a factorization
enum { PRED_OFF = 0, PRED_RECORD = 1, PRED_PREDICT = 2 };
// per-level counters (int) written by the factor kernels
enum { LS_EMAX = 0, LS_KPMAX = 1, LS_DPMAX = 2, LS_PASSES = 3, LS_FALLBACK = 4, LS_PREDICTED = 5, LS_N = 8 };

// Inference copy of the network: feature standardisation and bfloat16 parameters
// (W1 64x16 row-major | b1 | W2 2x64 | b2).
struct PredDev {
  float mu[PRED_NFEAT];
  float isd[PRED_NFEAT];
  __nv_bfloat16 wb[PRED_NPARAM];
};

struct Geo {
  int bx, by, w, h;
  __host__ __device__ int nbox() const { return bx * by; }
  __host__ __device__ int nh() const { return bx * (by - 1); }
  __host__ __device__ int nv() const { return (bx - 1) * by; }
  __host__ __device__ int nseg() const { return nh() + nv(); }
  __host__ __device__ int ncorner() const { return (bx - 1) * (by - 1); }
  __host__ __device__ int D() const { return (bx * by == 1) ? 0 : 2 * w + 2 * h + 4; }
  __host__ __device__ int side_pos(int side) const {
    return side == SIDE_BOTTOM ? 0 : side == SIDE_TOP ? w : side == SIDE_LEFT ? 2 * w : 2 * w + h;
  }
  __host__ __device__ int corner_pos(int c) const { return 2 * w + 2 * h + c; }
  __host__ __device__ int side_len(int side) const { return side < 2 ? w : h; }
  __host__ __device__ int cap() const { return w > h ? w : h; }
  // segment id of a side of box (I,J), or -1 when the side lies on the domain boundary
  __host__ __device__ int box_side(int I, int J, int side) const {
    switch (side) {
      case SIDE_BOTTOM: return J >= 1 ? I + bx * (J - 1) : -1;
      case SIDE_TOP: return J + 1 < by ? I + bx * J : -1;
      case SIDE_LEFT: return I >= 1 ? nh() + (I - 1) + (bx - 1) * J : -1;
      default: return I + 1 < bx ? nh() + I + (bx - 1) * J : -1;
    }
  }
  // junction id of a corner of box (I,J), or -1 on the boundary
  __host__ __device__ int box_corner(int I, int J, int c) const {
    int ci = I + (c & 1), cj = J + (c >> 1);
    if (ci < 1 || ci >= bx || cj < 1 || cj >= by) return -1;
    return (ci - 1) + (bx - 1) * (cj - 1);
  }
  __host__ __device__ int junction_node(int cid, int nx) const {
    int ci = cid % (bx - 1) + 1, cj = cid / (bx - 1) + 1;
    return (ci * (w + 1) - 1) + nx * (cj * (h + 1) - 1);
  }
  // node of the t-th grid point of segment sid (geometric order, increasing coordinate)
  __host__ __device__ int seg_node(int sid, int t, int nx) const {
    if (sid < nh()) {
      int I = sid % bx, J = sid / bx + 1;
      return (I * (w + 1) + t) + nx * (J * (h + 1) - 1);
    }
    int s = sid - nh();
    int I = s % (bx - 1) + 1, J = s / (bx - 1);
    return (I * (w + 1) - 1) + nx * (J * (h + 1) + t);
  }
};

// Merge table (Sec. 4.3, E_(l)) of a depth-(l-1) parent box: one entry of MERGE_TABW ints per
// unknown of its extended block [dP | p]: [0] position in the parent block, [1..3]
// (position, side, skeleton index) in child 1, [4..6] the same in child 2 (-1 when absent;
// side 4 = corner), [7] grid node.
constexpr int MERGE_TABW = 8;

// Resident sparsify CTAs per SM that the occupancy autotuner tries (0: the uncut worst case)
constexpr int SPARS_NCAND = 7;
constexpr int SPARS_CAND_CTAS[SPARS_NCAND] = {0, 2, 3, 4, 6, 8, 12};

struct LevelPlan {          // host-side description of level l (1..L)
  int l;
  int vcut;                 // level-l cut is vertical (children left/right)
  Geo g;                    // depth-l tiling (boxes whose sides are the level-l segments)
  Geo gp;                   // depth-(l-1) tiling (parents)
  int capS;                 // segment capacity at level l = max(w, h)
  int ldF;                  // leading dimension of the depth-l frontal store
  int ldFp;                 // leading dimension of the depth-(l-1) frontal store
  int sepcap;               // length of a level-l separator
  int Ycap;                 // rows of the per-segment sketch buffer
  size_t spars_smem;        // dynamic shared memory of the sparsify kernel
  int spars_global;         // 1 when the worst case needs global scratch
  size_t spars_cand[SPARS_NCAND];   // candidate values of spars_smem (autotuner)
};

// Device view of one level, passed by value to the kernels.
struct LevelDev {
  int l, nx, ny, vcut;
  int fp32;         // real arrays below hold FP32 (mixed mode) instead of FP64
  Geo g, gp;
  int capS, ldF, ldFp, Ycap, sepcap;
  void* F;          // depth-l frontals: nbox * ldF * ldF
  void* Fp;         // depth-(l-1) frontals (merge target): gp.nbox * ldFp * ldFp
  int* cnt;         // [nseg] unknowns per segment before compression
  int* kk;          // [nseg] skeleton size
  int* hs;          // [nseg] final sketch size (statistics)
  int* nodes;       // [nseg * capS] grid nodes in pre-ID order
  int* perm;        // [nseg * capS] column order of the ID (first kk = skeleton)
  int* snodes;      // [nseg * capS] grid nodes in the ID order (nodes[perm[a]]), for the solve
  int* piv;         // [nseg * capS] pivots of the remainder LU
  void* T;          // [nseg * capS * capS] interpolation matrices, k x (e-k), ld capS
  void* Dm;         // [nseg * capS * capS] [A_ss' | Z ; W | LU(A_rr)], ld capS
  void* Dinv;       // [nseg * capS] reciprocal pivots of U(A_rr)
  void* Yg;         // global sketch scratch (nseg * Ycap * capS) or null
  void* Pinv;       // [gp.nbox * sepcap] reciprocal pivots of the separator U
  int* ptab;        // merge tables: gp.nbox * ldFp * 8 ints
  int* order;       // [nseg] launch order of the sparsify CTAs (largest segments first)
  int use_order;    // 1: order is built before each sparsify launch; 0: CTA b is segment b
  int* pcount;      // [gp.nbox * 2]: unknowns of dP, skeleton size of the separator
  int* ppiv;        // [gp.nbox * sepcap] pivots of the separator LU
  int* cnt_up;      // level-(l-1) segment counts (merge target) or null at l = 1
  int* nodes_up;    // level-(l-1) segment nodes or null
  int capS_up;
  // options
  double eps;
  int symmetric, p_over, near_radius, h0;
  int schur_tc;     // separator Schur updates on the tensor cores (mixed path only)
  int sketch_tc;    // sketch products G B_F on the tensor cores (mixed path only)
  unsigned long long seed;
  int* err;
  int* lstat;       // [LS_N] counters of this level (maxima of e, kp, |dP|; ID passes, ...)
  unsigned long long* flops;   // [4] of this level: algorithmic FLOPs of the sparsification and of
                               // the separator eliminations (work.cuh), and the bytes of the
                               // segment factors (T, transformed block, remainder LU, pivots)
                               // and of the separator factors (LU, W, Z, pivots) the solve reads
  int L;            // number of levels of the dissection
  // learned rank predictor
  int pred_mode;            // PRED_OFF / PRED_RECORD / PRED_PREDICT
  double pred_margin;
  double log10eps;          // log10(eps) (features 11-15)
  const PredDev* pred;      // device copy of the network (PRED_PREDICT)
  float* feat;              // [nseg * 16] features (PRED_RECORD)
  int* tgt;                 // [nseg * 4] {k, far rows, valid, ID passes} (PRED_RECORD)
  const int* rowptr;        // original matrix (features 5-10)
  const int* colind;
  const double* val;
  const float4* nstat;      // per grid node {log|A_uu|, log(|A_uu|/off), |row sum|/|A_uu|, asymmetry}
};

// Shared-memory capacities of the solve kernels of one level, set by the host from the
// largest sizes the factor met at that level.
struct SolveCaps {
  int vrows;     // segment: rows of the right-hand-side block (>= every e of the level)
  int lucap;     // order up to which a triangular block is staged
  int pcap;      // segment: elements of each of the two staged panels
  int qcap;      // separator: elements of the staged boundary panel
  int drows;     // separator: parent-boundary rows staged
  int yrows;     // separator: skeleton rows of the right-hand-side block (>= every kp)
  size_t seg_smem, sep_smem;
  int seg_nt, sep_nt;   // CTA widths of the segment / separator solve kernels (64 or 256)
  int seg_split, sep_split;   // right-hand-side groups per segment / separator (CTAs along y)
};

struct LeafDev {
  int nx, ny, L;
  int fp32;         // factors, frontals and solves in FP32 (the LU itself stays FP64)
  Geo g;            // depth-L tiling (leaf boxes, 15 x 15)
  int ldF;          // = g.D()
  void* F;          // depth-L frontals (FP64 or FP32)
  // Band LU of the leaf interiors (FP64 or FP32), one 16-value record per column j of a leaf
  // (leaf b's records start at b * 225 * 16):
  void* lrec;       //   L(j+1+r, j) at slot r = 0..14, slot 15 = pivot row - j (0..15, exact)
  void* urec;       //   1/U_jj at slot 0, U(j-r, j) at slot r = 1..15
  void* uext;       //   U(j-r, j) at slot r - 16 for r = 16..30 (fill of the interchanges), slot 15 = 0
  void* ybuf;       // [nbox * 225 * 64] intermediate vectors of the band sweeps
  void* G;          // [nbox * 225 * 60] FP32 A_II^{-1} A_Id per leaf (row-major, column = side
                    // unknown); mixed path on grids of fewer than LEAF_G_MAX leaves only, where
                    // it replaces the backward sweeps
  void* cpl;        // [nbox * 60] coupling of each side unknown q to its interior neighbour m,
                    // A(m, q) (FP64 or FP32; 0 where the side node is outside the grid)
  double* band5;    // [nbox * 225 * 5] the leaf matrix's nonzeros by column c: A(c + o, c) for
                    // o = -15, -1, 0, 1, 15 (0 where the stencil neighbour is outside the leaf)
  int* kumax;       // largest upper bandwidth of U produced by the interchanges, at least 16
                    // when any leaf made one (<= 15: the sweeps need no interchange step)
  int* kur;         // [nbox] upper bandwidth of each leaf's U
  const int* rowptr;
  const int* colind;
  const double* val;
  const float* fval;  // FP32 copy of val (mixed path)
  int* err;
};

constexpr int LEAF = 15;
constexpr int LEAF_G_MAX = 2048;       // leaves below which the mixed backward leaf step uses G
constexpr int NI = LEAF * LEAF;        // interior unknowns of a leaf
constexpr int KL = LEAF;               // lower bandwidth of the leaf matrix (natural order)
constexpr int KU = LEAF;               // upper bandwidth
constexpr int LDAB = 2 * KL + KU + 1;  // band storage rows (LAPACK layout with pivot fill)

// Kernels launched by this library in this process (diagnostics, spalu_kernel_launches).
void note_launch();

// Programmatic dependent launch: kernels of the solve and refinement sequences are launched
// with launch_pdl, so that a kernel's blocks are set up while its predecessor finishes; each
// such kernel calls pdl_enter() first, which waits until the predecessor grid has completed
// and its writes are visible, then lets the successor launch.  The level-solve kernels split
// the two: pdl_trigger() at entry, then they stage their factor data (written by the
// factorization, whose kernels are launched plainly and so have completed before any solve
// kernel starts), and pdl_wait() before their first read of the solve vector.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Placement of a solve vector: element (grid node u, right-hand side c) at X[u * rs + c * cs];
// the solve kernels take the right-hand sides in chunks of 16, chunk k at X + k * chunk.
// Column-major (ld): {1, ld, 16 ld}; chunk-interleaved (16 values per node): {16, 1, 16 N}.
struct VecLayout {
  long long rs, cs, chunk;
  __host__ __device__ __forceinline__ size_t at(int u, int c) const { return (size_t)(u * rs + c * cs); }
  // any right-hand side c (chunk c / 16, position c % 16 in it)
  __host__ __device__ __forceinline__ size_t atc(int u, int c) const {
    return (size_t)((c >> 4) * chunk + u * rs + (c & 15) * cs);
  }
};

// launch helpers (defined in the .cu files).  The solve launchers take the vector in the
// precision of the factors: float in the mixed path, double otherwise.
void launch_leaf_factor(const LeafDev& d, cudaStream_t s);
void launch_level_init_L(const LevelDev& d, cudaStream_t s);
void launch_sparsify(const LevelDev& d, const LevelPlan& p, cudaStream_t s);
void launch_merge(const LevelDev& d, const LevelPlan& p, cudaStream_t s);

cudaError_t leaf_init_tables();
void launch_leaf_solve(const LeafDev& d, void* X, int nrhs, VecLayout lay, int bwd, int kumax, cudaStream_t s);
void launch_sep_update_fwd(const LeafDev& d, void* X, int nrhs, VecLayout lay, cudaStream_t s);
// Capacities for the level-solve kernels from the level maxima {e, kp, |dP|}; false when
// the right-hand-side blocks alone do not fit in shared memory.
bool level_solve_caps(const LevelDev& d, const int* lstat, SolveCaps* out);
void launch_level_solve_fwd(const LevelDev& d, const SolveCaps& c, void* X, int nrhs, VecLayout lay, cudaStream_t s);
void launch_level_solve_bwd(const LevelDev& d, const SolveCaps& c, void* X, int nrhs, VecLayout lay, cudaStream_t s);

void launch_node_stats(const int* rowptr, const int* colind, const double* val, const float* fval, int n,
                       float4* out, cudaStream_t s);
void launch_pred_fit_norm(const float* X, int n, PredDev* P, cudaStream_t s);
void launch_pred_grad(const float* params, const PredDev* P, const float* X, const float* Y, int r0, int nb,
                      float* partial, float* grad, int* step, cudaStream_t s);
void launch_pred_adam(float* params, float* m, float* v, const float* grad, const int* step, float lr,
                      PredDev* P, cudaStream_t s);
void launch_pred_to_bf16(const float* params, PredDev* P, cudaStream_t s);
void launch_pred_infer(const PredDev* P, const float* X, int n, float* out, cudaStream_t s);
void launch_pred_export(const float* feat, const int* tgt, int nseg, int p, float* X, float* Y, int cap,
                        int* count, cudaStream_t s);

size_t sparsify_smem_need(int e, int symmetric, int h0, int p_over, int tbytes, int chunk);
size_t sparsify_smem_min(int e, int symmetric, int h0, int p_over, int tbytes);
// Dynamic shared memory per sparsify CTA that lets `ctas` of them be resident on one SM
// (the variant that a level of segment capacity capS launches; 0 when that many cannot fit)
size_t sparsify_smem_budget(int fp32, int capS, int ctas);
// Streaming multiprocessors of the current device
int sm_count();

spalu_status residual_noalloc(int n, const int* rowptr, const int* colind, const double* val,
                              const double* B, const double* X, int nrhs, int ld, double* relres,
                              cudaStream_t s);

void launch_nd_perm(int nx, int ny, int L, const int* vcut_host, int* d_perm, int* d_iperm,
                    cudaStream_t s);

}  // namespace spalu
