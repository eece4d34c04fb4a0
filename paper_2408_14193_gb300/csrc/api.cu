// C ABI of the spaLU library: nested-dissection handle, factor handle (one device arena
// planned from the grid), numeric factorization (Alg. 2), tree-ordered solve (Eq. (WV)) and
// GMRES refinement.  See include/spalu.h for the contract of every entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "spalu_internal.h"

using namespace spalu;

struct spalu_nd_s {
  int nx, ny, L;
  std::vector<Geo> depth;   // depth 0..L tilings
  std::vector<int> vcut;    // [1..L]
  int* d_perm = nullptr;
  int* d_iperm = nullptr;
  cudaStream_t stream = nullptr;
};

struct GmresWork {
  int nrhs = 0, m = 0;
  double* V = nullptr;      // (m+1) * N * nrhs   Krylov basis
  double* Z = nullptr;      // m * N * nrhs       M^{-1} V_j, kept for the update (no final solve)
  unsigned* cnt = nullptr;  // ticket counters of the column sums, one per column chunk
  double* part = nullptr;   // partial sums
  double* hcol = nullptr;   // device coefficients (m+2) * nrhs
  double* vs = nullptr;     // (m+2) * nrhs: basis vector j is vs[j] x V_j (stored unnormalized)
  double* vec = nullptr;    // nrhs scalars
  // device-side least-squares state of the Arnoldi cycle (one column per right-hand side)
  double* H = nullptr;      // nrhs * (m+1) * m  rotated Hessenberg columns
  double* cs = nullptr;     // nrhs * m          Givens cosines
  double* sn = nullptr;     // nrhs * m          Givens sines
  double* g = nullptr;      // nrhs * (m+1)      rotated right-hand side
  double* y = nullptr;      // m * nrhs          coefficients of the update
  double* bn = nullptr;     // nrhs              ||b_c||
  double* beta = nullptr;   // nrhs              ||b_c - A x_c||
  int* st = nullptr;        // 4 * nrhs: [active, kdim, its, converged-at-start] per column
  int* flag = nullptr;      // [0]: some column still active
  int* hflag = nullptr;     // page-locked copy of flag[0]
};

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void spalu::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void note_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

struct PhaseTimer {
  bool on = false;
  struct Rec { std::string name; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, double> ms;
  std::map<std::string, long long> count;
  cudaEvent_t take() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // While the step graph is captured, intervals on its top-level stream become event nodes of
  // the graph (kept in grecs and read after every replay); other capturing streams (the bodies
  // of conditional nodes, which cannot hold event nodes) record nothing.
  cudaStream_t cap_top = nullptr;
  std::vector<Rec> grecs;
  // open an interval on stream s; returns its index (-1 when timing is off or not possible)
  int begin(const std::string& name, cudaStream_t s) {
    if (!on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return -1;
    if (cs != cudaStreamCaptureStatusNone) {
      if (s != cap_top) return -1;
      Rec r{name, take(), take()};
      // external: an event-record node of the graph (a plain record in a capture only orders
      // the captured work)
      if (cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal) != cudaSuccess) {
        cudaGetLastError();
        pool.push_back(r.a);
        pool.push_back(r.b);
        return -1;
      }
      grecs.push_back(r);
      return -2 - ((int)grecs.size() - 1);
    }
    Rec r{name, take(), take()};
    cudaEventRecord(r.a, s);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int i, cudaStream_t s) {
    if (i >= 0) cudaEventRecord(recs[i].b, s);
    else if (i <= -2) cudaEventRecordWithFlags(grecs[-2 - i].b, s, cudaEventRecordExternal);
  }
  // add the intervals of the last replay of the step graph to the sums (events kept)
  void collect_graph() {
    for (auto& r : grecs) {
      float t = 0.f;
      cudaEventSynchronize(r.b);
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) { ms[r.name] += t; count[r.name] += 1; }
      else cudaGetLastError();
    }
  }
  void drop_graph() {
    for (auto& r : grecs) { pool.push_back(r.a); pool.push_back(r.b); }
    grecs.clear();
  }
  // fold the finished intervals into the sums
  void collect() {
    for (auto& r : recs) {
      float t = 0.f;
      cudaEventSynchronize(r.b);
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) { ms[r.name] += t; count[r.name] += 1; }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  void reset() { collect(); ms.clear(); count.clear(); }
  ~PhaseTimer() {
    for (auto& r : recs) { pool.push_back(r.a); pool.push_back(r.b); }
    drop_graph();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct spalu_factor_s {
  spalu_nd_s* nd = nullptr;
  spalu_opts o{};
  int N = 0, nnz_cap = 0;
  std::vector<LevelPlan> plan;   // [1..L]
  std::vector<LevelDev> lev;     // [1..L]
  LeafDev leaf{};
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int* d_err = nullptr;
  int* rowptr = nullptr;
  int* colind = nullptr;
  double* val = nullptr;
  float* fval = nullptr;     // FP32 copy of val (mixed path: the solve's separator update)
  int nnz = 0;
  bool factored = false;
  float* xf = nullptr;       // FP32 solve vector of the mixed path, N x xf_cols
  int xf_cols = 0;
  int* hpin = nullptr;       // page-locked readback after a factorization: err, kumax, lstat
  std::vector<int> tuned_nt; // [4 * (L + 1)] per level: segment / separator solve CTA widths and
                             // right-hand-side groups chosen by spalu_tune_solve (0: none)
  cudaStream_t up = nullptr; // second stream of spalu_factor_solve_host (right-hand-side upload)
  cudaEvent_t up_go = nullptr, up_done = nullptr;
  double* hB = nullptr;      // device B and X of spalu_factor_solve_host, hcap doubles each
  double* hX = nullptr;
  size_t hcap = 0;
  cudaStream_t last_stream = nullptr;
  GmresWork gw;
  PhaseTimer timer;
  int kumax = 30;            // upper bandwidth of the leaf U factors (read after each factor)
  int gmres_hint = 1;        // Arnoldi steps the last single-cycle refinement needed
  struct StepGraph {         // spalu_factor_solve_graph: the captured step and what it was captured for
    cudaGraphExec_t exec = nullptr;
    const void* key[6] = {};
    int nnz = -1, nrhs = -1, ld = -1, K = 0;
    bool timed = false;      // captured with per-phase timing on (event nodes in the graph)
    int* d_ref = nullptr;    // guard references: captured level maxima (3 per level) and kumax
    int* d_ok = nullptr;     // guard result
    int* h_out = nullptr;    // page-locked: guard result, some column active
    long long n_pre = 0, n_ok = 0;   // kernels of the graph: before the guard's node, in its body
    long long captures = 0, replays = 0, refits = 0, continued = 0;   // statistics (spalu_stats)
    std::vector<long long> n_step;   // ... and in each Arnoldi step's node
  } sg;
  int* d_lstat = nullptr;    // [LS_N * (L + 1)] per-level counters (factor kernels)
  unsigned long long* d_flops = nullptr;   // [4 * (L + 1)] per level: algorithmic FLOPs of the sparsify
                                           // and merge phases, bytes of the segment and separator factors
  std::vector<int> lstat;    // host copy after the last factor
  std::vector<SolveCaps> caps;   // [1..L] solve-kernel capacities from the last factor
  int* d_tgt_all = nullptr;  // recorded targets of all levels (4 ints per segment)
  int* d_count = nullptr;    // export row counter
  float4* d_nstat = nullptr; // per-node matrix statistics (predictor features)
  size_t tgt_ints = 0;
  spalu_predictor_t pred = nullptr;
  int pred_mode = PRED_OFF;
};

struct spalu_predictor_s {
  float* params = nullptr;   // FP32 master parameters
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;     // PRED_NPARAM + 1 (last: sum of squared residuals)
  float* partial = nullptr;  // PRED_MAXBLK x (PRED_NPARAM + 1)
  int* step = nullptr;       // Adam step counter
  PredDev* dev = nullptr;    // inference copy (standardisation + bfloat16 parameters)
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  cudaGraphExec_t epoch = nullptr;     // captured training epoch
  const float* g_X = nullptr;          // the arguments the epoch graph was captured with
  const float* g_Y = nullptr;
  int g_n = 0, g_batch = 0;
  float g_lr = 0.f;
};

namespace {

const int kPitch = 16;

bool side_ok(int n) {
  if (n < LEAF || (n + 1) % kPitch) return false;
  int q = (n + 1) / kPitch;
  return (q & (q - 1)) == 0;
}

// With SPALU_DEBUG set in the environment, a failing CUDA call is reported on stderr.
void report_cuda(const char* what, cudaError_t e, int line) {
  static const bool on = std::getenv("SPALU_DEBUG") != nullptr;
  if (on) std::fprintf(stderr, "spalu: %s failed at api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
}

#define CUDA_TRY(x)                                   \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) {                          \
      report_cuda(#x, _e, __LINE__);                  \
      return SPALU_ERR_CUDA;                          \
    }                                                 \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <class T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// ------------------------------------------------------------ GMRES helper kernels
// Vector kernels over N rows x nrhs columns: one thread per row and RC columns (blockIdx.y =
// column chunk), so a row of the CSR matrix is read once per chunk.  Column sums are
// deterministic: each block writes one partial per column, and the last block of a chunk to
// finish (ticket counter, reset by that block) adds the partials in block order.
constexpr int RC = 8;
constexpr int VB = 256;                  // threads per block of the vector kernels
constexpr int VNB = 1024;                // most blocks per column chunk (partial buffer width)

static_assert(VB == 32 * RC, "one warp per column of a chunk in the block sums");
__device__ void column_sums(double (&s)[RC], int c0, int nrhs, double* part, unsigned* cnt,
                            double* out, int sq, const double* oscale = nullptr, double* inv_out = nullptr) {
  __shared__ double red[RC][VB];
  __shared__ int last;
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;   // warp k sums column c0 + k
  const int nb = gridDim.x;
  const bool valid = c0 + k < nrhs;
#pragma unroll
  for (int i = 0; i < RC; ++i) red[i][threadIdx.x] = s[i];
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int m = 0; m < VB / 32; ++m) t += red[k][lane + 32 * m];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0 && valid) {
    part[(size_t)(c0 + k) * nb + blockIdx.x] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt + blockIdx.y, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  t = 0.0;
  if (valid)
    for (int i = lane; i < nb; i += 32) t += __ldcg(part + (size_t)(c0 + k) * nb + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0 && valid) {
    double o = sq ? sqrt(t) : t;
    if (oscale) o *= oscale[c0 + k];
    out[c0 + k] = o;
    if (inv_out) inv_out[c0 + k] = o != 0.0 ? 1.0 / o : 0.0;
  }
  if (threadIdx.x == 0) cnt[blockIdx.y] = 0u;
}

// y = b - A x (b null: y = A x); when part is set, out[c] = <y_c, d_c> (d null: ||y_c||, sq).
// No array aliases another, so the loads of b and d need not wait for the stores of y.
__global__ void __launch_bounds__(VB, 4) spmv_kernel(int n, int nrhs, const int* __restrict__ rowptr,
                                                  const int* __restrict__ colind,
                                                  const double* __restrict__ val, const double* __restrict__ x,
                                                  int ldx, const double* __restrict__ b, int ldb,
                                                  double* __restrict__ y, int ldy, const double* __restrict__ d,
                                                  int ldd, const double* dscale, double* part, unsigned* cnt,
                                                  double* out, int sq) {
  pdl_enter();
  const int c0 = blockIdx.y * RC;
  const int nc = nrhs - c0 < RC ? nrhs - c0 : RC;
  double s[RC];
#pragma unroll
  for (int k = 0; k < RC; ++k) s[k] = 0.0;
  for (long long r = blockIdx.x * (long long)VB + threadIdx.x; r < n; r += (long long)gridDim.x * VB) {
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    const int p0 = __ldg(rowptr + r), p1 = __ldg(rowptr + r + 1);
    for (int p = p0; p < p1; ++p) {
      const int col = __ldg(colind + p);
      const double v = __ldg(val + p);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < nc) acc[k] += v * __ldg(x + col + (size_t)ldx * (c0 + k));
    }
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k < nc) {
        const double yv = b ? __ldcs(b + r + (size_t)ldb * (c0 + k)) - acc[k] : acc[k];
        y[r + (size_t)ldy * (c0 + k)] = yv;
        s[k] += yv * (d ? __ldcs(d + r + (size_t)ldd * (c0 + k)) : yv);
      }
  }
  if (part) column_sums(s, c0, nrhs, part, cnt, out, sq, dscale);
}

// One modified Gram-Schmidt pass on unnormalized basis vectors (vector i stands for
// scale_i x stored_i): w_c -= h_c ps_c p_c (skipped when p is null), then
// out[c] = qs_c <w_c, q_c> (q null: ||w_c|| (sq) and inv_out[c] = 1 / out[c]).  The operands
// of four columns of a row are loaded before their stores (w, p and q never alias), so a row
// costs two memory round trips rather than two per column.
constexpr int RH = RC / 2;
__global__ void __launch_bounds__(VB, 4) mgs_kernel(int n, int nrhs, const double* h,
                                                 const double* __restrict__ p, int ldp, const double* ps,
                                                 double* __restrict__ w, int ldw, const double* __restrict__ q,
                                                 int ldq, const double* qs, double* part, unsigned* cnt,
                                                 double* out, int sq, double* inv_out) {
  pdl_enter();
  const int c0 = blockIdx.y * RC;
  const int nc = nrhs - c0 < RC ? nrhs - c0 : RC;
  double s[RC], hc[RC];
#pragma unroll
  for (int k = 0; k < RC; ++k) {
    s[k] = 0.0;
    hc[k] = (p && k < nc) ? (ps ? h[c0 + k] * ps[c0 + k] : h[c0 + k]) : 0.0;
  }
  for (long long r = blockIdx.x * (long long)VB + threadIdx.x; r < n; r += (long long)gridDim.x * VB) {
#pragma unroll
    for (int k0 = 0; k0 < RC; k0 += RH) {
      double wv[RH], pv[RH], qv[RH];
#pragma unroll
      for (int j = 0; j < RH; ++j) {
        const int k = k0 + j;
        wv[j] = k < nc ? w[r + (size_t)ldw * (c0 + k)] : 0.0;
        pv[j] = (p && k < nc) ? __ldcs(p + r + (size_t)ldp * (c0 + k)) : 0.0;
        qv[j] = (q && k < nc) ? __ldcs(q + r + (size_t)ldq * (c0 + k)) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < RH; ++j) {
        const int k = k0 + j;
        if (k < nc) {
          if (p) {
            wv[j] -= hc[k] * pv[j];
            w[r + (size_t)ldw * (c0 + k)] = wv[j];
          }
          s[k] += wv[j] * (q ? qv[j] : wv[j]);
        }
      }
    }
  }
  column_sums(s, c0, nrhs, part, cnt, out, sq, q ? qs : nullptr, inv_out);
}

// X_c += sum_i y[i][c] Z_i,c for i = 0..k_c-1, in that order (Z_i = Z + i * ldz * nrhs); k_c = k,
// or with st the steps column c took in the cycle (later Z_i were not written for it)
__global__ void __launch_bounds__(VB, 4) combine_kernel(int n, int nrhs, int k, const double* __restrict__ y,
                                                     const double* __restrict__ Z, size_t ldz,
                                                     double* __restrict__ X, int ldx, const int* st) {
  pdl_enter();
  const int c0 = blockIdx.y * RC;
  const int nc = nrhs - c0 < RC ? nrhs - c0 : RC;
  int kc[RC];
#pragma unroll
  for (int kk = 0; kk < RC; ++kk) {
    const int c = c0 + kk;
    kc[kk] = (st && kk < nc) ? (st[4 * c + 3] ? 0 : min(k, st[4 * c + 1])) : k;
  }
  for (long long r = blockIdx.x * (long long)VB + threadIdx.x; r < n; r += (long long)gridDim.x * VB) {
#pragma unroll
    for (int kk = 0; kk < RC; ++kk)
      if (kk < nc) {
        const int c = c0 + kk;
        double xv = X[r + (size_t)ldx * c];
        for (int i = 0; i < kc[kk]; ++i) xv += y[(size_t)i * nrhs + c] * Z[(size_t)i * ldz * nrhs + r + ldz * c];
        X[r + (size_t)ldx * c] = xv;
      }
  }
}

// ---- least-squares side of GMRES on the device (one thread per column, one block): the
// Givens rotations that keep the Hessenberg matrix upper triangular, the residual estimate
// |g_{j+1}| (the stop test) and the back substitution for the update coefficients, so the
// Arnoldi loop needs no host round trip.  Column c's state st[4c..4c+3] = {active, steps of
// this cycle, steps in all, converged when the cycle began}; flag[0] = some column active,
// also passed to a graph conditional node when one is given.
constexpr int GB = 256;

__device__ __forceinline__ void publish_active(int any, int* flag, cudaGraphConditionalHandle h, int use_h) {
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    flag[0] = any;
    if (use_h) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// start of a cycle: beta = ||b - A x|| is in; V_0 = r / beta (scale vs_0), g = beta e_1;
// columns already at the tolerance stay out of the cycle (scale 0)
__global__ void __launch_bounds__(GB) gmres_begin_kernel(int nrhs, int m, double tol, const double* bn,
                                                       const double* beta, double* vs, double* g, int* st,
                                                       int first, int* flag, cudaGraphConditionalHandle h,
                                                       int use_h) {
  int any = 0;
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    const double b = bn[c], r = beta[c];
    const bool done = b == 0.0 || r <= tol * b;
    const double bsc = done ? 0.0 : r;
    vs[c] = bsc != 0.0 ? 1.0 / bsc : 0.0;
    g[(size_t)c * (m + 1)] = bsc;
    int* sc = st + 4 * c;
    sc[0] = done ? 0 : 1;
    sc[1] = 0;
    if (first) sc[2] = 0;
    sc[3] = done ? 1 : 0;
    any |= done ? 0 : 1;
  }
  publish_active(any, flag, h, use_h);
}

// after Arnoldi step j: the new Hessenberg column h_0..h_{j+1} (hcol) is rotated by the
// previous rotations, a new rotation zeroes h_{j+1}, and g follows; a column whose |g_{j+1}|
// reaches tol ||b|| leaves the cycle (its later basis vectors get scale 0)
__global__ void __launch_bounds__(GB) gmres_givens_kernel(int nrhs, int m, int j, double tol, const double* hcol,
                                                        const double* bn, double* H, double* cs, double* sn,
                                                        double* g, double* vs, int* st, int* flag,
                                                        cudaGraphConditionalHandle h, int use_h) {
  pdl_enter();
  int any = 0;
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    int* sc = st + 4 * c;
    if (!sc[0]) {
      vs[(size_t)(j + 1) * nrhs + c] = 0.0;
      continue;
    }
    double* Hc = H + (size_t)c * (m + 1) * m + (size_t)(m + 1) * j;
    double* csc = cs + (size_t)c * m;
    double* snc = sn + (size_t)c * m;
    double* gc = g + (size_t)c * (m + 1);
    for (int i = 0; i <= j + 1; ++i) Hc[i] = hcol[(size_t)i * nrhs + c];
    for (int i = 0; i < j; ++i) {
      const double a = Hc[i], b = Hc[i + 1];
      Hc[i] = csc[i] * a + snc[i] * b;
      Hc[i + 1] = -snc[i] * a + csc[i] * b;
    }
    const double a = Hc[j], b = Hc[j + 1];
    const double den = hypot(a, b);
    csc[j] = den == 0.0 ? 1.0 : a / den;
    snc[j] = den == 0.0 ? 0.0 : b / den;
    Hc[j] = den;
    Hc[j + 1] = 0.0;
    gc[j + 1] = -snc[j] * gc[j];
    gc[j] = csc[j] * gc[j];
    sc[1] = j + 1;
    if (fabs(gc[j + 1]) <= tol * bn[c]) {
      sc[0] = 0;
      vs[(size_t)(j + 1) * nrhs + c] = 0.0;
    }
    any |= sc[0];
  }
  publish_active(any, flag, h, use_h);
}

// end of a cycle: y (kmax x nrhs, row-major by step) from the triangular system R y = g
// over each column's own steps; zero beyond them and for columns that sat the cycle out
__global__ void __launch_bounds__(GB) gmres_ysolve_kernel(int nrhs, int m, int kmax, const double* H,
                                                        const double* g, double* y, int* st) {
  pdl_enter();
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    int* sc = st + 4 * c;
    const int k = sc[3] ? 0 : sc[1];
    const double* Hc = H + (size_t)c * (m + 1) * m;
    const double* gc = g + (size_t)c * (m + 1);
    for (int i = kmax - 1; i >= 0; --i) {
      if (i >= k) {
        y[(size_t)i * nrhs + c] = 0.0;
        continue;
      }
      double sum = gc[i];
      for (int q = i + 1; q < k; ++q) sum -= Hc[i + (size_t)(m + 1) * q] * y[(size_t)q * nrhs + c];
      const double d = Hc[i + (size_t)(m + 1) * i];
      y[(size_t)i * nrhs + c] = d == 0.0 ? 0.0 : sum / d;
    }
    sc[2] += k;
  }
}

// dst[:, c] = src[:, c] in the other precision (round to nearest), n rows, nc columns
template <typename S, typename D>
__global__ void convert_kernel(long long n, int nc, const S* src, int lds, D* dst, int ldd) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nc;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % n;
    const int c = (int)(e / n);
    dst[r + (size_t)ldd * c] = (D)src[r + (size_t)lds * c];
  }
}

// Column-major FP64 vectors <-> chunk-interleaved FP32 (chunk k = right-hand sides 16k..16k+15,
// 16 consecutive values per grid node), through a 64-node x 16-column tile in shared memory so
// that both sides are read and written in whole sectors.  grid = (ceil(n / 64), chunks).
constexpr int CT = 64;
__global__ void __launch_bounds__(256) to_chunked_kernel(int n, int nrhs, const double* B, int ldb,
                                                         const double* bscale, float* xf) {
  pdl_enter();
  __shared__ float tile[16][CT + 1];
  __shared__ float bs[16];                    // the column scales, converted once per block
  const int u0 = blockIdx.x * CT, k = blockIdx.y;
  if (bscale && threadIdx.x < 16) bs[threadIdx.x] = 16 * k + threadIdx.x < nrhs ? (float)bscale[16 * k + threadIdx.x] : 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * CT; i += 256) {
    const int cc = i / CT, uu = i % CT, c = 16 * k + cc;
    float v = (u0 + uu < n && c < nrhs) ? (float)B[(size_t)(u0 + uu) + (size_t)ldb * c] : 0.f;
    if (bscale && c < nrhs) v *= bs[cc];
    tile[cc][uu] = v;
  }
  __syncthreads();
  float* dst = xf + ((size_t)k * n + u0) * 16;
  for (int i = threadIdx.x; i < 16 * CT; i += 256) {
    const int uu = i / 16, cc = i % 16;
    if (u0 + uu < n) dst[i] = tile[cc][uu];
  }
}

__global__ void __launch_bounds__(256) from_chunked_kernel(int n, int nrhs, const float* xf, double* X, int ldx) {
  pdl_enter();
  __shared__ float tile[16][CT + 1];
  const int u0 = blockIdx.x * CT, k = blockIdx.y;
  const float* src = xf + ((size_t)k * n + u0) * 16;
  for (int i = threadIdx.x; i < 16 * CT; i += 256) {
    const int uu = i / 16, cc = i % 16;
    if (u0 + uu < n) tile[cc][uu] = src[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * CT; i += 256) {
    const int cc = i / CT, uu = i % CT, c = 16 * k + cc;
    if (u0 + uu < n && c < nrhs) X[(size_t)(u0 + uu) + (size_t)ldx * c] = (double)tile[cc][uu];
  }
}

// X[:, c] = s_c B[:, c]
__global__ void scaled_copy_kernel(int n, int nrhs, const double* B, int ldb, const double* sc, double* X, int ldx) {
  pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * nrhs;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    X[r + (size_t)ldx * c] = B[r + (size_t)ldb * c] * sc[c];
  }
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)std::max(1ll, b);
}

}  // namespace

// ============================================================ public entry points
extern "C" {

void spalu_default_opts(spalu_opts* o) {
  if (!o) return;
  o->eps_id = 1e-8;
  o->precision = 0;
  o->symmetric = 0;
  o->p_oversample = 5;
  o->near_radius = 2;
  o->h0 = 16;
  o->seed = 0;
  o->gmres_m = 30;
  o->gmres_maxit = 200;
  o->gmres_tol = 1e-10;
  o->spars_ctas = 4;
  o->schur_tc = 1;
  o->sketch_tc = 0;
  o->leaf_bwd = -1;
}

const char* spalu_status_string(spalu_status s) {
  switch (s) {
    case SPALU_OK: return "ok";
    case SPALU_ERR_ARG: return "invalid argument";
    case SPALU_ERR_ALLOC: return "allocation failed";
    case SPALU_ERR_SINGULAR: return "zero pivot in an LU";
    case SPALU_ERR_NOCONV: return "refinement did not converge";
    case SPALU_ERR_TIMEOUT: return "bounded device wait expired";
    case SPALU_ERR_CUDA: return "CUDA runtime error";
    case SPALU_ERR_UNSUPPORTED: return "unsupported request";
    case SPALU_ERR_NONFINITE: return "non-finite value in the factor";
    case SPALU_ERR_STATE: return "handle in the wrong state";
  }
  return "unknown status";
}

spalu_status spalu_nd_build_grid(int nx, int ny, int leaf_pitch, spalu_stream_t stream,
                                 spalu_nd_t* out) {
  if (!out) return SPALU_ERR_ARG;
  *out = nullptr;
  if (leaf_pitch != kPitch) return SPALU_ERR_UNSUPPORTED;
  if (!side_ok(nx) || !side_ok(ny)) return SPALU_ERR_ARG;
  if ((long long)nx * ny > (1ll << 30)) return SPALU_ERR_UNSUPPORTED;
  auto* nd = new spalu_nd_s();
  nd->nx = nx;
  nd->ny = ny;
  nd->stream = (cudaStream_t)stream;
  Geo g{1, 1, nx, ny};
  nd->depth.push_back(g);
  nd->vcut.push_back(0);
  while (!(g.w == LEAF && g.h == LEAF)) {
    Geo c = g;
    if (g.w < g.h) { c.h = (g.h - 1) / 2; c.by = 2 * g.by; nd->vcut.push_back(0); }
    else { c.w = (g.w - 1) / 2; c.bx = 2 * g.bx; nd->vcut.push_back(1); }
    nd->depth.push_back(c);
    g = c;
  }
  nd->L = (int)nd->depth.size() - 1;
  size_t n = (size_t)nx * ny;
  if (cudaMalloc(&nd->d_perm, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&nd->d_iperm, n * sizeof(int)) != cudaSuccess) {
    cudaFree(nd->d_perm);
    delete nd;
    return SPALU_ERR_ALLOC;
  }
  launch_nd_perm(nx, ny, nd->L, nd->vcut.data(), nd->d_perm, nd->d_iperm, nd->stream);
  if (cudaGetLastError() != cudaSuccess) {
    spalu_nd_destroy(nd);
    return SPALU_ERR_CUDA;
  }
  *out = nd;
  return SPALU_OK;
}

spalu_status spalu_nd_export(spalu_nd_t nd, int* perm, int* iperm, int* levels, int cap) {
  if (!nd) return SPALU_ERR_ARG;
  size_t n = (size_t)nd->nx * nd->ny;
  if (perm) CUDA_TRY(cudaMemcpyAsync(perm, nd->d_perm, n * sizeof(int), cudaMemcpyDeviceToHost, nd->stream));
  if (iperm) CUDA_TRY(cudaMemcpyAsync(iperm, nd->d_iperm, n * sizeof(int), cudaMemcpyDeviceToHost, nd->stream));
  CUDA_TRY(cudaStreamSynchronize(nd->stream));
  if (levels) {
    if (cap < 8 * (nd->L + 1)) return SPALU_ERR_ARG;
    levels[0] = nd->L;
    for (int l = 1; l <= nd->L; ++l) {
      const Geo& g = nd->depth[l];
      int* v = levels + 8 * l;
      v[0] = g.bx; v[1] = g.by; v[2] = g.w; v[3] = g.h; v[4] = nd->vcut[l];
      v[5] = g.nseg(); v[6] = g.ncorner(); v[7] = nd->depth[l - 1].nbox();
    }
  }
  return SPALU_OK;
}

spalu_status spalu_nd_export_segments(spalu_nd_t nd, int* nodes, int cap) {
  if (!nd || !nodes) return SPALU_ERR_ARG;
  if (nd->L == 0) return SPALU_OK;
  const Geo& g = nd->depth[nd->L];
  if (cap < LEAF * g.nseg()) return SPALU_ERR_ARG;
  for (int s = 0; s < g.nseg(); ++s)
    for (int t = 0; t < LEAF; ++t) nodes[(size_t)s * LEAF + t] = g.seg_node(s, t, nd->nx);
  return SPALU_OK;
}

void spalu_nd_destroy(spalu_nd_t nd) {
  if (!nd) return;
  cudaFree(nd->d_perm);
  cudaFree(nd->d_iperm);
  delete nd;
}

spalu_status spalu_factor_create(spalu_nd_t nd, const spalu_opts* o, spalu_factor_t* out) {
  if (!nd || !o || !out) return SPALU_ERR_ARG;
  *out = nullptr;
  if (!(o->eps_id >= 0.0) || o->p_oversample < 0 || o->h0 < 1 || o->near_radius < -1 ||
      o->gmres_m < 1 || o->gmres_maxit < 0 || o->spars_ctas < 0 || o->spars_ctas > 32 ||
      (o->schur_tc != 0 && o->schur_tc != 1) || (o->sketch_tc != 0 && o->sketch_tc != 1) ||
      o->leaf_bwd < -1 || o->leaf_bwd > 1)
    return SPALU_ERR_ARG;
  if (o->precision != 0 && o->precision != 1) return SPALU_ERR_ARG;
  if (leaf_init_tables() != cudaSuccess) return SPALU_ERR_CUDA;
  auto* f = new spalu_factor_s();
  f->nd = nd;
  f->o = *o;
  f->N = nd->nx * nd->ny;
  f->nnz_cap = 5 * f->N;
  const int L = nd->L;
  f->plan.resize(L + 1);
  f->lev.resize(L + 1);
  // leading dimensions of the frontal stores per depth
  std::vector<int> ldF(L + 1, 0);
  for (int dd = 0; dd <= L; ++dd) {
    const Geo& g = nd->depth[dd];
    int sep = 0;
    if (dd < L) sep = nd->vcut[dd + 1] ? g.h : g.w;
    ldF[dd] = g.D() + sep;
  }
  for (int l = 1; l <= L; ++l) {
    LevelPlan& p = f->plan[l];
    p.l = l;
    p.vcut = nd->vcut[l];
    p.g = nd->depth[l];
    p.gp = nd->depth[l - 1];
    p.capS = p.g.cap();
    p.ldF = ldF[l];
    p.ldFp = ldF[l - 1];
    p.sepcap = p.vcut ? p.gp.h : p.gp.w;
    p.Ycap = 2 * 16 + std::max(o->h0, 2 * (p.capS + o->p_oversample));
    const int tb = o->precision == 1 ? 4 : 8;
    // need: the uncut working set with the smallest sketch chunk (below it the kernel keeps
    // its sketch rows in global scratch).  A level that runs one segment per SM (or the uncut
    // candidate of the tuner) gets 160 KB: what a segment does not need for its working set
    // goes to larger sketch chunks and the staged B block
    size_t need = sparsify_smem_need(p.capS, o->symmetric, o->h0, o->p_oversample, tb, 16);
    size_t lim = 160 * 1024;
    size_t mn = sparsify_smem_min(p.capS, o->symmetric, o->h0, o->p_oversample, tb);
    const size_t roomy = std::max(lim, mn);
    const size_t full = std::min(need, roomy);
    // trade worst-case room for resident segments (the phases of one segment are
    // latency-bound): as many per SM as the level has segments per SM, up to spars_ctas;
    // segments that do not fit the budget fall back to global scratch inside the kernel
    auto budget = [&](int ctas) {
      if (ctas <= 1) return roomy;
      const size_t b = sparsify_smem_budget(tb == 4, p.capS, ctas);
      return b >= mn ? std::min(full, b) : full;
    };
    p.spars_smem = full;
    if (o->spars_ctas > 0 && p.g.nseg() > 0) {
      const int nsm = sm_count();
      p.spars_smem = budget((int)std::min<long long>(o->spars_ctas, ((long long)p.g.nseg() + nsm - 1) / nsm));
    }
    size_t least = p.spars_smem;
    for (int c = 0; c < SPARS_NCAND; ++c) {
      p.spars_cand[c] = budget(SPARS_CAND_CTAS[c]);
      least = std::min(least, p.spars_cand[c]);
    }
    p.spars_global = need > least;   // global scratch for every budget the tuner may pick
  }
  // plan the arena (two passes: sizes, then pointers)
  for (int pass = 0; pass < 2; ++pass) {
    Carver cv;
    cv.base = pass ? f->arena : nullptr;
    f->d_err = cv.take<int>(4);
    f->d_lstat = cv.take<int>((size_t)LS_N * (L + 1));
    f->d_flops = cv.take<unsigned long long>((size_t)4 * (L + 1));
    {
      size_t nt = 0;
      for (int l = 1; l <= L; ++l) nt += (size_t)f->plan[l].g.nseg() * 4;
      f->tgt_ints = nt;
      f->d_tgt_all = cv.take<int>(nt > 0 ? nt : 1);
    }
    size_t tgt_off = 0;
    f->d_count = cv.take<int>(1);
    f->d_nstat = cv.take<float4>((size_t)f->N);
    f->rowptr = cv.take<int>(f->N + 1);
    f->colind = cv.take<int>(f->nnz_cap);
    f->val = cv.take<double>(f->nnz_cap);
    f->fval = o->precision == 1 ? cv.take<float>(f->nnz_cap) : nullptr;
    const Geo& gl = nd->depth[L];
    LeafDev& lf = f->leaf;
    lf.nx = nd->nx; lf.ny = nd->ny; lf.L = L; lf.g = gl; lf.ldF = ldF[L];
    const bool f32 = o->precision == 1;
    auto real = [&](size_t n) -> void* { return f32 ? (void*)cv.take<float>(n) : (void*)cv.take<double>(n); };
    lf.fp32 = f32 ? 1 : 0;
    lf.F = real((size_t)gl.nbox() * ldF[L] * ldF[L]);
    lf.lrec = real((size_t)gl.nbox() * NI * 16);
    lf.urec = real((size_t)gl.nbox() * NI * 16);
    lf.uext = real((size_t)gl.nbox() * NI * 16);
    lf.ybuf = real((size_t)gl.nbox() * NI * 64);
    lf.cpl = real((size_t)gl.nbox() * 4 * LEAF);
    const bool useG = f32 && (o->leaf_bwd == 0 || (o->leaf_bwd < 0 && gl.nbox() < LEAF_G_MAX));
    lf.G = useG ? (void*)cv.take<float>((size_t)gl.nbox() * NI * 4 * LEAF) : nullptr;
    lf.band5 = cv.take<double>((size_t)gl.nbox() * NI * 5);
    lf.kumax = cv.take<int>(4);
    lf.kur = cv.take<int>((size_t)gl.nbox());
    std::vector<void*> Fst(L + 1, nullptr);
    Fst[L] = lf.F;
    for (int l = L; l >= 1; --l) {
      const LevelPlan& p = f->plan[l];
      LevelDev& d = f->lev[l];
      const int nseg = p.g.nseg();
      d.l = l; d.nx = nd->nx; d.ny = nd->ny; d.vcut = p.vcut;
      d.g = p.g; d.gp = p.gp;
      d.capS = p.capS; d.ldF = p.ldF; d.ldFp = p.ldFp; d.Ycap = p.Ycap; d.sepcap = p.sepcap;
      d.cnt = cv.take<int>(nseg);
      d.order = cv.take<int>(nseg);
      // levels with at least two segments per SM and segments that can exceed 16 unknowns:
      // the sparsify CTAs take the largest first (the finest level's segments are all alike,
      // and there index order keeps neighbouring segments' reads together)
      d.use_order = (long long)nseg >= 2LL * sm_count() && p.capS > 16 ? 1 : 0;
      d.kk = cv.take<int>(nseg);
      d.hs = cv.take<int>(nseg);
      d.nodes = cv.take<int>((size_t)nseg * p.capS);
      d.perm = cv.take<int>((size_t)nseg * p.capS);
      d.snodes = cv.take<int>((size_t)nseg * p.capS);
      d.piv = cv.take<int>((size_t)nseg * p.capS);
      d.fp32 = f32 ? 1 : 0;
      d.T = real((size_t)nseg * p.capS * p.capS);
      d.Dm = real((size_t)nseg * p.capS * p.capS);
      d.Dinv = real((size_t)nseg * p.capS);
      d.Yg = p.spars_global ? real((size_t)nseg * p.Ycap * p.capS) : nullptr;
      Fst[l - 1] = real((size_t)p.gp.nbox() * p.ldFp * p.ldFp);
      d.Pinv = real((size_t)p.gp.nbox() * p.sepcap);
      d.F = Fst[l];
      d.Fp = Fst[l - 1];
      d.ptab = cv.take<int>((size_t)p.gp.nbox() * p.ldFp * 8);
      d.pcount = cv.take<int>((size_t)p.gp.nbox() * 2);
      d.ppiv = cv.take<int>((size_t)p.gp.nbox() * p.sepcap);
      d.eps = o->eps_id; d.symmetric = o->symmetric; d.p_over = o->p_oversample;
      d.near_radius = o->near_radius; d.h0 = o->h0; d.seed = o->seed;
      d.schur_tc = (o->schur_tc && f32) ? 1 : 0;
      d.sketch_tc = (o->sketch_tc && f32) ? 1 : 0;
      d.L = L;
      d.pred_mode = PRED_OFF; d.pred_margin = 0.35; d.pred = nullptr;
      d.log10eps = o->eps_id > 0.0 ? std::log10(o->eps_id) : -16.0;
      d.feat = cv.take<float>((size_t)nseg * PRED_NFEAT);
      d.tgt = f->d_tgt_all ? f->d_tgt_all + tgt_off : nullptr;
      tgt_off += (size_t)nseg * 4;
    }
    for (int l = L; l >= 1; --l) {
      LevelDev& d = f->lev[l];
      if (l > 1) { d.cnt_up = f->lev[l - 1].cnt; d.nodes_up = f->lev[l - 1].nodes; d.capS_up = f->lev[l - 1].capS; }
      else { d.cnt_up = nullptr; d.nodes_up = nullptr; d.capS_up = 0; }
    }
    if (pass == 0) {
      f->arena_bytes = align_up(cv.off, 256);
      if (cudaMalloc(&f->arena, f->arena_bytes) != cudaSuccess) {
        delete f;
        return SPALU_ERR_ALLOC;
      }
      if (cudaMallocHost(&f->hpin, sizeof(int) * (2 + LS_N * (L + 1))) != cudaSuccess) {
        cudaFree(f->arena);
        delete f;
        return SPALU_ERR_ALLOC;
      }
    }
  }
  f->leaf.rowptr = f->rowptr;
  f->leaf.colind = f->colind;
  f->leaf.val = f->val;
  f->leaf.fval = f->fval;
  f->leaf.err = f->d_err;
  for (int l = 1; l <= L; ++l) {
    f->lev[l].err = f->d_err;
    f->lev[l].lstat = f->d_lstat + LS_N * l;
    f->lev[l].flops = f->d_flops + 4 * l;
    f->lev[l].rowptr = f->rowptr;
    f->lev[l].colind = f->colind;
    f->lev[l].val = f->val;
    f->lev[l].nstat = f->d_nstat;
  }
  f->caps.resize(L + 1);
  *out = f;
  return SPALU_OK;
}

// A factorization in two halves: enqueue() puts every kernel and the readback of the error
// word, the leaf bandwidth and the level counters on the stream; finish() waits for that
// stream and sets the solve capacities.  A batch enqueues all problems before finishing any.
static spalu_status factor_enqueue(spalu_factor_t f, cudaStream_t s) {
  const int L = f->nd->L;
  PhaseTimer& tm = f->timer;
  int t_all = tm.begin("factor", s);
  CUDA_TRY(cudaMemsetAsync(f->d_err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(f->leaf.kumax, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(f->d_lstat, 0, sizeof(int) * LS_N * (L + 1), s));
  CUDA_TRY(cudaMemsetAsync(f->d_flops, 0, sizeof(unsigned long long) * 4 * (L + 1), s));
  if (f->pred_mode == PRED_RECORD && f->tgt_ints)
    CUDA_TRY(cudaMemsetAsync(f->d_tgt_all, 0, sizeof(int) * f->tgt_ints, s));
  if (L >= 1) launch_level_init_L(f->lev[L], s);
  if (f->fval && f->nnz > 0) {
    note_launch();
    convert_kernel<double, float><<<grid_for(f->nnz), 256, 0, s>>>(f->nnz, 1, f->val, 0, f->fval, 0);
  }
  if (f->pred_mode != PRED_OFF) launch_node_stats(f->rowptr, f->colind, f->val, f->fval, f->N, f->d_nstat, s);
  int t = tm.begin("leaf_factor", s);
  launch_leaf_factor(f->leaf, s);
  tm.end(t, s);
  for (int l = L; l >= 1; --l) {
    t = tm.begin("sparsify_l" + std::to_string(l), s);
    launch_sparsify(f->lev[l], f->plan[l], s);
    tm.end(t, s);
    t = tm.begin("merge_l" + std::to_string(l), s);
    launch_merge(f->lev[l], f->plan[l], s);
    tm.end(t, s);
  }
  tm.end(t_all, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(f->hpin, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(f->hpin + 1, f->leaf.kumax, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(f->hpin + 2, f->d_lstat, sizeof(int) * LS_N * (L + 1), cudaMemcpyDeviceToHost, s));
  return SPALU_OK;
}

static spalu_status factor_finish(spalu_factor_t f, cudaStream_t s) {
  const int L = f->nd->L;
  CUDA_TRY(cudaStreamSynchronize(s));
  const int h = f->hpin[0];
  spalu_status st = SPALU_OK;
  if (h & ERR_SINGULAR) st = SPALU_ERR_SINGULAR;
  else if (h & ERR_NONFINITE) st = SPALU_ERR_NONFINITE;
  else if (h & ERR_TIMEOUT) st = SPALU_ERR_TIMEOUT;
  else if (h & ERR_CAPACITY) st = SPALU_ERR_UNSUPPORTED;
  f->kumax = f->hpin[1];
  f->lstat.assign(f->hpin + 2, f->hpin + 2 + LS_N * (L + 1));
  // the solve kernels hold a segment's (or separator's) right-hand-side block in shared memory
  for (int l = 1; l <= L && st == SPALU_OK; ++l) {
    if (!level_solve_caps(f->lev[l], f->lstat.data() + LS_N * l, &f->caps[l])) st = SPALU_ERR_UNSUPPORTED;
    if ((int)f->tuned_nt.size() == 4 * (L + 1) && f->tuned_nt[4 * l] > 0) {
      f->caps[l].seg_nt = f->tuned_nt[4 * l];
      f->caps[l].sep_nt = f->tuned_nt[4 * l + 1];
      f->caps[l].seg_split = f->tuned_nt[4 * l + 2];
      f->caps[l].sep_split = f->tuned_nt[4 * l + 3];
    }
  }
  f->factored = (st == SPALU_OK);
  f->last_stream = s;
  return st;
}

static spalu_status factor_run(spalu_factor_t f, cudaStream_t s) {
  spalu_status st = factor_enqueue(f, s);
  if (st != SPALU_OK) return st;
  return factor_finish(f, s);
}

spalu_status spalu_factor_numeric(spalu_factor_t f, const int* rowptr, const int* colind,
                                  const double* val, int nnz, spalu_stream_t stream) {
  if (!f || !rowptr || !colind || !val || nnz < 0 || nnz > f->nnz_cap) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  f->nnz = nnz;
  CUDA_TRY(cudaMemcpyAsync(f->rowptr, rowptr, (f->N + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->colind, colind, (size_t)nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->val, val, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return factor_run(f, s);
}

spalu_status spalu_factor_numeric_batch(int n, const spalu_factor_t* f, const int* const* rowptr,
                                        const int* const* colind, const double* const* val, const int* nnz,
                                        spalu_stream_t const* streams) {
  if (n < 0 || (n > 0 && (!f || !rowptr || !colind || !val || !nnz || !streams))) return SPALU_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!f[i] || !rowptr[i] || !colind[i] || !val[i] || nnz[i] < 0 || nnz[i] > f[i]->nnz_cap) return SPALU_ERR_ARG;
  spalu_status first = SPALU_OK;
  std::vector<char> queued(n, 0);
  for (int i = 0; i < n; ++i) {          // every problem's copies and kernels, on its stream
    spalu_factor_t g = f[i];
    cudaStream_t s = (cudaStream_t)streams[i];
    g->nnz = nnz[i];
    spalu_status st = SPALU_OK;
    if (cudaMemcpyAsync(g->rowptr, rowptr[i], (g->N + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(g->colind, colind[i], (size_t)nnz[i] * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(g->val, val[i], (size_t)nnz[i] * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      st = SPALU_ERR_CUDA;
    if (st == SPALU_OK) st = factor_enqueue(g, s);
    if (st == SPALU_OK) queued[i] = 1;
    else { g->factored = false; if (first == SPALU_OK) first = st; }
  }
  for (int i = 0; i < n; ++i) {          // then wait for each and set its solve capacities
    if (!queued[i]) continue;
    const spalu_status st = factor_finish(f[i], (cudaStream_t)streams[i]);
    if (st != SPALU_OK && first == SPALU_OK) first = st;
  }
  return first;
}

static void step_graph_free(spalu_factor_t f);

spalu_status spalu_tune_solve(spalu_factor_t f, int nrhs, spalu_stream_t stream) {
  if (!f || nrhs < 1 || nrhs > 16) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  step_graph_free(f);        // a captured step holds the old CTA widths
  cudaStream_t s = (cudaStream_t)stream;
  const int L = f->nd->L, N = f->N;
  // the solve's working vector (zeros: the timing does not depend on the values)
  void* W = nullptr;
  VecLayout lay{1, N, 16LL * N};
  double* tmp = nullptr;
  if (f->leaf.fp32) {
    if (f->xf_cols < 16) {
      cudaFree(f->xf);
      f->xf = nullptr;
      f->xf_cols = 0;
      if (cudaMalloc(&f->xf, sizeof(float) * (size_t)N * 16) != cudaSuccess) return SPALU_ERR_ALLOC;
      f->xf_cols = 16;
    }
    CUDA_TRY(cudaMemsetAsync(f->xf, 0, sizeof(float) * (size_t)N * 16, s));
    W = f->xf;
    lay = VecLayout{16, 1, 16LL * N};
  } else {
    if (cudaMalloc(&tmp, sizeof(double) * (size_t)N * nrhs) != cudaSuccess) return SPALU_ERR_ALLOC;
    CUDA_TRY(cudaMemsetAsync(tmp, 0, sizeof(double) * (size_t)N * nrhs, s));
    W = tmp;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f->tuned_nt.assign(4 * (L + 1), 0);
  // per level: the CTA widths (64 or 256) and the right-hand-side groups (1, 2, 4, 8: more
  // CTAs per segment or separator on levels with few of them) of the two solve kernels, the
  // fastest forward + backward pass; the first repetition of each candidate warms up
  auto time_cfg = [&](int l, const SolveCaps& sc, float* out) -> bool {
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      launch_level_solve_fwd(f->lev[l], sc, W, nrhs, lay, s);
      launch_level_solve_bwd(f->lev[l], sc, W, nrhs, lay, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = ms < tmin ? ms : tmin;
    }
    *out = tmin;
    return true;
  };
  const int nts[2] = {64, 256}, splits[4] = {1, 2, 4, 8};
  spalu_status st = SPALU_OK;
  for (int l = 1; l <= L && st == SPALU_OK; ++l) {
    SolveCaps best = f->caps[l];
    float tbest = 1e30f;
    for (int a = 0; a < 2 && st == SPALU_OK; ++a)
      for (int b = 0; b < 2 && st == SPALU_OK; ++b)
        for (int g = 0; g < 4 && st == SPALU_OK; ++g)
          for (int h = 0; h < 4 && st == SPALU_OK; ++h) {
            if (splits[g] > nrhs || splits[h] > nrhs) continue;
            SolveCaps sc = f->caps[l];
            sc.seg_nt = nts[a];
            sc.sep_nt = nts[b];
            sc.seg_split = splits[g];
            sc.sep_split = splits[h];
            float t = 0.f;
            if (!time_cfg(l, sc, &t)) { st = SPALU_ERR_CUDA; break; }
            if (t < tbest) { tbest = t; best = sc; }
          }
    f->caps[l] = best;
    f->tuned_nt[4 * l] = best.seg_nt;
    f->tuned_nt[4 * l + 1] = best.sep_nt;
    f->tuned_nt[4 * l + 2] = best.seg_split;
    f->tuned_nt[4 * l + 3] = best.sep_split;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tmp);
  CUDA_TRY(cudaGetLastError());
  return st;
}

spalu_status spalu_tune_factor(spalu_factor_t f, spalu_stream_t stream) {
  if (!f) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  step_graph_free(f);        // a captured step holds the old shared-memory budgets
  cudaStream_t s = (cudaStream_t)stream;
  const int L = f->nd->L;
  PhaseTimer& tm = f->timer;
  tm.collect();
  const bool was_on = tm.on;
  const auto keep_ms = tm.ms;
  const auto keep_count = tm.count;
  std::vector<size_t> best_smem(L + 1, 0);
  std::vector<double> best_ms(L + 1, 1e30);
  for (int l = 1; l <= L; ++l) best_smem[l] = f->plan[l].spars_smem;
  spalu_status st = SPALU_OK;
  for (int c = 0; c < SPARS_NCAND && st == SPALU_OK; ++c) {
    bool fresh = false;                  // skip budgets that repeat an earlier one everywhere
    for (int l = 1; l <= L && !fresh; ++l) {
      bool seen = false;
      for (int c2 = 0; c2 < c; ++c2) seen = seen || f->plan[l].spars_cand[c2] == f->plan[l].spars_cand[c];
      fresh = !seen;
    }
    if (!fresh) continue;
    for (int l = 1; l <= L; ++l) f->plan[l].spars_smem = f->plan[l].spars_cand[c];
    std::vector<double> tmin(L + 1, 1e30);
    for (int rep = 0; rep < 3 && st == SPALU_OK; ++rep) {   // the first repetition warms up
      tm.on = true;
      tm.ms.clear();
      tm.count.clear();
      st = factor_run(f, s);
      tm.collect();
      if (st != SPALU_OK || rep == 0) continue;
      for (int l = 1; l <= L; ++l) {
        auto it = tm.ms.find("sparsify_l" + std::to_string(l));
        if (it != tm.ms.end()) tmin[l] = std::min(tmin[l], it->second);
      }
    }
    for (int l = 1; l <= L; ++l)
      if (tmin[l] < best_ms[l]) { best_ms[l] = tmin[l]; best_smem[l] = f->plan[l].spars_cand[c]; }
  }
  for (int l = 1; l <= L; ++l) f->plan[l].spars_smem = best_smem[l];
  // predict mode: keep the network only on the levels where it measured faster than the
  // adaptive schedule (its one-pass sketches against the probe, network and error-test
  // overhead and the fallbacks)
  if (st == SPALU_OK && f->pred_mode == PRED_PREDICT) {
    std::vector<double> lt[2];
    for (int on = 0; on < 2 && st == SPALU_OK; ++on) {
      for (int l = 1; l <= L; ++l) f->lev[l].pred_mode = on ? PRED_PREDICT : PRED_OFF;
      lt[on].assign(L + 1, 1e30);
      for (int rep = 0; rep < 3 && st == SPALU_OK; ++rep) {
        tm.on = true;
        tm.ms.clear();
        tm.count.clear();
        st = factor_run(f, s);
        tm.collect();
        if (st != SPALU_OK || rep == 0) continue;
        for (int l = 1; l <= L; ++l) {
          auto it = tm.ms.find("sparsify_l" + std::to_string(l));
          if (it != tm.ms.end()) lt[on][l] = std::min(lt[on][l], it->second);
        }
      }
    }
    for (int l = 1; l <= L; ++l)
      f->lev[l].pred_mode = (st == SPALU_OK && lt[1][l] < lt[0][l]) ? PRED_PREDICT : PRED_OFF;
  }
  tm.on = false;
  if (st == SPALU_OK) st = factor_run(f, s);
  tm.collect();
  tm.on = was_on;
  tm.ms = keep_ms;
  tm.count = keep_count;
  return st;
}

spalu_status spalu_solve_batch(int n, const spalu_factor_t* f, const double* const* B, double* const* X,
                               const int* nrhs, const int* ld, spalu_stream_t const* streams) {
  if (n < 0 || (n > 0 && (!f || !B || !X || !nrhs || !ld || !streams))) return SPALU_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    const spalu_status st = spalu_solve(f[i], B[i], X[i], nrhs[i], ld[i], streams[i]);
    if (st != SPALU_OK) return st;
  }
  return SPALU_OK;
}

spalu_status spalu_factor_numeric_host(spalu_factor_t f, const int* rowptr, const int* colind,
                                       const double* val, int nnz, spalu_stream_t stream) {
  if (!f || !rowptr || !colind || !val || nnz < 0 || nnz > f->nnz_cap) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  f->nnz = nnz;
  CUDA_TRY(cudaMemcpyAsync(f->rowptr, rowptr, (f->N + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->colind, colind, (size_t)nnz * sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->val, val, (size_t)nnz * sizeof(double), cudaMemcpyHostToDevice, s));
  return factor_run(f, s);
}

// X = spaLU^{-1} (B diag(bscale)) (bscale: device, one factor per column, or null)
static spalu_status solve_impl(spalu_factor_t f, const double* B, const double* bscale, double* X, int nrhs,
                               int ld, spalu_stream_t stream);

spalu_status spalu_solve(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                         spalu_stream_t stream) {
  return solve_impl(f, B, nullptr, X, nrhs, ld, stream);
}

static spalu_status solve_impl(spalu_factor_t f, const double* B, const double* bscale, double* X, int nrhs,
                               int ld, spalu_stream_t stream) {
  if (!f || !B || !X || nrhs < 0 || ld < f->N) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  if (nrhs == 0) return SPALU_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int L = f->nd->L;
  const int N = f->N;
  PhaseTimer& tm = f->timer;
  int t_all = tm.begin("solve", s);
  // the mixed path solves on an FP32 copy, 16 right-hand sides interleaved per grid node:
  // every kernel of the solve reads and writes the precision of the factors, a node's values
  // for one chunk share sectors, and B and X are converted once each
  void* W = X;
  VecLayout lay{1, ld, 16LL * ld};
  const int nch = (nrhs + 15) / 16;
  const dim3 cgrid((N + CT - 1) / CT, nch);
  if (f->leaf.fp32) {
    if (f->xf_cols < 16 * nch) {
      cudaFree(f->xf);
      f->xf = nullptr;
      f->xf_cols = 0;
      if (cudaMalloc(&f->xf, sizeof(float) * (size_t)N * 16 * nch) != cudaSuccess) return SPALU_ERR_ALLOC;
      f->xf_cols = 16 * nch;
    }
    note_launch();
    launch_pdl(to_chunked_kernel, cgrid, dim3(256), 0, s, N, nrhs, B, ld, bscale, f->xf);
    W = f->xf;
    lay = VecLayout{16, 1, 16LL * N};
  } else if (bscale) {
    note_launch();
    launch_pdl(scaled_copy_kernel, dim3(grid_for((long long)N * nrhs)), dim3(256), 0, s, N, nrhs, B, ld, bscale, X, ld);
  } else if (X != B) {
    CUDA_TRY(cudaMemcpy2DAsync(X, (size_t)ld * sizeof(double), B, (size_t)ld * sizeof(double),
                               (size_t)N * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, s));
  }
  int t = tm.begin("leaf_solve_fwd", s);
  launch_leaf_solve(f->leaf, W, nrhs, lay, 0, f->kumax, s);
  tm.end(t, s);
  t = tm.begin("sep_update", s);
  if (L >= 1) launch_sep_update_fwd(f->leaf, W, nrhs, lay, s);
  tm.end(t, s);
  t = tm.begin("level_solve", s);
  for (int l = L; l >= 1; --l) launch_level_solve_fwd(f->lev[l], f->caps[l], W, nrhs, lay, s);
  for (int l = 1; l <= L; ++l) launch_level_solve_bwd(f->lev[l], f->caps[l], W, nrhs, lay, s);
  tm.end(t, s);
  t = tm.begin("leaf_solve_bwd", s);
  launch_leaf_solve(f->leaf, W, nrhs, lay, 1, f->kumax, s);
  tm.end(t, s);
  if (f->leaf.fp32) {
    note_launch();
    launch_pdl(from_chunked_kernel, cgrid, dim3(256), 0, s, N, nrhs, (const float*)f->xf, X, ld);
  }
  tm.end(t_all, s);
  CUDA_TRY(cudaGetLastError());
  return SPALU_OK;
}

static void gmres_free(GmresWork& w) {
  cudaFree(w.V); cudaFree(w.Z); cudaFree(w.cnt); cudaFree(w.part); cudaFree(w.hcol); cudaFree(w.vs); cudaFree(w.vec);
  cudaFree(w.H); cudaFree(w.cs); cudaFree(w.sn); cudaFree(w.g); cudaFree(w.y); cudaFree(w.bn); cudaFree(w.beta);
  cudaFree(w.st); cudaFree(w.flag); cudaFreeHost(w.hflag);
  w = GmresWork();
}

static spalu_status gmres_alloc(spalu_factor_t f, int nrhs) {
  GmresWork& w = f->gw;
  const int m = f->o.gmres_m;
  if (w.nrhs >= nrhs && w.m == m) return SPALU_OK;
  gmres_free(w);
  size_t N = f->N;
  if (cudaMalloc(&w.V, sizeof(double) * (m + 1) * N * nrhs) != cudaSuccess ||
      cudaMalloc(&w.Z, sizeof(double) * (size_t)m * N * nrhs) != cudaSuccess ||
      cudaMalloc(&w.cnt, sizeof(unsigned) * ((nrhs + RC - 1) / RC)) != cudaSuccess ||
      cudaMemset(w.cnt, 0, sizeof(unsigned) * ((nrhs + RC - 1) / RC)) != cudaSuccess ||
      cudaMalloc(&w.part, sizeof(double) * VNB * nrhs) != cudaSuccess ||
      cudaMalloc(&w.hcol, sizeof(double) * (m + 2) * nrhs) != cudaSuccess ||
      cudaMalloc(&w.vs, sizeof(double) * (m + 2) * nrhs) != cudaSuccess ||
      cudaMalloc(&w.vec, sizeof(double) * 4 * nrhs) != cudaSuccess ||
      cudaMalloc(&w.H, sizeof(double) * (size_t)nrhs * (m + 1) * m) != cudaSuccess ||
      cudaMalloc(&w.cs, sizeof(double) * (size_t)nrhs * m) != cudaSuccess ||
      cudaMalloc(&w.sn, sizeof(double) * (size_t)nrhs * m) != cudaSuccess ||
      cudaMalloc(&w.g, sizeof(double) * (size_t)nrhs * (m + 1)) != cudaSuccess ||
      cudaMalloc(&w.y, sizeof(double) * (size_t)nrhs * m) != cudaSuccess ||
      cudaMalloc(&w.bn, sizeof(double) * nrhs) != cudaSuccess ||
      cudaMalloc(&w.beta, sizeof(double) * nrhs) != cudaSuccess ||
      cudaMalloc(&w.st, sizeof(int) * 4 * nrhs) != cudaSuccess ||
      cudaMalloc(&w.flag, sizeof(int) * 4) != cudaSuccess ||
      cudaMallocHost(&w.hflag, sizeof(int) * 4) != cudaSuccess) {
    gmres_free(w);
    return SPALU_ERR_ALLOC;
  }
  w.nrhs = nrhs;
  w.m = m;
  return SPALU_OK;
}

// about four blocks per SM in all: few blocks keep the per-block column sums (FP64 adds, slow
// on this part) small next to the streamed work
static dim3 vec_grid(int n, int nrhs) {
  static const int nsm = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  const int nch = (nrhs + RC - 1) / RC;
  int nb = 4 * nsm / nch;
  const int need = (n + VB - 1) / VB;
  nb = nb < need ? nb : need;
  nb = nb < VNB ? nb : VNB;
  return dim3(nb > 0 ? nb : 1, nch);
}

// w -= h ps p (p null: w unchanged), out[c] = qs <w_c, q_c> (q null: ||w_c||, sq; inv_out = 1 / out)
static void vec_mgs(spalu_factor_t f, int nrhs, const double* h, const double* p, int ldp, const double* ps,
                    double* w, int ldw, const double* q, int ldq, const double* qs, double* out, int sq,
                    double* inv_out, cudaStream_t s) {
  note_launch();
  launch_pdl(mgs_kernel, vec_grid(f->N, nrhs), dim3(VB), 0, s, f->N, nrhs, h, p, ldp, ps, w, ldw, q, ldq, qs,
             f->gw.part, f->gw.cnt, out, sq, inv_out);
}

// y = b - A x (b null: A x); out set: out[c] = ds_c <y_c, d_c> (d null: ||y_c||, sq)
static void vec_spmv(spalu_factor_t f, int nrhs, const double* x, int ldx, const double* b, int ldb,
                     double* y, int ldy, const double* d, int ldd, const double* ds, double* out, int sq,
                     cudaStream_t s) {
  note_launch();
  launch_pdl(spmv_kernel, vec_grid(f->N, nrhs), dim3(VB), 0, s, f->N, nrhs, f->rowptr, f->colind, f->val, x,
             ldx, b, ldb, y, ldy, d, ldd, ds, out ? f->gw.part : nullptr, f->gw.cnt, out, sq);
}

// dl (optional): after every update of X, X is also copied to the host array dl->h on the
// stream dl->s, so the copy of the final X overlaps the last residual; dl->n counts the copies
struct HostDownload {
  double* h;
  int ldh;
  cudaStream_t s;
  cudaEvent_t ev;
  int n;
};
static spalu_status refine_impl(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                                int* iters, double* relres, spalu_stream_t stream, HostDownload* dl = nullptr);

spalu_status spalu_refine(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                          int* iters, double* relres, spalu_stream_t stream) {
  if (!f) return SPALU_ERR_ARG;
  int t = f->timer.begin("refine", (cudaStream_t)stream);
  spalu_status st = refine_impl(f, B, X, nrhs, ld, iters, relres, stream);
  f->timer.end(t, (cudaStream_t)stream);
  return st;
}

static spalu_status refine_impl(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                                int* iters, double* relres, spalu_stream_t stream, HostDownload* dl) {
  if (!f || !B || !X || nrhs < 0 || ld < f->N) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  if (nrhs == 0) return SPALU_OK;
  cudaStream_t s = (cudaStream_t)stream;
  spalu_status st = gmres_alloc(f, nrhs);
  if (st != SPALU_OK) return st;
  GmresWork& w = f->gw;
  const int N = f->N, m = f->o.gmres_m;
  const double tol = f->o.gmres_tol;
  const int maxit = f->o.gmres_maxit;
  const size_t ldv = (size_t)N;
  auto Vj = [&](int j) { return w.V + (size_t)j * ldv * nrhs; };
  auto Zj = [&](int j) { return w.Z + (size_t)j * ldv * nrhs; };
  vec_mgs(f, nrhs, nullptr, nullptr, 0, nullptr, const_cast<double*>(B), ld, nullptr, 0, nullptr, w.bn, 1,
          nullptr, s);
  bool first = true;
  // the residual goes straight into V_0 (stored unnormalized, scale 1 / beta); then the cycle
  // set-up on the device, and one read of "some column still active"
  auto residual = [&]() -> spalu_status {
    vec_spmv(f, nrhs, X, ld, B, ld, Vj(0), (int)ldv, nullptr, 0, nullptr, w.beta, 1, s);
    note_launch();
    gmres_begin_kernel<<<1, GB, 0, s>>>(nrhs, m, tol, w.bn, w.beta, w.vs, w.g, w.st, first ? 1 : 0, w.flag,
                                        cudaGraphConditionalHandle{}, 0);
    first = false;
    CUDA_TRY(cudaMemcpyAsync(w.hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SPALU_OK;
  };
  if ((st = residual()) != SPALU_OK) return st;
  int it = 0;
  int cycles = 0, first_cycle_steps = 0;
  while (it < maxit && w.hflag[0]) {
    // the first check of the cycle comes after one step fewer than the last call needed (it
    // cannot have converged before); later checks after every step
    int batch = cycles == 0 ? std::max(1, f->gmres_hint - 1) : 1;
    int jl = -1, since = 0;
    for (int j = 0; j < m && it < maxit; ++j) {
      // Z_j = M^{-1} V_j (kept), V_{j+1} = A Z_j
      const double* sj = w.vs + (size_t)j * nrhs;
      if ((st = solve_impl(f, Vj(j), sj, Zj(j), nrhs, (int)ldv, stream)) != SPALU_OK) return st;
      // modified Gram-Schmidt on the unnormalized basis (vector i = vs_i x V_i), each subtraction
      // fused with the next inner product: h_0 = <A Z_j, V_0> in the product's pass, then
      // w -= h_{i-1} V_{i-1}, h_i = <w, V_i>; the last pass gives ||w|| and vs_{j+1} = 1 / ||w||
      vec_spmv(f, nrhs, Zj(j), (int)ldv, nullptr, 0, Vj(j + 1), (int)ldv, Vj(0), (int)ldv, w.vs, w.hcol, 0, s);
      for (int i = 1; i <= j + 1; ++i)
        vec_mgs(f, nrhs, w.hcol + (size_t)(i - 1) * nrhs, Vj(i - 1), (int)ldv, w.vs + (size_t)(i - 1) * nrhs,
                Vj(j + 1), (int)ldv, i <= j ? Vj(i) : nullptr, (int)ldv, w.vs + (size_t)i * nrhs,
                w.hcol + (size_t)i * nrhs, i > j, i > j ? w.vs + (size_t)(j + 1) * nrhs : nullptr, s);
      note_launch();
      launch_pdl(gmres_givens_kernel, dim3(1), dim3(GB), 0, s, nrhs, m, j, tol, (const double*)w.hcol,
                 (const double*)w.bn, w.H, w.cs, w.sn, w.g, w.vs, w.st, w.flag, cudaGraphConditionalHandle{}, 0);
      ++it;
      jl = j;
      if (++since >= batch || it >= maxit || j == m - 1) {
        CUDA_TRY(cudaMemcpyAsync(w.hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        since = 0;
        batch = 1;
        if (!w.hflag[0]) break;
      }
    }
    if (cycles == 0) first_cycle_steps = jl + 1;
    ++cycles;
    // y from the triangular system, X += M^{-1} V y = sum_i y_i Z_i
    const int kdim = jl + 1;
    note_launch();
    launch_pdl(gmres_ysolve_kernel, dim3(1), dim3(GB), 0, s, nrhs, m, kdim, (const double*)w.H,
               (const double*)w.g, w.y, w.st);
    note_launch();
    launch_pdl(combine_kernel, vec_grid(N, nrhs), dim3(VB), 0, s, N, nrhs, kdim, (const double*)w.y,
               (const double*)w.Z, ldv, X, ld, (const int*)w.st);
    if (dl) {        // X changes only here: its copy runs while the residual is checked
      CUDA_TRY(cudaEventRecord(dl->ev, s));
      CUDA_TRY(cudaStreamWaitEvent(dl->s, dl->ev, 0));
      CUDA_TRY(cudaMemcpy2DAsync(dl->h, (size_t)dl->ldh * sizeof(double), X, (size_t)ld * sizeof(double),
                                 (size_t)N * sizeof(double), nrhs, cudaMemcpyDeviceToHost, dl->s));
      ++dl->n;
    }
    if ((st = residual()) != SPALU_OK) return st;
  }
  if (cycles == 1) f->gmres_hint = first_cycle_steps;
  std::vector<double> bn(nrhs), beta(nrhs);
  std::vector<int> stc(4 * (size_t)nrhs);
  CUDA_TRY(cudaMemcpyAsync(bn.data(), w.bn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(beta.data(), w.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(stc.data(), w.st, sizeof(int) * 4 * nrhs, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  bool conv = true;
  int its = 0;
  for (int c = 0; c < nrhs; ++c) {
    if (relres) relres[c] = bn[c] == 0.0 ? 0.0 : beta[c] / bn[c];
    conv = conv && stc[4 * c + 3] == 1;
    its = std::max(its, stc[4 * c + 2]);
  }
  if (iters) *iters = its;
  CUDA_TRY(cudaGetLastError());
  return conv ? SPALU_OK : SPALU_ERR_NOCONV;
}

// ------------------------------------------------------------ one graph over the whole step
// Factorization, direct solve and GMRES refinement captured once as a CUDA graph and replayed
// (scheduling; not in the paper).  The solve kernels' shared-memory capacities and the leaf
// sweep variant are fixed by the factorization the graph was captured after, so a guard kernel
// after the factorization checks the new factor's level maxima and leaf bandwidth against
// those: the solve and refinement run inside a conditional node only when they still fit (else
// the host redoes them outside the graph).  The refinement inside the graph is one GMRES cycle
// of at most K Arnoldi steps, each in a conditional node that the previous step's Givens
// kernel switches off once every column has converged.
__global__ void step_guard_kernel(const int* err, const int* kumax, int kumax_ref, const int* lstat,
                                  const int* ref, int L, int* ok_out, cudaGraphConditionalHandle h,
                                  cudaGraphConditionalHandle h2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int ok = (*err == 0 && *kumax <= kumax_ref) ? 1 : 0;
  for (int l = 1; l <= L; ++l)
    for (int q = 0; q < 3; ++q)
      if (lstat[LS_N * l + q] > ref[3 * l + q]) ok = 0;      // LS_EMAX, LS_KPMAX, LS_DPMAX
  *ok_out = ok;
  cudaGraphSetConditional(h, ok ? 1u : 0u);
  cudaGraphSetConditional(h2, ok ? 1u : 0u);
}

static void step_graph_free(spalu_factor_t f) {
  auto& g = f->sg;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  f->timer.drop_graph();
  cudaFree(g.d_ref);
  cudaFree(g.d_ok);
  cudaFreeHost(g.h_out);
  const long long c = g.captures, r = g.replays, rf = g.refits, ct = g.continued;
  g = spalu_factor_s::StepGraph();
  g.captures = c; g.replays = r; g.refits = rf; g.continued = ct;
}

// add an IF node on handle h after what stream s (capturing) has so far; returns its body
static cudaError_t add_if_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) { report_cuda("cudaStreamGetCaptureInfo", e, __LINE__); return e; }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp)) != cudaSuccess) {
    report_cuda("cudaGraphAddNode", e, __LINE__);
    return e;
  }
  *body = cp.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) report_cuda("cudaStreamUpdateCaptureDependencies", e, __LINE__);
  return e;
}

// the cycle's Arnoldi step j (as in refine_impl), enqueued on s
static spalu_status arnoldi_step(spalu_factor_t f, int nrhs, int j, cudaGraphConditionalHandle h, int use_h,
                                 cudaStream_t s) {
  GmresWork& w = f->gw;
  const int m = f->o.gmres_m;
  const size_t ldv = (size_t)f->N;
  auto Vj = [&](int i) { return w.V + (size_t)i * ldv * nrhs; };
  auto Zj = [&](int i) { return w.Z + (size_t)i * ldv * nrhs; };
  spalu_status st = solve_impl(f, Vj(j), w.vs + (size_t)j * nrhs, Zj(j), nrhs, (int)ldv, (spalu_stream_t)s);
  if (st != SPALU_OK) return st;
  vec_spmv(f, nrhs, Zj(j), (int)ldv, nullptr, 0, Vj(j + 1), (int)ldv, Vj(0), (int)ldv, w.vs, w.hcol, 0, s);
  for (int i = 1; i <= j + 1; ++i)
    vec_mgs(f, nrhs, w.hcol + (size_t)(i - 1) * nrhs, Vj(i - 1), (int)ldv, w.vs + (size_t)(i - 1) * nrhs,
            Vj(j + 1), (int)ldv, i <= j ? Vj(i) : nullptr, (int)ldv, w.vs + (size_t)i * nrhs,
            w.hcol + (size_t)i * nrhs, i > j, i > j ? w.vs + (size_t)(j + 1) * nrhs : nullptr, s);
  note_launch();
  launch_pdl(gmres_givens_kernel, dim3(1), dim3(GB), 0, s, nrhs, m, j, f->o.gmres_tol, (const double*)w.hcol,
             (const double*)w.bn, w.H, w.cs, w.sn, w.g, w.vs, w.st, w.flag, h, use_h);
  return SPALU_OK;
}

// Guard references and solve capacities for a capture: the level maxima with some headroom
// (skeleton sizes move by a few unknowns between factorizations of the same matrix: FP32
// rounding, learned sketch sizes), the solve capacities of the captured kernels set from them,
// and the leaf-sweep variant; uploaded before the capture starts.
static spalu_status step_prepare(spalu_factor_t f, spalu_factor_s::StepGraph& G) {
  const int L = f->nd->L;
  if (!G.d_ref) {
    if (cudaMalloc(&G.d_ref, sizeof(int) * 3 * (L + 1)) != cudaSuccess || cudaMalloc(&G.d_ok, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&G.h_out, sizeof(int) * 2) != cudaSuccess)
      return SPALU_ERR_ALLOC;
  }
  std::vector<int> ref(3 * (L + 1), 0);
  for (int l = 1; l <= L; ++l) {
    int lm[LS_N] = {};
    for (int q = 0; q < 3; ++q) {
      const int v = f->lstat[LS_N * l + q];
      lm[q] = v + std::max(4, v / 4);
    }
    SolveCaps c;
    if (level_solve_caps(f->lev[l], lm, &c)) {
      c.seg_nt = f->caps[l].seg_nt;
      c.sep_nt = f->caps[l].sep_nt;
      c.seg_split = f->caps[l].seg_split;
      c.sep_split = f->caps[l].sep_split;
      f->caps[l] = c;
    } else {
      for (int q = 0; q < 3; ++q) lm[q] = f->lstat[LS_N * l + q];
    }
    for (int q = 0; q < 3; ++q) ref[3 * l + q] = lm[q];
  }
  f->kumax = f->kumax <= 15 ? 15 : 30;       // the two leaf-sweep variants
  CUDA_TRY(cudaMemcpy(G.d_ref, ref.data(), sizeof(int) * ref.size(), cudaMemcpyHostToDevice));
  G.K = std::min(f->o.gmres_m, std::max(4, f->gmres_hint + 2));
  return SPALU_OK;
}

// One problem's step enqueued into the capture in progress on stream s (its top-level graph
// takes every node; s2 captures the bodies of the conditional nodes): the matrix copy, the
// factorization, the guard, then in conditional nodes the solve and (refine != 0) one GMRES
// cycle of G.K steps and the update of X; finally the guard result and the "still active" flag
// copied to G.h_out.
static spalu_status capture_step_into(spalu_factor_t f, spalu_factor_s::StepGraph& G, const int* rowptr,
                                      const int* colind, const double* val, int nnz, const double* B, double* X,
                                      int nrhs, int ld, int refine, cudaStream_t s, cudaStream_t s2) {
  const int L = f->nd->L;
  const int N = f->N, m = f->o.gmres_m;
  const int K = refine ? G.K : 0;
  GmresWork& w = f->gw;
  const size_t ldv = (size_t)N;
  G.n_step.assign(K, 0);
  unsigned long long c0 = g_launches.load();
  cudaGraph_t top = nullptr;
#define CAP_TRY(x)                                        \
  do {                                                    \
    cudaError_t _e = (x);                                 \
    if (_e != cudaSuccess) { report_cuda(#x, _e, __LINE__); return SPALU_ERR_CUDA; } \
  } while (0)
  {
    cudaStreamCaptureStatus cs;
    CAP_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &top, nullptr, nullptr, nullptr));
  }
  // every conditional node sits in the top-level graph with a handle of its own (a handle
  // serves one node), reset to 0 at each launch: when the guard fails nothing after it runs;
  // h_act[j] (set by the cycle's set-up or by step j-1) opens Arnoldi step j
  cudaGraphConditionalHandle h_ok, h_ok2;
  std::vector<cudaGraphConditionalHandle> h_act(K + 1);
  CAP_TRY(cudaGraphConditionalHandleCreate(&h_ok, top, 0, cudaGraphCondAssignDefault));
  CAP_TRY(cudaGraphConditionalHandleCreate(&h_ok2, top, 0, cudaGraphCondAssignDefault));
  for (int j = 0; j < K; ++j) CAP_TRY(cudaGraphConditionalHandleCreate(&h_act[j], top, 0, cudaGraphCondAssignDefault));
  CAP_TRY(cudaMemcpyAsync(f->rowptr, rowptr, (N + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CAP_TRY(cudaMemcpyAsync(f->colind, colind, (size_t)nnz * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CAP_TRY(cudaMemcpyAsync(f->val, val, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
  spalu_status st = factor_enqueue(f, s);
  if (st != SPALU_OK) return st;
  note_launch();
  step_guard_kernel<<<1, 32, 0, s>>>(f->d_err, f->leaf.kumax, f->kumax, f->d_lstat, G.d_ref, L, G.d_ok, h_ok, h_ok2);
  CAP_TRY(cudaGetLastError());
  G.n_pre = (long long)(g_launches.load() - c0);
  c0 = g_launches.load();
  // solve, then the cycle's set-up
  cudaGraph_t body;
  CAP_TRY(add_if_node(s, h_ok, &body));
  CAP_TRY(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  st = solve_impl(f, B, nullptr, X, nrhs, ld, (spalu_stream_t)s2);
  if (st == SPALU_OK && refine) {
    vec_mgs(f, nrhs, nullptr, nullptr, 0, nullptr, const_cast<double*>(B), ld, nullptr, 0, nullptr, w.bn, 1,
            nullptr, s2);
    vec_spmv(f, nrhs, X, ld, B, ld, w.V, (int)ldv, nullptr, 0, nullptr, w.beta, 1, s2);
    note_launch();
    gmres_begin_kernel<<<1, GB, 0, s2>>>(nrhs, m, f->o.gmres_tol, w.bn, w.beta, w.vs, w.g, w.st, 1, w.flag, h_act[0],
                                         1);
  }
  {
    cudaGraph_t out2 = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s2, &out2);
    if (st != SPALU_OK) return st;
    CAP_TRY(e);
  }
  // the Arnoldi steps, each while some column is active
  for (int j = 0; j < K; ++j) {
    CAP_TRY(add_if_node(s, h_act[j], &body));
    CAP_TRY(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const unsigned long long cj = g_launches.load();
    st = arnoldi_step(f, nrhs, j, h_act[j + 1], j + 1 < K ? 1 : 0, s2);
    G.n_step[j] = (long long)(g_launches.load() - cj);
    c0 += G.n_step[j];
    cudaGraph_t out2 = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s2, &out2);
    if (st != SPALU_OK) return st;
    CAP_TRY(e);
  }
  if (refine) {
    // the update of X and the residual of the result
    CAP_TRY(add_if_node(s, h_ok2, &body));
    CAP_TRY(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    note_launch();
    launch_pdl(gmres_ysolve_kernel, dim3(1), dim3(GB), 0, s2, nrhs, m, K, (const double*)w.H, (const double*)w.g,
               w.y, w.st);
    note_launch();
    launch_pdl(combine_kernel, vec_grid(N, nrhs), dim3(VB), 0, s2, N, nrhs, K, (const double*)w.y,
               (const double*)w.Z, ldv, X, ld, (const int*)w.st);
    vec_spmv(f, nrhs, X, ld, B, ld, w.V, (int)ldv, nullptr, 0, nullptr, w.beta, 1, s2);
    note_launch();
    gmres_begin_kernel<<<1, GB, 0, s2>>>(nrhs, m, f->o.gmres_tol, w.bn, w.beta, w.vs, w.g, w.st, 0, w.flag,
                                         cudaGraphConditionalHandle{}, 0);
    cudaGraph_t out2 = nullptr;
    CAP_TRY(cudaStreamEndCapture(s2, &out2));
  }
  G.n_ok = (long long)(g_launches.load() - c0);
  CAP_TRY(cudaMemcpyAsync(G.h_out, G.d_ok, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (refine) CAP_TRY(cudaMemcpyAsync(G.h_out + 1, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
#undef CAP_TRY
  return SPALU_OK;
}

// End every capture still open on the given streams (after a failure) and clear the error.
static void abandon_capture(std::initializer_list<cudaStream_t> ss) {
  for (cudaStream_t x : ss) {
    if (!x) continue;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(x, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(x, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
  }
  cudaGetLastError();
}

static spalu_status capture_step(spalu_factor_t f, const int* rowptr, const int* colind, const double* val,
                                 int nnz, const double* B, double* X, int nrhs, int ld) {
  // captured on streams of the call's own (the caller's may be the legacy default stream,
  // which cannot be captured); the graph is launched on the caller's stream
  auto& G = f->sg;
  spalu_status st = step_prepare(f, G);
  if (st != SPALU_OK) return st;
  cudaStream_t s1 = nullptr, s2 = nullptr;
  if (cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) {
    if (s1) cudaStreamDestroy(s1);
    return SPALU_ERR_CUDA;
  }
  f->timer.drop_graph();
  f->timer.cap_top = s1;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s1, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = SPALU_ERR_CUDA;
  if (st == SPALU_OK) st = capture_step_into(f, G, rowptr, colind, val, nnz, B, X, nrhs, ld, 1, s1, s2);
  if (st == SPALU_OK && cudaStreamEndCapture(s1, &graph) != cudaSuccess) st = SPALU_ERR_CUDA;
  if (st != SPALU_OK) abandon_capture({s2, s1});
  if (st == SPALU_OK && cudaGraphInstantiate(&G.exec, graph, 0) != cudaSuccess) {
    G.exec = nullptr;
    st = SPALU_ERR_CUDA;
  }
  f->timer.cap_top = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s1);
  cudaStreamDestroy(s2);
  if (st != SPALU_OK) return st;
  G.key[0] = rowptr; G.key[1] = colind; G.key[2] = val; G.key[3] = B; G.key[4] = X; G.key[5] = f->gw.V;
  G.nnz = nnz; G.nrhs = nrhs; G.ld = ld; G.timed = f->timer.on;
  ++G.captures;
  return SPALU_OK;
}

// After a replay (stream synchronised): the factorization's readback, the launch count of what
// ran, and the cases the graph left open: a failed guard (solve and refine redone outside;
// *refit = true) and columns still above the tolerance (more cycles outside).
static spalu_status step_finish(spalu_factor_t f, spalu_factor_s::StepGraph& G, const double* B, double* X,
                                int nrhs, int ld, int refine, int* iters, double* relres, spalu_stream_t stream,
                                bool* refit) {
  cudaStream_t s = (cudaStream_t)stream;
  *refit = false;
  note_launches(G.n_pre);
  spalu_status st = factor_finish(f, s);
  if (st != SPALU_OK) return st;
  if (!G.h_out[0]) {
    *refit = true;
    if ((st = spalu_solve(f, B, X, nrhs, ld, stream)) != SPALU_OK) return st;
    if (!refine) return SPALU_OK;
    return spalu_refine(f, B, X, nrhs, ld, iters, relres, stream);
  }
  if (!refine) {
    note_launches(G.n_ok);
    return SPALU_OK;
  }
  std::vector<double> bn(nrhs), beta(nrhs);
  std::vector<int> stc(4 * (size_t)nrhs);
  CUDA_TRY(cudaMemcpy(stc.data(), f->gw.st, sizeof(int) * 4 * nrhs, cudaMemcpyDeviceToHost));
  int its = 0;
  for (int c = 0; c < nrhs; ++c) its = std::max(its, stc[4 * c + 2]);
  long long n = G.n_ok;                      // kernels that ran inside the conditional nodes
  for (int j = 0; j < its && j < G.K; ++j) n += G.n_step[j];
  note_launches(n);
  if (G.h_out[1]) {
    // not converged within the captured steps: continue with more cycles outside the graph
    ++G.continued;
    int it2 = 0;
    st = spalu_refine(f, B, X, nrhs, ld, &it2, relres, stream);
    if (iters) *iters = its + it2;
    return st;
  }
  CUDA_TRY(cudaMemcpy(bn.data(), f->gw.bn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(beta.data(), f->gw.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost));
  for (int c = 0; c < nrhs; ++c)
    if (relres) relres[c] = bn[c] == 0.0 ? 0.0 : beta[c] / bn[c];
  if (iters) *iters = its;
  return SPALU_OK;
}

spalu_status spalu_factor_solve_graph(spalu_factor_t f, const int* rowptr, const int* colind, const double* val,
                                      int nnz, const double* B, double* X, int nrhs, int ld, int* iters,
                                      double* relres, spalu_stream_t stream) {
  if (!f || !rowptr || !colind || !val || nnz < 0 || nnz > f->nnz_cap || !B || !X || nrhs < 1 || ld < f->N ||
      X == B)
    return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  auto& G = f->sg;
  const bool fits = G.exec && G.key[0] == rowptr && G.key[1] == colind && G.key[2] == val && G.key[3] == B &&
                    G.key[4] == X && G.nnz == nnz && G.nrhs == nrhs && G.ld == ld && f->gw.nrhs >= nrhs &&
                    G.key[5] == f->gw.V && f->factored && G.timed == f->timer.on;
  if (!fits) {
    // the plain path once (it sets the capacities, the allocations and the step count), then
    // capture the step for the next calls
    if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
    f->timer.drop_graph();
    spalu_status st = spalu_factor_numeric(f, rowptr, colind, val, nnz, stream);
    if (st != SPALU_OK) return st;
    if ((st = spalu_solve(f, B, X, nrhs, ld, stream)) != SPALU_OK) return st;
    st = spalu_refine(f, B, X, nrhs, ld, iters, relres, stream);
    if (st != SPALU_OK && st != SPALU_ERR_NOCONV) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    const spalu_status cst = capture_step(f, rowptr, colind, val, nnz, B, X, nrhs, ld);
    if (cst != SPALU_OK) step_graph_free(f);
    return cst != SPALU_OK ? cst : st;
  }
  f->nnz = nnz;
  int t_step = f->timer.begin("step_graph", s);
  CUDA_TRY(cudaGraphLaunch(G.exec, s));
  f->timer.end(t_step, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  if (G.timed) f->timer.collect_graph();
  ++G.replays;
  bool refit = false;
  const spalu_status st = step_finish(f, G, B, X, nrhs, ld, 1, iters, relres, stream, &refit);
  if (refit) {
    // the new factor outgrew the captured capacities: capture again next time
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    f->timer.drop_graph();
    ++G.refits;
  }
  return st;
}

// ------------------------------------------------------------ many problems as one graph
struct spalu_batch_s {
  int n = 0, refine = 0, nstreams = 1;
  std::vector<spalu_factor_t> f;
  std::vector<spalu_factor_s::StepGraph> G;
  std::vector<const int*> rowptr, colind;
  std::vector<const double*> val, B;
  std::vector<double*> X;
  std::vector<int> nnz, nrhs, ld;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
};

static void batch_release(spalu_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (auto& g : b->G) {
    cudaFree(g.d_ref);
    cudaFree(g.d_ok);
    cudaFreeHost(g.h_out);
    g.d_ref = nullptr; g.d_ok = nullptr; g.h_out = nullptr;
  }
}

// capture every problem's step into one graph: each on one of nstreams forked streams
static spalu_status batch_capture(spalu_batch_s* b) {
  const int n = b->n, K = std::max(1, std::min(b->nstreams, n));
  for (int i = 0; i < n; ++i) {
    const spalu_status st = step_prepare(b->f[i], b->G[i]);
    if (st != SPALU_OK) return st;
  }
  std::vector<cudaStream_t> ss(K, nullptr);
  std::vector<cudaEvent_t> ev(K + 1, nullptr);
  cudaStream_t s0 = nullptr, s2 = nullptr;
  spalu_status st = SPALU_OK;
  if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess)
    st = SPALU_ERR_CUDA;
  for (int k = 0; k < K && st == SPALU_OK; ++k)
    if (cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking) != cudaSuccess) st = SPALU_ERR_CUDA;
  for (int k = 0; k <= K && st == SPALU_OK; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) st = SPALU_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  const unsigned long long c0 = g_launches.load();
  if (st == SPALU_OK && cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = SPALU_ERR_CUDA;
  if (st == SPALU_OK && cudaEventRecord(ev[K], s0) != cudaSuccess) st = SPALU_ERR_CUDA;
  for (int k = 0; k < K && st == SPALU_OK; ++k)
    if (cudaStreamWaitEvent(ss[k], ev[K], 0) != cudaSuccess) st = SPALU_ERR_CUDA;
  for (int i = 0; i < n && st == SPALU_OK; ++i)
    st = capture_step_into(b->f[i], b->G[i], b->rowptr[i], b->colind[i], b->val[i], b->nnz[i], b->B[i], b->X[i],
                           b->nrhs[i], b->ld[i], b->refine, ss[i % K], s2);
  for (int k = 0; k < K && st == SPALU_OK; ++k)
    if (cudaEventRecord(ev[k], ss[k]) != cudaSuccess || cudaStreamWaitEvent(s0, ev[k], 0) != cudaSuccess)
      st = SPALU_ERR_CUDA;
  if (st == SPALU_OK && cudaStreamEndCapture(s0, &graph) != cudaSuccess) st = SPALU_ERR_CUDA;
  if (st != SPALU_OK) {
    std::vector<cudaStream_t> all(ss);
    all.push_back(s2);
    all.push_back(s0);
    for (cudaStream_t x : all) abandon_capture({x});
  }
  if (st == SPALU_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    b->exec = nullptr;
    st = SPALU_ERR_CUDA;
  }
  b->kernels = (long long)(g_launches.load() - c0);
  if (graph) cudaGraphDestroy(graph);
  for (auto e : ev) if (e) cudaEventDestroy(e);
  for (auto x : ss) if (x) cudaStreamDestroy(x);
  if (s2) cudaStreamDestroy(s2);
  if (s0) cudaStreamDestroy(s0);
  return st;
}

spalu_status spalu_batch_graph_create(int n, const spalu_factor_t* f, const int* const* rowptr,
                                      const int* const* colind, const double* const* val, const int* nnz,
                                      const double* const* B, double* const* X, const int* nrhs, const int* ld,
                                      int nstreams, int refine, spalu_stream_t stream, spalu_batch_t* out) {
  if (!out) return SPALU_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !f || !rowptr || !colind || !val || !nnz || !B || !X || !nrhs || !ld || nstreams < 1)
    return SPALU_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!f[i] || !rowptr[i] || !colind[i] || !val[i] || nnz[i] < 0 || nnz[i] > f[i]->nnz_cap || !B[i] || !X[i] ||
        nrhs[i] < 1 || ld[i] < f[i]->N || B[i] == X[i])
      return SPALU_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (f[j] == f[i]) return SPALU_ERR_ARG;       // a handle's buffers serve one problem
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto* b = new spalu_batch_s();
  b->n = n; b->refine = refine ? 1 : 0; b->nstreams = nstreams;
  b->f.assign(f, f + n);
  b->G.resize(n);
  b->rowptr.assign(rowptr, rowptr + n); b->colind.assign(colind, colind + n); b->val.assign(val, val + n);
  b->B.assign(B, B + n); b->X.assign(X, X + n);
  b->nnz.assign(nnz, nnz + n); b->nrhs.assign(nrhs, nrhs + n); b->ld.assign(ld, ld + n);
  // the plain path once per problem (capacities, allocations, step counts)
  spalu_status st = SPALU_OK;
  for (int i = 0; i < n && st == SPALU_OK; ++i) {
    step_graph_free(f[i]);                   // a single-step graph of the handle is given up
    st = spalu_factor_numeric(f[i], rowptr[i], colind[i], val[i], nnz[i], stream);
    if (st == SPALU_OK) st = spalu_solve(f[i], B[i], X[i], nrhs[i], ld[i], stream);
    if (st == SPALU_OK && refine) {
      st = spalu_refine(f[i], B[i], X[i], nrhs[i], ld[i], nullptr, nullptr, stream);
      if (st == SPALU_ERR_NOCONV) st = SPALU_OK;
    }
  }
  if (st == SPALU_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPALU_ERR_CUDA;
  if (st == SPALU_OK) st = batch_capture(b);
  if (st != SPALU_OK) {
    batch_release(b);
    delete b;
    return st;
  }
  *out = b;
  return SPALU_OK;
}

spalu_status spalu_batch_graph_run(spalu_batch_t b, int* iters, double* relres, spalu_stream_t stream) {
  if (!b || !b->exec) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaGraphLaunch(b->exec, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  spalu_status first = SPALU_OK;
  bool any_refit = false;
  std::vector<double> rel;
  for (int i = 0; i < b->n; ++i) {
    rel.assign(b->nrhs[i], 0.0);
    int it = 0;
    bool refit = false;
    spalu_status st = step_finish(b->f[i], b->G[i], b->B[i], b->X[i], b->nrhs[i], b->ld[i], b->refine, &it,
                                  rel.data(), stream, &refit);
    any_refit = any_refit || refit;
    if (iters) iters[i] = it;
    if (relres) relres[i] = rel.empty() ? 0.0 : *std::max_element(rel.begin(), rel.end());
    if (st != SPALU_OK && first == SPALU_OK) first = st;
  }
  if (any_refit && first == SPALU_OK) {        // some factor outgrew its captured capacities
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    first = batch_capture(b);
  }
  return first;
}

void spalu_batch_graph_destroy(spalu_batch_t b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

spalu_status spalu_solve_host(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                              int refine, int* iters, double* relres, spalu_stream_t stream) {
  if (!f || !B || !X || nrhs < 0 || ld < f->N) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  double *dB = nullptr, *dX = nullptr;
  size_t bytes = sizeof(double) * (size_t)f->N * nrhs;
  if (cudaMallocAsync(&dB, bytes, s) != cudaSuccess || cudaMallocAsync(&dX, bytes, s) != cudaSuccess)
    return SPALU_ERR_ALLOC;
  spalu_status st = SPALU_OK;
  if (cudaMemcpy2DAsync(dB, (size_t)f->N * sizeof(double), B, (size_t)ld * sizeof(double),
                        (size_t)f->N * sizeof(double), nrhs, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = SPALU_ERR_CUDA;
  if (st == SPALU_OK) st = spalu_solve(f, dB, dX, nrhs, f->N, stream);
  if (st == SPALU_OK && refine) st = spalu_refine(f, dB, dX, nrhs, f->N, iters, relres, stream);
  spalu_status st2 = SPALU_OK;
  if (st == SPALU_OK || st == SPALU_ERR_NOCONV) {
    if (cudaMemcpy2DAsync(X, (size_t)ld * sizeof(double), dX, (size_t)f->N * sizeof(double),
                          (size_t)f->N * sizeof(double), nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st2 = SPALU_ERR_CUDA;
  }
  cudaFreeAsync(dB, s);
  cudaFreeAsync(dX, s);
  return st != SPALU_OK ? st : st2;
}

spalu_status spalu_factor_solve_host(spalu_factor_t f, const int* rowptr, const int* colind,
                                     const double* val, int nnz, const double* B, double* X, int nrhs,
                                     int ld, int refine, int* iters, double* relres,
                                     spalu_stream_t stream) {
  if (!f || !rowptr || !colind || !val || nnz < 0 || nnz > f->nnz_cap || !B || !X || nrhs < 0 || ld < f->N)
    return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)f->N, need = N * (size_t)nrhs;
  if (!f->up) {
    CUDA_TRY(cudaStreamCreateWithFlags(&f->up, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&f->up_go, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&f->up_done, cudaEventDisableTiming));
  }
  if (need > f->hcap) {
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaStreamSynchronize(f->up));
    cudaFree(f->hB);
    cudaFree(f->hX);
    f->hB = f->hX = nullptr;
    f->hcap = 0;
    if (cudaMalloc(&f->hB, need * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f->hX, need * sizeof(double)) != cudaSuccess)
      return SPALU_ERR_ALLOC;
    f->hcap = need;
  }
  f->nnz = nnz;
  CUDA_TRY(cudaMemcpyAsync(f->rowptr, rowptr, (N + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->colind, colind, (size_t)nnz * sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f->val, val, (size_t)nnz * sizeof(double), cudaMemcpyHostToDevice, s));
  // B follows the matrix (so that it does not slow the matrix upload) on the second stream,
  // after everything earlier on stream (an earlier call's solve may still read hB)
  CUDA_TRY(cudaEventRecord(f->up_go, s));
  CUDA_TRY(cudaStreamWaitEvent(f->up, f->up_go, 0));
  if (nrhs > 0)
    CUDA_TRY(cudaMemcpy2DAsync(f->hB, N * sizeof(double), B, (size_t)ld * sizeof(double), N * sizeof(double),
                               nrhs, cudaMemcpyHostToDevice, f->up));
  CUDA_TRY(cudaEventRecord(f->up_done, f->up));
  spalu_status st = factor_enqueue(f, s);
  if (st == SPALU_OK) st = factor_finish(f, s);
  if (st != SPALU_OK) {
    cudaStreamSynchronize(f->up);
    return st;
  }
  if (nrhs == 0) return SPALU_OK;
  CUDA_TRY(cudaStreamWaitEvent(s, f->up_done, 0));
  st = spalu_solve(f, f->hB, f->hX, nrhs, f->N, stream);
  HostDownload dl{X, ld, f->up, f->up_go, 0};
  if (st == SPALU_OK && refine) {
    const int t = f->timer.begin("refine", s);
    st = refine_impl(f, f->hB, f->hX, nrhs, f->N, iters, relres, stream, &dl);
    f->timer.end(t, s);
  }
  const bool ok = cudaStreamSynchronize(f->up) == cudaSuccess;
  if (st != SPALU_OK && st != SPALU_ERR_NOCONV) return st;
  if (dl.n == 0 &&           // no update of X in the refinement: copy the direct solve
      cudaMemcpy2DAsync(X, (size_t)ld * sizeof(double), f->hX, N * sizeof(double), N * sizeof(double), nrhs,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SPALU_ERR_CUDA;
  if (!ok || cudaStreamSynchronize(s) != cudaSuccess) return SPALU_ERR_CUDA;
  return st;
}

spalu_status spalu_stats(spalu_factor_t f, char* json, size_t cap) {
  if (!f || !json || cap == 0) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  const int L = f->nd->L;
  std::string out = "{\"L\": " + std::to_string(L) + ", \"arena_bytes\": " + std::to_string(f->arena_bytes) + ", \"levels\": [";
  double qt = 0.0;
  std::vector<unsigned long long> fl(4 * (size_t)(L + 1));
  CUDA_TRY(cudaMemcpy(fl.data(), f->d_flops, sizeof(unsigned long long) * fl.size(), cudaMemcpyDeviceToHost));
  for (int l = 1; l <= L; ++l) {
    const LevelDev& d = f->lev[l];
    int n = d.g.nseg();
    std::vector<int> cnt(n), kk(n), hs(n);
    CUDA_TRY(cudaMemcpy(cnt.data(), d.cnt, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(kk.data(), d.kk, sizeof(int) * n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(hs.data(), d.hs, sizeof(int) * n, cudaMemcpyDeviceToHost));
    int emax = 0, kmax = 0;
    long long esum = 0, ksum = 0;
    for (int i = 0; i < n; ++i) {
      emax = std::max(emax, cnt[i]);
      kmax = std::max(kmax, kk[i]);
      esum += cnt[i];
      ksum += kk[i];
    }
    if (emax > 0) qt = std::max(qt, (double)kmax / emax);
    char buf[640];
    const int* ls = f->lstat.data() + LS_N * l;
    std::snprintf(buf, sizeof buf, "%s{\"level\": %d, \"nseg\": %d, \"e_max\": %d, \"k_max\": %d, \"e_sum\": %lld, \"k_sum\": %lld, \"sep_k_max\": %d, \"passes\": %d, \"fallbacks\": %d, \"predicted\": %d, \"flops_sparsify\": %llu, \"flops_merge\": %llu, \"bytes_seg\": %llu, \"bytes_sep\": %llu, \"predictor\": %d}",
                  l == 1 ? "" : ", ", l, n, emax, kmax, esum, ksum, ls[LS_KPMAX], ls[LS_PASSES],
                  ls[LS_FALLBACK], ls[LS_PREDICTED], fl[4 * l], fl[4 * l + 1], fl[4 * l + 2], fl[4 * l + 3],
                  d.pred_mode);
    out += buf;
  }
  char buf[256];
  std::snprintf(buf, sizeof buf, "], \"q_tilde\": %.6f, \"step_graph\": {\"captures\": %lld, \"replays\": %lld, "
                "\"refits\": %lld, \"continued\": %lld}", qt, f->sg.captures, f->sg.replays, f->sg.refits,
                f->sg.continued);
  out += buf;
  f->timer.collect();
  out += ", \"timing_ms\": {";
  bool first = true;
  for (auto& kv : f->timer.ms) {
    char b2[160];
    std::snprintf(b2, sizeof b2, "%s\"%s\": %.6f", first ? "" : ", ", kv.first.c_str(), kv.second);
    out += b2;
    first = false;
  }
  out += "}, \"timing_count\": {";
  first = true;
  for (auto& kv : f->timer.count) {
    char b2[160];
    std::snprintf(b2, sizeof b2, "%s\"%s\": %lld", first ? "" : ", ", kv.first.c_str(), kv.second);
    out += b2;
    first = false;
  }
  out += "}}";
  if (out.size() + 1 > cap) return SPALU_ERR_ARG;
  std::memcpy(json, out.c_str(), out.size() + 1);
  return SPALU_OK;
}

spalu_status spalu_factor_export_level(spalu_factor_t f, int l, int* info, int* cnt, int* kk, int* nodes,
                                       int* skel, int* pcnt, int* pmap) {
  if (!f || !info) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  const int L = f->nd->L;
  if (l < 1 || l > L) return SPALU_ERR_ARG;
  const LevelDev& d = f->lev[l];
  const int nseg = d.g.nseg(), np = d.gp.nbox();
  info[0] = nseg;
  info[1] = d.capS;
  info[2] = np;
  info[3] = d.ldFp;
  cudaStream_t s = f->last_stream;
  const size_t segs = (size_t)nseg * d.capS;
  if (cnt) CUDA_TRY(cudaMemcpyAsync(cnt, d.cnt, sizeof(int) * nseg, cudaMemcpyDeviceToHost, s));
  if (kk) CUDA_TRY(cudaMemcpyAsync(kk, d.kk, sizeof(int) * nseg, cudaMemcpyDeviceToHost, s));
  if (nodes) CUDA_TRY(cudaMemcpyAsync(nodes, d.nodes, sizeof(int) * segs, cudaMemcpyDeviceToHost, s));
  if (skel) CUDA_TRY(cudaMemcpyAsync(skel, d.snodes, sizeof(int) * segs, cudaMemcpyDeviceToHost, s));
  std::vector<int> pc(2 * (size_t)np), tab;
  CUDA_TRY(cudaMemcpyAsync(pc.data(), d.pcount, sizeof(int) * 2 * np, cudaMemcpyDeviceToHost, s));
  if (pmap) {
    tab.resize((size_t)np * d.ldFp * MERGE_TABW);
    CUDA_TRY(cudaMemcpyAsync(tab.data(), d.ptab, sizeof(int) * tab.size(), cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  if (pcnt) std::memcpy(pcnt, pc.data(), sizeof(int) * 2 * np);
  if (pmap) {
    for (int P = 0; P < np; ++P) {
      const int n = pc[2 * P] + pc[2 * P + 1];
      if (n < 0 || n > d.ldFp) return SPALU_ERR_CUDA;
      for (int x = 0; x < n; ++x) {
        const int* e = tab.data() + ((size_t)P * d.ldFp + x) * MERGE_TABW;
        pmap[((size_t)P * d.ldFp + x) * 2] = e[0];
        pmap[((size_t)P * d.ldFp + x) * 2 + 1] = e[7];
      }
    }
  }
  return SPALU_OK;
}

spalu_status spalu_residual_noalloc(spalu_factor_t f, const double* B, const double* X, int nrhs,
                                    int ld, double* relres, spalu_stream_t stream) {
  if (!f) return SPALU_ERR_ARG;
  if (!f->factored) return SPALU_ERR_STATE;
  return residual_noalloc(f->N, f->rowptr, f->colind, f->val, B, X, nrhs, ld, relres,
                          (cudaStream_t)stream);
}

spalu_status spalu_set_timing(spalu_factor_t f, int on) {
  if (!f) return SPALU_ERR_ARG;
  f->timer.reset();
  f->timer.on = on != 0;
  return SPALU_OK;
}

unsigned long long spalu_kernel_launches(void) { return g_launches.load(); }

// ---------------------------------------------------------------- learned rank predictor
void spalu_predictor_destroy(spalu_predictor_t p) {
  if (!p) return;
  if (p->epoch) cudaGraphExecDestroy(p->epoch);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->params); cudaFree(p->m); cudaFree(p->v); cudaFree(p->grad); cudaFree(p->partial);
  cudaFree(p->step); cudaFree(p->dev);
  delete p;
}

spalu_status spalu_predictor_create(const float* params, spalu_predictor_t* out) {
  if (!params || !out) return SPALU_ERR_ARG;
  *out = nullptr;
  auto* p = new spalu_predictor_s();
  const size_t np = PRED_NPARAM;
  if (cudaMalloc(&p->params, np * 4) != cudaSuccess || cudaMalloc(&p->m, np * 4) != cudaSuccess ||
      cudaMalloc(&p->v, np * 4) != cudaSuccess || cudaMalloc(&p->grad, (np + 1) * 4) != cudaSuccess ||
      cudaMalloc(&p->partial, (size_t)PRED_MAXBLK * (np + 1) * 4) != cudaSuccess ||
      cudaMalloc(&p->step, sizeof(int)) != cudaSuccess || cudaMalloc(&p->dev, sizeof(PredDev)) != cudaSuccess) {
    spalu_predictor_destroy(p);
    return SPALU_ERR_ALLOC;
  }
  PredDev h{};
  for (int i = 0; i < PRED_NFEAT; ++i) { h.mu[i] = 0.0f; h.isd[i] = 1.0f; }
  bool ok = cudaMemcpy(p->params, params, np * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(p->m, 0, np * 4) == cudaSuccess && cudaMemset(p->v, 0, np * 4) == cudaSuccess &&
            cudaMemset(p->step, 0, sizeof(int)) == cudaSuccess &&
            cudaMemcpy(p->dev, &h, sizeof(PredDev), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    launch_pred_to_bf16(p->params, p->dev, nullptr);
    ok = cudaStreamSynchronize(nullptr) == cudaSuccess;
  }
  if (!ok) {
    spalu_predictor_destroy(p);
    return SPALU_ERR_CUDA;
  }
  *out = p;
  return SPALU_OK;
}

spalu_status spalu_predictor_get_params(spalu_predictor_t p, float* params, spalu_stream_t stream) {
  if (!p || !params) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(params, p->params, PRED_NPARAM * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SPALU_OK;
}

spalu_status spalu_predictor_set_norm(spalu_predictor_t p, const float* mu, const float* isd,
                                      spalu_stream_t stream) {
  if (!p || !mu || !isd) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(p->dev->mu, mu, PRED_NFEAT * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(p->dev->isd, isd, PRED_NFEAT * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SPALU_OK;
}

spalu_status spalu_predictor_get_norm(spalu_predictor_t p, float* mu, float* isd, spalu_stream_t stream) {
  if (!p || !mu || !isd) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(mu, p->dev->mu, PRED_NFEAT * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(isd, p->dev->isd, PRED_NFEAT * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return SPALU_OK;
}

spalu_status spalu_predictor_fit_norm(spalu_predictor_t p, const float* X, int n, spalu_stream_t stream) {
  if (!p || !X || n < 1) return SPALU_ERR_ARG;
  launch_pred_fit_norm(X, n, p->dev, (cudaStream_t)stream);
  CUDA_TRY(cudaGetLastError());
  return SPALU_OK;
}

spalu_status spalu_predictor_loss_grad(spalu_predictor_t p, const float* X, const float* Y, int n,
                                       float* loss, float* grad, spalu_stream_t stream) {
  if (!p || !X || !Y || n < 1 || !loss) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  launch_pred_grad(p->params, p->dev, X, Y, 0, n, p->partial, p->grad, nullptr, s);
  std::vector<float> g(PRED_NPARAM + 1);
  CUDA_TRY(cudaMemcpyAsync(g.data(), p->grad, g.size() * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *loss = g[PRED_NPARAM] / (2.0f * n);
  if (grad) std::memcpy(grad, g.data(), PRED_NPARAM * 4);
  return SPALU_OK;
}

spalu_status spalu_predictor_train(spalu_predictor_t p, const float* X, const float* Y, int n, int epochs,
                                   int batch, float lr, float* loss, spalu_stream_t stream) {
  if (!p || !X || !Y || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0f)) return SPALU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nbatch = (n + batch - 1) / batch;
  // one epoch (gradient, reduction and Adam per batch) is captured once as a CUDA graph and
  // replayed; it is recaptured when the data, sizes or learning rate change
  if (!p->epoch || p->g_X != X || p->g_Y != Y || p->g_n != n || p->g_batch != batch || p->g_lr != lr) {
    if (p->epoch) { cudaGraphExecDestroy(p->epoch); p->epoch = nullptr; }
    if (!p->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    const unsigned long long l0 = g_launches.load();
    CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int b = 0; b < nbatch; ++b) {
      const int r0 = b * batch, nb = std::min(batch, n - r0);
      launch_pred_grad(p->params, p->dev, X, Y, r0, nb, p->partial, p->grad, p->step, p->cap_stream);
      launch_pred_adam(p->params, p->m, p->v, p->grad, p->step, lr, p->dev, p->cap_stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
    const long long captured = (long long)(g_launches.load() - l0);
    note_launches(-captured);                      // nothing ran during the capture
    if (ce != cudaSuccess) return SPALU_ERR_CUDA;
    ce = cudaGraphInstantiate(&p->epoch, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { p->epoch = nullptr; return SPALU_ERR_CUDA; }
    p->g_X = X; p->g_Y = Y; p->g_n = n; p->g_batch = batch; p->g_lr = lr;
  }
  for (int e = 0; e < epochs; ++e) {
    CUDA_TRY(cudaGraphLaunch(p->epoch, s));
    note_launches(3LL * nbatch);
  }
  if (loss) {
    launch_pred_grad(p->params, p->dev, X, Y, 0, n, p->partial, p->grad, nullptr, s);
    float l2 = 0.0f;
    CUDA_TRY(cudaMemcpyAsync(&l2, p->grad + PRED_NPARAM, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *loss = l2 / (2.0f * n);
  }
  CUDA_TRY(cudaGetLastError());
  return SPALU_OK;
}

spalu_status spalu_predictor_infer(spalu_predictor_t p, const float* X, int n, float* out,
                                   spalu_stream_t stream) {
  if (!p || !X || !out || n < 0) return SPALU_ERR_ARG;
  launch_pred_infer(p->dev, X, n, out, (cudaStream_t)stream);
  CUDA_TRY(cudaGetLastError());
  return SPALU_OK;
}

spalu_status spalu_factor_set_predictor(spalu_factor_t f, spalu_predictor_t p, int mode, double margin) {
  if (!f || mode < PRED_OFF || mode > PRED_PREDICT || !(margin >= 0.0)) return SPALU_ERR_ARG;
  if (mode == PRED_PREDICT && !p) return SPALU_ERR_ARG;
  step_graph_free(f);        // a captured step holds the old predictor settings
  f->pred = p;
  f->pred_mode = mode;
  for (int l = 1; l <= f->nd->L; ++l) {
    f->lev[l].pred_mode = mode;
    f->lev[l].pred_margin = margin;
    f->lev[l].pred = p ? p->dev : nullptr;
  }
  return SPALU_OK;
}

spalu_status spalu_factor_export_training(spalu_factor_t f, float* X, float* Y, int cap, int* n_out,
                                          spalu_stream_t stream) {
  if (!f || !X || !Y || cap < 0 || !n_out) return SPALU_ERR_ARG;
  if (!f->factored || f->pred_mode != PRED_RECORD) return SPALU_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemsetAsync(f->d_count, 0, sizeof(int), s));
  for (int l = f->nd->L; l >= 1; --l)
    launch_pred_export(f->lev[l].feat, f->lev[l].tgt, f->lev[l].g.nseg(), f->o.p_oversample, X, Y, cap,
                       f->d_count, s);
  int n = 0;
  CUDA_TRY(cudaMemcpyAsync(&n, f->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *n_out = n;
  return SPALU_OK;
}

void spalu_factor_destroy(spalu_factor_t f) {
  if (!f) return;
  cudaFree(f->arena);
  cudaFree(f->xf);
  cudaFreeHost(f->hpin);
  gmres_free(f->gw);
  step_graph_free(f);
  if (f->up) {
    cudaStreamSynchronize(f->up);
    cudaStreamDestroy(f->up);
    cudaEventDestroy(f->up_go);
    cudaEventDestroy(f->up_done);
  }
  cudaFree(f->hB);
  cudaFree(f->hX);
  delete f;
}

}  // extern "C"
