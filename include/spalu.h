/*
 * spalu.h - C ABI of the GB300 implementation of the recursive sparse LU ("spaLU") fast
 * direct solver for 5-point finite-difference matrices on regular 2-D grids.
 *
 * The method (Zhu & Lai, arXiv 2408.14193):
 *   - nested dissection of the grid into leaf boxes and separators (Sec. 2.2, Alg. 1);
 *   - elimination of every leaf interior by LU, leaving the Schur complement on the
 *     separators (Sec. 4.3, first step);
 *   - for levels l = L..1: sparsification of every separator segment by an interpolative
 *     decomposition of its sampled interaction block (Secs. 4.1-4.2, 4.5), elimination of
 *     the redundant (remainder) unknowns, elimination of the level-l separators, and the
 *     merge of the remaining skeletons into the segments of level l-1 (Sec. 4.3, Alg. 2);
 *   - the tree-ordered forward / backward solve A ~= W~^{-1} V~^{-1} (Eq. (WV)).
 *
 * Conventions shared by every call:
 *   - Grid: nx x ny interior nodes, natural index g = x + nx*y.  nx+1 and ny+1 must be
 *     16 * 2^k (leaf boxes of 15 x 15 interior nodes with 1-wide separators).
 *   - Matrix: CSR in natural order, int32 row pointers / column indices, float64 values,
 *     device memory owned by the caller; its pattern must be the 5-point stencil (entries
 *     only between grid neighbours and on the diagonal).
 *   - Right-hand sides / solutions: float64, column-major, leading dimension ld >= N.
 *   - Streams: every call enqueues on the given stream (NULL = legacy default stream);
 *     calls that return results to the host synchronise that stream.
 *   - Ownership: handles are created and destroyed by the library; all memory passed in
 *     stays owned by the caller.  A handle is not safe for concurrent use from several
 *     host threads.
 *   - Errors: every call returns a status; the library never aborts, exits or traps on the
 *     device.  Device-side failures (zero pivot, non-finite value) are reported through an
 *     error word read by the host at the end of the call.
 */
#ifndef SPALU_H
#define SPALU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* spalu_stream_t;          /* same type as cudaStream_t */
typedef struct spalu_nd_s* spalu_nd_t;               /* opaque, library-owned */
typedef struct spalu_factor_s* spalu_factor_t;       /* opaque, library-owned, owns device memory */
typedef struct spalu_predictor_s* spalu_predictor_t; /* opaque, library-owned, owns device memory */
typedef struct spalu_batch_s* spalu_batch_t;         /* opaque, library-owned */

typedef enum {
  SPALU_OK = 0,
  SPALU_ERR_ARG = -1,          /* invalid argument (sizes, pointers, grid shape) */
  SPALU_ERR_ALLOC = -2,        /* device or host allocation failed */
  SPALU_ERR_SINGULAR = -3,     /* an exactly zero pivot met in an LU */
  SPALU_ERR_NOCONV = -4,       /* refinement did not reach the tolerance */
  SPALU_ERR_TIMEOUT = -5,      /* a bounded device wait expired */
  SPALU_ERR_CUDA = -6,         /* a CUDA runtime call failed */
  SPALU_ERR_UNSUPPORTED = -7,  /* valid request the library does not implement */
  SPALU_ERR_NONFINITE = -8,    /* a NaN or Inf appeared in the factor */
  SPALU_ERR_STATE = -9         /* call made on a handle in the wrong state */
} spalu_status;

/* Options fixed at factor time. */
typedef struct {
  double eps_id;              /* ID tolerance, relative: stop at the first |R_kk| <= eps |R_11|
                                 (Sec. 4.1).  0 = no sparsification (exact block LU). */
  int precision;              /* 0 = FP64 throughout; 1 = mixed (FP32 Schur updates / solve,
                                 FP64 pivoted LU and CPQR pivots/norms) */
  int symmetric;              /* 1: caller asserts A = A^T and B = A_{n,i} is sampled;
                                 0: B = [A_{n,i}; A_{i,n}^T] (Sec. 4.5, Eq. (ID [A_ni; A_in])) */
  int p_oversample;           /* p of h = k + p (Sec. 4.2.3), default 5 */
  int near_radius;            /* Chebyshev radius of the near field, default 2 (hybrid
                                 sampling, Sec. 4.2.3: near rows kept exactly, far rows
                                 sketched); -1: no near field, every neighbour row is
                                 sketched (pure randomized sampling, Sec. 4.2.1) */
  int h0;                     /* first sketch size, default 16 (segments with e + p <= 2 h0 are
                                 sketched once with h = 2 h0: their rank is <= e <= h - p) */
  unsigned long long seed;    /* key of the Philox4x32-10 stream of the sketch */
  int gmres_m;                /* restart length of the refinement, default 30 */
  int gmres_maxit;            /* total iteration cap of the refinement, default 200 */
  double gmres_tol;           /* target ||b - A x|| / ||b||, default 1e-10 */
  int spars_ctas;             /* performance only: the sparsification's per-segment shared
                                 memory is cut to what lets min(spars_ctas, ceil(segments of
                                 the level / SMs)) segments (at most what the register file
                                 holds) run at once on an SM; a segment that does not fit
                                 keeps its sketch rows in global memory (results agree up to
                                 rounding).  A level with at most one segment per SM gets
                                 160 KB (room for larger sketch chunks and the staged
                                 neighbour block).  0 = size for the largest segment the
                                 geometry allows.  Default 4. */
  int schur_tc;               /* mixed precision only: 1 (default) = the separators' Schur
                                 updates M -= Z W run on the tensor cores (mma.sync TF32 with
                                 the operands split into high and low TF32 parts, three
                                 products per tile: FP32-level accuracy); 0 = FP32 FMA on the
                                 CUDA cores.  Ignored in FP64 mode. */
  int sketch_tc;              /* mixed precision only: 1 = the sketch products G B_F
                                 (Sec. 4.2.3) on the tensor cores (the same split-TF32
                                 mma.sync); 0 (default) = FP32 FMA on the CUDA cores (the
                                 random entries of G, not the product, dominate the sketch's
                                 cost).  Ignored in FP64 mode. */
  int leaf_bwd;               /* mixed precision only, performance only: the backward leaf
                                 step x_I -= A_II^{-1} A_Id x_d (Eq. (WV)) as 0 = one product
                                 with G = A_II^{-1} A_Id, stored by the factorization (225 x 60
                                 FP32 per leaf, independent rows); 1 = a band sweep pair per
                                 leaf on the stored factors (no G: less memory and traffic, but
                                 225 dependent steps); -1 (default) = G on grids of fewer than
                                 2048 leaves, the sweeps otherwise.  FP64 mode always sweeps. */
} spalu_opts;

/* Fill *o with the defaults listed above (eps_id = 1e-8, precision 0, symmetric 0). */
void spalu_default_opts(spalu_opts* o);

const char* spalu_status_string(spalu_status s);

/* Nested dissection of an nx x ny grid (Alg. 1 on a regular grid, Sec. 3).
 * leaf_pitch must be 16.  Builds the order I (Sec. 2.2) on the device and the level
 * tables on the host.  *out receives a new handle (release with spalu_nd_destroy). */
spalu_status spalu_nd_build_grid(int nx, int ny, int leaf_pitch, spalu_stream_t stream,
                                 spalu_nd_t* out);

/* Copy the ND order to host memory: perm[i] = grid node of the i-th unknown of order I,
 * iperm[g] = position of node g (either pointer may be NULL).  levels[0] receives L and,
 * for level l = 1..L, levels[8*l .. 8*l+7] = {bx, by, w, h, vertical_cut, nseg, ncorner,
 * nsep} of the depth-l box tiling (levels may be NULL; cap = its length in ints).
 * Synchronises the stream the handle was built on. */
spalu_status spalu_nd_export(spalu_nd_t nd, int* perm, int* iperm, int* levels, int cap);

/* Grid nodes of the finest-level segments (sides of leaf boxes), segment after segment in
 * segment-id order, 15 each in increasing coordinate; nodes must hold 15 * nseg(L) ints. */
spalu_status spalu_nd_export_segments(spalu_nd_t nd, int* nodes, int cap);

/* Nested dissection of a general graph with vertex coordinates (Sec. 3.1, Alg. 1; the
 * separator walk of Eq. (degreebias) with theta = 0.1), computed on the host: the ordering
 * only (the factorization takes regular grids, spalu_nd_build_grid).  Host arrays: rowptr
 * (n + 1) and colind, the symmetric sparsity pattern of the matrix (diagonal entries
 * ignored); xy (2n doubles: x, y of vertex v at xy[2v], xy[2v + 1]); boundary (n flags for
 * the domain's boundary vertices, may be NULL: then the vertices with fewer neighbours than
 * the most connected one, the boundary of a grid).  A part with at most leaf_size >= 1
 * vertices is a leaf.  Out: perm (n) = order I (leaves in depth-first order, each in
 * increasing vertex id, then the separators by level L..1, each in walk order); level (n,
 * may be NULL) = 0 for a leaf vertex, l for a vertex of a level-l separator.  The walk ends
 * at D <= 0, at a dead end or at the first vertex on the part's boundary; D values within
 * 1e-12 count as equal (first neighbour in adjacency order wins); the rest of a part goes to
 * the separator's sides by connected component.  On a grid with leaf_size 225 the result is
 * the order of spalu_nd_build_grid.  Errors: SPALU_ERR_ARG (sizes, indices out of range,
 * non-finite coordinates). */
spalu_status spalu_nd_order_csr(int n, const int* rowptr, const int* colind, const double* xy,
                                const unsigned char* boundary, int leaf_size, int* perm, int* level);

void spalu_nd_destroy(spalu_nd_t nd);

/* Allocate a factor for the grid of nd with options o (all device memory is allocated here,
 * once).  nd must outlive the factor. */
spalu_status spalu_factor_create(spalu_nd_t nd, const spalu_opts* o, spalu_factor_t* out);

/* Numeric factorization (Alg. 2) of the CSR matrix (device pointers, natural order,
 * nnz entries).  Enqueued on stream; synchronises it at the end to read the device
 * error word. */
spalu_status spalu_factor_numeric(spalu_factor_t f, const int* rowptr, const int* colind,
                                  const double* val, int nnz, spalu_stream_t stream);

/* Same, with rowptr / colind / val in host memory, copied to the device inside the call
 * (page-locked host memory gives full copy bandwidth). */
spalu_status spalu_factor_numeric_host(spalu_factor_t f, const int* rowptr, const int* colind,
                                       const double* val, int nnz, spalu_stream_t stream);

/* Direct solve X = V~ W~ B (Eq. (WV)) for nrhs columns (device pointers, column-major,
 * leading dimension ld).  X may alias B.  Does not synchronise. */
spalu_status spalu_solve(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                         spalu_stream_t stream);

/* Batched numeric factorization of n independent problems (Sec. 4.3 per problem): problem i
 * factors f[i] (created for its own grid) from the device CSR arrays rowptr[i], colind[i],
 * val[i] (nnz[i] entries) on streams[i].  Every problem's copies and kernels are enqueued
 * first, then each stream is synchronised and its factor finished, so problems on different
 * streams run concurrently.  Host arrays of n pointers / counts; the handles and the CSR
 * arrays stay owned by the caller; a stream may serve several problems (they then run in
 * order).  Returns the first non-OK status (SPALU_ERR_ARG before anything is enqueued when an
 * argument is invalid); every problem that was enqueued is finished either way. */
spalu_status spalu_factor_numeric_batch(int n, const spalu_factor_t* f, const int* const* rowptr,
                                        const int* const* colind, const double* const* val,
                                        const int* nnz, spalu_stream_t const* streams);

/* Autotuning of the level solves (scheduling, not in the paper): for every level, time the
 * segment and separator solve kernels with 2-warp and 8-warp CTAs and with the right-hand
 * sides split into 1, 2, 4 or 8 groups of one CTA each (more CTAs on levels with few
 * segments or separators) -- every combination, on a zero vector of nrhs columns,
 * 1 <= nrhs <= 16, CUDA events on stream -- and keep the fastest for later solves of this
 * handle, also across re-factorizations.  Requires a factored handle (SPALU_ERR_STATE
 * otherwise); synchronises the stream.  Results do not depend on the choice beyond the order
 * of the atomic separator updates. */
spalu_status spalu_tune_solve(spalu_factor_t f, int nrhs, spalu_stream_t stream);

/* Autotuning of the sparsification's occupancy (scheduling, not in the paper): re-factor the
 * handle's last matrix once per candidate shared-memory budget of the sparsify kernel (the
 * uncut worst case, then budgets for 2, 3, 4, 6, 8 and 12 resident segments per SM, see
 * spars_ctas), time every level's sparsification with CUDA events on stream, and keep the
 * fastest budget per level for later factorizations of this handle.  Ends with one more
 * factorization under the chosen budgets, so the handle is factored on return.  In predict
 * mode (spalu_factor_set_predictor) it also times every level with and without the network
 * and keeps the network only on the levels where it was faster (per-level "predictor" in
 * spalu_stats; the next spalu_factor_set_predictor call resets the choice).  Requires a
 * factored handle (SPALU_ERR_STATE otherwise); synchronises the stream; leaves the phase
 * timings of spalu_factor_stats as they were.  With the predictor choice unchanged the
 * factors agree with untuned ones up to rounding. */
spalu_status spalu_tune_factor(spalu_factor_t f, spalu_stream_t stream);

/* Batched direct solve: spalu_solve(f[i], B[i], X[i], nrhs[i], ld[i], streams[i]) for
 * i < n, enqueued in order; does not synchronise.  Returns the first non-OK status (the
 * problems after it are not enqueued). */
spalu_status spalu_solve_batch(int n, const spalu_factor_t* f, const double* const* B, double* const* X,
                               const int* nrhs, const int* ld, spalu_stream_t const* streams);

/* Iterative refinement by right-preconditioned GMRES(m) with the factor as preconditioner
 * and an FP64 residual with the last factored matrix: every column is iterated until
 * ||b - A x|| <= tol ||b||.  X holds the initial guess on entry (e.g. from spalu_solve)
 * and the result on exit.  iters (host, may be NULL) receives the largest iteration count
 * over the columns, relres (host, nrhs entries, may be NULL) the final relative residuals.
 * Returns SPALU_ERR_NOCONV when a column did not converge within gmres_maxit.
 * Synchronises the stream. */
spalu_status spalu_refine(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                          int* iters, double* relres, spalu_stream_t stream);

/* Host-memory variant of solve + refine: B and X are host arrays; the copies to and from
 * the device happen inside the call.  refine = 0 returns the direct solve. */
spalu_status spalu_solve_host(spalu_factor_t f, const double* B, double* X, int nrhs, int ld,
                              int refine, int* iters, double* relres, spalu_stream_t stream);

/* Factor and solve from host memory in one call (Secs. 4.3-4.4): the numeric factorization of
 * the host CSR arrays (as spalu_factor_numeric_host), then X = spaLU^{-1} B refined as
 * spalu_refine when refine != 0 (as spalu_solve_host).  The upload of B runs on a second
 * stream owned by the handle while the factorization's kernels run, and the copy of X back
 * runs there too, after each update of X, while the refinement checks its residual; B and X
 * live in device
 * buffers the handle keeps (grown on demand, freed with it), so a repeated call allocates
 * nothing.  Host arrays: rowptr (N + 1), colind and val (nnz), B and X (nrhs columns of
 * leading dimension ld >= N; page-locked memory gives full copy bandwidth).  Synchronises
 * stream.  Returns the factorization's status if it fails (nothing is solved), else the
 * solve's (SPALU_ERR_NOCONV still fills X). */
spalu_status spalu_factor_solve_host(spalu_factor_t f, const int* rowptr, const int* colind,
                                     const double* val, int nnz, const double* B, double* X, int nrhs,
                                     int ld, int refine, int* iters, double* relres,
                                     spalu_stream_t stream);

/* The whole step as one CUDA graph (scheduling; not in the paper): the numeric factorization
 * of the device CSR arrays (as spalu_factor_numeric), the direct solve X = spaLU^{-1} B (as
 * spalu_solve) and GMRES refinement of X (as spalu_refine), with one host synchronisation at
 * the end.  The first call for a given set of arguments (the same pointers, nnz, nrhs, ld)
 * runs the three calls plainly and then captures the step; later calls with the same
 * arguments replay the graph.  Inside it, a guard kernel after the factorization checks that
 * the new factor still fits the solve kernels' capacities fixed at capture (per-level largest
 * segment, separator skeleton and separator boundary, leaf upper bandwidth); when it does not,
 * the solve and refinement are skipped in the graph and redone outside it (the next call
 * captures again).  The refinement inside the graph is one GMRES cycle of up to K =
 * min(m, max(4, steps of the last plain refinement + 2)) Arnoldi steps, each a conditional
 * node that runs only while a column is above the tolerance; columns still above it after
 * the graph continue with spalu_refine.  B and X: device, column-major, leading dimension ld;
 * X must not alias B; 1 <= nrhs.  The arrays must stay valid between calls that reuse them.
 * iters / relres (host, may be NULL) as in spalu_refine.  Per-phase timing
 * (spalu_set_timing) records nothing inside the graph.  Synchronises the stream. */
spalu_status spalu_factor_solve_graph(spalu_factor_t f, const int* rowptr, const int* colind, const double* val,
                                      int nnz, const double* B, double* X, int nrhs, int ld, int* iters,
                                      double* relres, spalu_stream_t stream);

/* Many independent problems as one CUDA graph (scheduling; not in the paper): problem i is
 * the step of spalu_factor_solve_graph for handle f[i] (its own grid and options), CSR matrix
 * rowptr[i] / colind[i] / val[i] (nnz[i] entries), right-hand sides B[i] and solution X[i]
 * (nrhs[i] >= 1 columns, leading dimension ld[i], X[i] != B[i]): numeric factorization, direct
 * solve and, with refine != 0, one GMRES cycle in conditional nodes.  The problems' nodes are
 * spread over nstreams branches of the one graph so that they run concurrently.  create runs
 * every problem once plainly on stream (setting capacities, allocations and step counts),
 * then captures; *out receives the handle.  The handles f[i] must be distinct, stay alive and
 * unused by other calls while the batch exists, and every array must stay valid and in place
 * (new values may be written into them between runs).  SPALU_ERR_ARG on an invalid argument
 * (nothing is run). */
spalu_status spalu_batch_graph_create(int n, const spalu_factor_t* f, const int* const* rowptr,
                                      const int* const* colind, const double* const* val, const int* nnz,
                                      const double* const* B, double* const* X, const int* nrhs, const int* ld,
                                      int nstreams, int refine, spalu_stream_t stream, spalu_batch_t* out);
/* Launch the batch graph on stream and wait for it.  iters[i] / relres[i] (host arrays of n,
 * may be NULL): the GMRES steps and the largest relative residual of problem i (with
 * refine).  A problem whose new factor outgrew the captured solve capacities is solved and
 * refined outside the graph (the batch is captured again afterwards); columns still above
 * the tolerance after the graph's cycle continue with spalu_refine.  Returns the first
 * non-OK status of the problems (every problem is finished either way). */
spalu_status spalu_batch_graph_run(spalu_batch_t b, int* iters, double* relres, spalu_stream_t stream);
void spalu_batch_graph_destroy(spalu_batch_t b);

/* JSON summary of the last factorization: per level the segment sizes and ranks, the
 * largest separator skeleton, the number of IDs computed ("passes"), of predicted one-pass
 * IDs and of those that fell back to the adaptive schedule; q~ (Sec. 6); device bytes
 * held.  Synchronises the factor's stream. */
spalu_status spalu_stats(spalu_factor_t f, char* json, size_t cap);

/* Index tables of level l (1 <= l <= L) as the last factorization left them, for parity
 * checks of the segment bookkeeping (Secs. 2.3.1, 3.2), the IDs (Sec. 4.2) and the merge
 * E_(l) (Sec. 4.3).  info (host, 4 ints) receives {nseg, capS, nparent, ldFp}; call once with
 * only info to size the arrays.  Every other pointer is a host array and may be NULL:
 *   cnt   [nseg]           unknowns of segment s entering level l;
 *   kk    [nseg]           skeleton size k of segment s (k = cnt when eps_id = 0);
 *   nodes [nseg * capS]    grid nodes of segment s entering level l (first cnt[s] valid):
 *                          at the finest level the side in increasing coordinate, above it
 *                          the merge of the finer level's skeletons and junction;
 *   skel  [nseg * capS]    the same nodes in ID order: the first kk[s] are the skeleton in
 *                          pivot order, the rest the remainders;
 *   pcnt  [2 * nparent]    per depth-(l-1) box P (row-major in its tiling): |dP| (unknowns on
 *                          P's boundary after the merge) and k_p (skeleton size of the
 *                          level-l separator that cuts P);
 *   pmap  [2 * nparent * ldFp]  per box P, its first |dP| + k_p entries: pairs (position in
 *                          P's frontal block, grid node) in merge order: P's sides (bottom,
 *                          top, left, right; a side cut by the separator is skeleton of child
 *                          1, the junction, skeleton of child 2), P's corners (BL, BR, TL,
 *                          TR, those that exist), then the separator's skeleton; positions:
 *                          bottom [0, w), top [w, 2w), left [2w, 2w + h), right
 *                          [2w + h, 2w + 2h), corners 2w + 2h + {0..3}, separator from
 *                          2w + 2h + 4 (from 0 at l = 1, where P is the whole grid);
 *                          w x h is the box size of depth l - 1.
 * SPALU_ERR_STATE when f is not factored.  Synchronises the stream of the last factorization. */
spalu_status spalu_factor_export_level(spalu_factor_t f, int l, int* info, int* cnt, int* kk, int* nodes,
                                       int* skel, int* pcnt, int* pmap);

/* Relative residual norms relres[c] = ||B_c - A X_c||_2 / ||B_c||_2 (0 when B_c = 0) of nrhs
 * columns against the matrix of the last factorization, computed without allocating any
 * device memory.  The paper has no counterpart: this serves callers that cannot let the
 * library allocate when they check a solution, such as hosts that give all device memory to
 * their own pool and forbid later allocations by libraries, or processes so close to the
 * device-memory limit that a new allocation would fail.
 * B, X: device, column-major, leading dimension ld >= N; relres: host, nrhs entries.
 * The reduction goes through one fixed scratch array of 64 * 512 * 2 + 64 doubles
 * (about 0.5 MB) held by every GPU that loads the library until the process exits, so
 * nrhs may be at most 64 (larger values return SPALU_ERR_ARG and compute nothing).
 * The first call on a device looks the array's address up (with that device current) and
 * should come before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be serialised by the
 * caller.  The looked-up address is kept for the life of the process, so the call must not
 * be used across a cudaDeviceReset.  Synchronises the stream to return relres. */
spalu_status spalu_residual_noalloc(spalu_factor_t f, const double* B, const double* X, int nrhs,
                                    int ld, double* relres, spalu_stream_t stream);

/* Per-phase timing: with on != 0, every later factor / solve / refine call on f records a
 * pair of CUDA events around each of its kernel phases on the stream it launches on;
 * spalu_stats then reports, per phase name, the summed milliseconds and the count of
 * recorded intervals ("timing_ms", "timing_count").  Calling it resets the sums.
 * Off by default (no events are recorded). */
spalu_status spalu_set_timing(spalu_factor_t f, int on);

/* Number of CUDA kernels this library has launched so far in the calling process, over all
 * handles (a diagnostic counter; never reset). */
unsigned long long spalu_kernel_launches(void);

/* Measured FMA throughput of the current device's CUDA cores (a diagnostic; not in the paper):
 * precision 0 = FP64, 1 = FP32.  Runs a kernel of independent fused multiply-add chains on
 * every SM, timed with CUDA events on stream (best of three after a warm-up launch), and
 * writes the rate in FLOP/s (an FMA counts 2) to *flops.  These rates bound the small dense
 * kernels of the factorization (leaf LU, ID, block eliminations).  Synchronises the stream. */
spalu_status spalu_measure_fma_peak(int precision, double* flops, spalu_stream_t stream);

void spalu_factor_destroy(spalu_factor_t f);

/* ------------------------------------------------------------------------------------
 * Learned rank predictor.  No counterpart in the paper: the paper finds the rank k of each
 * segment's ID adaptively (Sec. 4.2.3, sketch size h = k + p with p = 5 and k unknown until
 * the ID is done).  A 16 -> 64 (ReLU) -> 2 network predicts log2(1 + k) and log2 of the
 * one-pass sketch size from 16 features of the segment; the factorization then sketches
 * once with that size and keeps the ID only if k <= h - p and the measured error
 * ||B_r - B_s T||_F <= 10 eps ||B||_F holds on the exact B, else it continues with the
 * adaptive doubling.  Features, targets and rules are fixed as follows (row layouts are
 * float32, row-major):
 *   features  0 L - l, 1 log2 e, 2 log2(1 + neighbours), 3 near neighbours,
 *             4 log2(1 + far neighbours), 5-7 min - mean, max - mean, std of log|A_uu| over
 *             the segment's nodes u, 8 mean log(|A_uu| / sum_{j!=u} |A_uj|), 9 mean
 *             |row sum| / |A_uu|, 10 mean relative asymmetry of the row's off-diagonal
 *             entries, 11-15 log10 of |R_jj| / |R_00| (j = 1, 2, 3, 5, 7, floored at
 *             1e-16) minus log10 eps, from the column-pivoted QR of an 8-row probe sketch
 *             (the first 8 rows of the sketch matrix) of the far rows;
 *   targets   y0 = log2(1 + k), y1 = log2(min(far rows, k + p));
 *   sketch    h = max(ceil(2^o1 (1 + margin)), ceil((2^o0 - 1)(1 + margin)) + p), clamped
 *             to [1, min(far rows, max(h0, 2 (e + p)))];
 *   applies   to segments whose far rows exceed max(h0, 8), with e + p > 2 h0 and e <= 128
 *             (a segment with e + p <= 2 h0 is sketched once with h = 2 h0 whatever the
 *             mode: its rank is at most e <= h - p).
 * Parameter vector (float32, SPALU_PRED_NPARAM): W1 (64 x 16 row-major) | b1 (64) |
 * W2 (2 x 64) | b2 (2).  Inference rounds the standardised features, the parameters and
 * the hidden activations to bfloat16 and accumulates in float32. */
#define SPALU_PRED_NFEAT 16
#define SPALU_PRED_NPARAM 1218

/* Create a predictor from host parameters (copied); standardisation starts as mean 0,
 * scale 1.  Errors: SPALU_ERR_ARG (null), SPALU_ERR_ALLOC, SPALU_ERR_CUDA. */
spalu_status spalu_predictor_create(const float* params, spalu_predictor_t* out);
/* Copy the FP32 parameters to host memory (SPALU_PRED_NPARAM floats); synchronises. */
spalu_status spalu_predictor_get_params(spalu_predictor_t p, float* params, spalu_stream_t stream);
/* Feature standardisation z = (x - mu) * isd: set from / copy to host arrays of 16 floats. */
spalu_status spalu_predictor_set_norm(spalu_predictor_t p, const float* mu, const float* isd,
                                      spalu_stream_t stream);
spalu_status spalu_predictor_get_norm(spalu_predictor_t p, float* mu, float* isd, spalu_stream_t stream);
/* Fit the standardisation on device rows X (n x 16): mu = column means, isd = 1 / population
 * standard deviation (1 where it is below 1e-6). */
spalu_status spalu_predictor_fit_norm(spalu_predictor_t p, const float* X, int n, spalu_stream_t stream);
/* FP32 loss sum (o - y)^2 / (2n) over device rows X (n x 16), Y (n x 2) and its gradient
 * (host, SPALU_PRED_NPARAM floats, may be NULL); synchronises. */
spalu_status spalu_predictor_loss_grad(spalu_predictor_t p, const float* X, const float* Y, int n,
                                       float* loss, float* grad, spalu_stream_t stream);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) over consecutive batches of
 * `batch` rows, `epochs` times, on the device; the step count and moments persist in the
 * handle across calls.  One epoch is captured once as a CUDA graph and replayed.  loss
 * (host, may be NULL) receives the loss of the trained parameters over all rows, which
 * synchronises the stream.  X and Y must stay valid and unchanged between calls that reuse
 * them. */
spalu_status spalu_predictor_train(spalu_predictor_t p, const float* X, const float* Y, int n, int epochs,
                                   int batch, float lr, float* loss, spalu_stream_t stream);
/* BF16 inference of device rows X (n x 16) into device out (n x 2). */
spalu_status spalu_predictor_infer(spalu_predictor_t p, const float* X, int n, float* out,
                                   spalu_stream_t stream);
void spalu_predictor_destroy(spalu_predictor_t p);

/* Predictor mode of the next factorizations of f: 0 off (adaptive ID), 1 record (adaptive ID;
 * the features and ranks of the segments it applies to are kept for
 * spalu_factor_export_training), 2 predict (one-pass sketch from p with the given margin,
 * adaptive fallback).  p must outlive its use by f.  Errors: SPALU_ERR_ARG. */
spalu_status spalu_factor_set_predictor(spalu_factor_t f, spalu_predictor_t p, int mode, double margin);
/* Rows recorded by the last factorization (mode 1), levels L..1, segments in id order:
 * features into device X (cap x 16), targets into device Y (cap x 2); *n_out receives the
 * number of rows recorded (rows beyond cap are not written).  SPALU_ERR_STATE when the last
 * factorization did not record. */
spalu_status spalu_factor_export_training(spalu_factor_t f, float* X, float* Y, int cap, int* n_out,
                                          spalu_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPALU_H */
