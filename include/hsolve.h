/*
 * hsolve.h -- C-ABI of the GB300 hierarchical sparse solver.
 *
 * The library computes the approximate factorization of Sec. 2 of
 * "A distributed-memory hierarchical solver for general sparse linear systems"
 * (Chen, Pouransari, Rajamanickam, Boman, Darve): clusters of unknowns are
 * processed level by level; at each cluster the fill-in block is compressed
 * (Eq. lra), the sparsification operator (Eq. scaling) splits the cluster into
 * fine and coarse unknowns, the elimination operator (Eq. elim) removes the
 * fine ones, and the coarse unknowns of sibling clusters form the next level
 * (Alg. 1).  The factorization is applied by the forward/backward substitution
 * of Alg. 2 and used as a preconditioner for CG or GMRES (Sec. 5).
 *
 * Everything runs on one CUDA device.  All entry points return an
 * hsolve_status; none aborts, traps or prints.  A handle is used by one host
 * thread at a time; distinct handles are independent.  Device work is
 * enqueued on the stream given to hsolve_analyze (NULL = legacy default
 * stream); calls return after that work has completed unless stated
 * otherwise.
 *
 * Matrix input: CSR with int64 row pointers, int32 column indices and float64
 * values, host memory, square n x n.  Vector blocks: column-major n x nrhs
 * with leading dimension ld >= n, float64.
 */
#ifndef HSOLVE_H
#define HSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSOLVE_OK = 0,
  HSOLVE_ERR_ARG = -1,            /* invalid argument (sizes, pointers, CSR) */
  HSOLVE_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  HSOLVE_ERR_OOM = -3,            /* device allocation failed */
  HSOLVE_ERR_SINGULAR = -4,       /* zero pivot in an LU factor */
  HSOLVE_ERR_NOT_SPD = -5,        /* Cholesky met a non-positive pivot */
  HSOLVE_ERR_NO_CONVERGENCE = -6, /* Krylov solve hit maxit */
  HSOLVE_ERR_BUDGET = -7,         /* request above a memory budget */
  HSOLVE_ERR_TIMEOUT = -8,        /* a bounded device wait gave up */
  HSOLVE_ERR_STATE = -9           /* call out of order (e.g. apply before factor) */
} hsolve_status;

typedef enum {
  HSOLVE_FP64 = 0,        /* every factor block and product in float64 */
  HSOLVE_MIXED_FP32 = 1,  /* float32 blocks and float32 SIMT products, except
                             the dense top: a recursive Cholesky whose
                             products run on tcgen05 tensor cores as 3xTF32
                             (float32-level accuracy); float64 rank
                             decision, float64 outer Krylov */
  HSOLVE_MIXED_TF32 = 2,  /* as MIXED_FP32, with the Schur-complement products
                             (Eq. elim) on tcgen05 tensor cores, TF32
                             operands and float32 accumulation */
  HSOLVE_MIXED_BF16 = 3,  /* as MIXED_TF32 with BF16 Schur operands */
  HSOLVE_MIXED_3XTF32 = 4 /* as MIXED_TF32 with 3xTF32 Schur products (each
                             operand split into TF32 hi + lo: float32-level
                             accuracy on the tensor cores) */
} hsolve_precision;

typedef enum { HSOLVE_PCG = 0, HSOLVE_GMRES = 1 } hsolve_krylov;

typedef struct {
  int64_t n;              /* rows = columns */
  int64_t nnz;
  const int64_t* rowptr;  /* [n+1], rowptr[0] = 0, non-decreasing */
  const int32_t* col;     /* [nnz], each in [0, n) */
  const double* val;      /* [nnz] */
} hsolve_csr;

typedef struct {
  int32_t leaf_size;      /* cluster size at level 0 (bisection stops at or
                             below it); default 128 */
  int32_t symmetric;      /* -1 = detect (exact value symmetry), 0 = general
                             (LU, two-sided compression), 1 = SPD (Cholesky) */
  int64_t top_size;       /* factor a level densely once it holds at most
                             this many unknowns (0 = only when one cluster
                             is left): blocked Cholesky (SPD) or blocked LU
                             with partial pivoting (general).  hsolve_factor
                             rejects (HSOLVE_ERR_ARG) a value above the
                             dense-top limit: 24,576 unknowns in fp64 and
                             49,152 in the float32 modes (one slot vector of
                             the sweeps in shared memory), and for a general
                             matrix also 24,816 (the first LU panel in one
                             16-CTA thread-block cluster); default 0 */
  int32_t max_rank;       /* > 0: cap every compression rank at this value
                             (the fixed-rank option of Sec. 5.1); 0 = none */
  int32_t gmres_restart;  /* GMRES restart length; default 50 */
  int32_t compress;       /* 0 = pivoted QR of the fill block itself (Eq. lra);
                             1 = randomized: when the fill block has more than
                             m + 8 columns, pivoted QR of its sketch G Omega
                             (m x (m + 8), Rademacher Omega); default 0 */
  int32_t cluster_qr;     /* 1 = run the pivoted QR of the fill blocks on
                             thread-block clusters (distributed shared
                             memory); 0 = one CTA per cluster; same result
                             either way; default 1 */
  int32_t equilibrate;    /* 1 = factor S A S with S = diag(|a_ii|)^{-1/2}
                             (1 where a_ii = 0) and apply M^{-1} = S Mh^{-1} S,
                             Mh the factorization of S A S; keeps truncation
                             from losing definiteness on coefficient contrasts
                             of 1e6 (Sec. 5.1 workloads); the Krylov methods
                             still solve A x = b.  0 = factor A itself;
                             default 0 */
} hsolve_opts;

typedef struct {
  int32_t iterations;     /* Krylov iterations of the slowest right-hand side */
  double rel_residual;    /* max over right-hand sides of ||b - A x|| / ||b|| */
  double factor_ms;       /* device time of the last hsolve_factor */
  double solve_ms;        /* device time of this solve */
} hsolve_solve_info;

typedef struct {
  int32_t levels;         /* levels factored (the dense top counts as one) */
  int32_t clusters0;      /* clusters at level 0 */
  int32_t colours_total;  /* sum over levels of colour classes */
  int32_t top_size;       /* unknowns in the dense top factor (0: none) */
  int64_t coarse_total;   /* sum over levels of coarse unknowns kept */
  int64_t factor_bytes;   /* device bytes held by the factorization */
  int64_t block_bytes;    /* device bytes of the largest level's blocks */
  int64_t apply_bytes;    /* algorithmic bytes one apply reads and writes
                             (operators once, vectors as touched), nrhs = 1 */
  double factor_flops;    /* algorithmic flops of the last factorization */
  double schur_flops;     /* of which Schur-complement products (Eq. elim) */
  double prep_flops;      /* of which per-cluster dense work (factor of
                             A_ss, pivoted QR, complement, T, F) */
  double gemm_flops;      /* of which coarse-row / fine-factor products
                             T' A_sN and coarse-to-far products C U^T A_sw */
  int32_t kernel_launches;/* kernels launched by the last hsolve_factor */
  int32_t precision;      /* hsolve_precision of the last factor */
  int64_t launches_total; /* kernels launched by the library in this process */
  double qr_flops;        /* of prep_flops: the pivoted QR of the fill blocks,
                             4 m c k per cluster (c = nonzero fill columns
                             where the count pass ran, else all gathered
                             columns; k = rank) */
} hsolve_stats;

typedef struct hsolve_handle hsolve_handle;

/* Default options. */
void hsolve_default_opts(hsolve_opts* opts);

/* Analysis (Alg. 1, partition step; Eq. quotient; Sec. 3.2 independence
 * rule).  Validates the CSR, builds the bisection clusters from coords
 * (n x dim, row-major, host; NULL = bisection of the index order), the block
 * pattern of every level and the distance-2 colouring, and uploads the matrix
 * into device blocks.  The caller keeps ownership of A and coords; the library
 * copies what it needs.  cuda_stream is a cudaStream_t (NULL = default
 * stream).  On success *out is a new handle the caller releases with
 * hsolve_destroy.  Errors: HSOLVE_ERR_ARG for malformed input (out of range
 * column, non-monotone rowptr, dim not in 1..3), HSOLVE_ERR_OOM,
 * HSOLVE_ERR_CUDA. */
hsolve_status hsolve_analyze(const hsolve_csr* A, const double* coords, int dim,
                             const hsolve_opts* opts, void* cuda_stream,
                             hsolve_handle** out);

/* Factorization (Alg. 1 with LowRank_Elimination: Eqs. lra, scaling, elim,
 * perm).  eps is the relative compression tolerance of Eq. lra (|r_jj| <=
 * eps |r_11| stops the pivoted QR; 0 keeps every nonzero direction, i.e. a
 * direct solver).  May be called again on the same analysis with another eps
 * or precision; the previous factorization is released first.  Once a level
 * holds at most opts.top_size unknowns (or one cluster is left) it is
 * factored densely: Cholesky for an SPD matrix, LU with partial pivoting
 * otherwise (Alg. 1's "small enough", Sec. 6).  Errors: HSOLVE_ERR_ARG for a
 * bad eps or precision, or a top_size above the dense-top limit (see
 * hsolve_opts.top_size); HSOLVE_ERR_NOT_SPD / HSOLVE_ERR_SINGULAR (pivot
 * failure in a cluster or the dense top; the handle then holds no
 * factorization), HSOLVE_ERR_OOM, HSOLVE_ERR_CUDA. */
hsolve_status hsolve_factor(hsolve_handle* h, double eps, hsolve_precision prec);

/* Test entry point: hsolve_factor with the rank of every cluster fixed in
 * advance (Eq. lra keeps exactly that many pivoted-QR directions, fewer only
 * where the fill block has no more nonzero ones; neither eps nor the
 * rounding-noise floor plays a part), and optionally the pivot order of every
 * cluster's pivoted QR too, so that a float32 factorization can be compared
 * block by block with a float64 reference at identical ranks and pivots (a
 * float32 search can legitimately break near-ties of the column norms the
 * other way, which changes the basis U).  ranks: the per-cluster ranks of
 * levels 0..nlevels-1 concatenated (clusters in index order); counts[l]:
 * clusters of level l, which must equal the level's cluster count
 * (HSOLVE_ERR_ARG otherwise).  pivots (may be NULL = search as usual): for
 * every level and cluster in the same order, ranks[s] column indices in the
 * numbering of hsolve_export_level's pivot array.  Levels beyond nlevels (and
 * the dense top) are factored as usual with eps = 0.  Host pointers; copied. */
hsolve_status hsolve_factor_forced(hsolve_handle* h, hsolve_precision prec,
                                   const int32_t* ranks, const int32_t* counts,
                                   int32_t nlevels, const int32_t* pivots);

/* Preconditioner application (Alg. 2): out = M^{-1} rhs where M is the
 * factorization.  rhs and out are DEVICE pointers, column-major n x nrhs with
 * leading dimension ld; they may alias.  Errors: HSOLVE_ERR_STATE before a
 * successful hsolve_factor, HSOLVE_ERR_ARG for nrhs < 1 or ld < n. */
hsolve_status hsolve_apply(hsolve_handle* h, const double* rhs, double* out,
                           int nrhs, int64_t ld);

/* Bytes of the fixed device scratch behind hsolve_apply_noalloc. */
#define HSOLVE_NOALLOC_SCRATCH_BYTES 33554432

/* The same out = M^{-1} rhs as hsolve_apply, for callers that cannot let the
 * library allocate device memory: no cudaMalloc, cudaFree or other
 * allocating call is made.  (The paper has no counterpart; this is a service
 * of the library.)  Callers this is for: code whose device memory belongs to
 * another allocator (a framework's caching allocator, a pre-reserved pool)
 * and code that must not incur the device synchronisation cudaMalloc and
 * cudaFree can imply.  The factorization made by hsolve_factor is an input;
 * every temporary vector of the sweeps comes from one file-scope device
 * array of HSOLVE_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until the process exits.
 * - The first call on a device looks up that array's device address (with
 *   the device current) and caches it; make that first call before any
 *   stream capture.  The CUDA runtime may also load the library's kernels
 *   into device memory on their first launch (lazy module loading), which
 *   the library does not control; after that, calls leave the device's
 *   free memory unchanged.
 * - All calls share the array and it keeps the last call's contents; calls
 *   whose device work overlaps in time (other streams, other handles) race
 *   on it, so serialise them.
 * - A factorization and nrhs needing more scratch than the array holds are
 *   rejected with HSOLVE_ERR_BUDGET (hsolve_last_error gives both sizes).
 * Other errors as hsolve_apply.  rhs and out are device pointers
 * (column-major n x nrhs, leading dimension ld). */
hsolve_status hsolve_apply_noalloc(hsolve_handle* h, const double* rhs, double* out,
                                   int nrhs, int64_t ld);

/* Krylov solve of A x = b with the factorization as preconditioner (Sec. 5:
 * CG for SPD matrices, right-preconditioned flexible GMRES otherwise), in
 * float64, starting from x = 0, until ||b - A x|| <= tol ||b|| for every
 * right-hand side or maxit iterations.  b and x are DEVICE pointers
 * (column-major n x nrhs, leading dimension ld).  info may be NULL.
 * Errors: HSOLVE_ERR_STATE, HSOLVE_ERR_ARG, HSOLVE_ERR_NO_CONVERGENCE (x
 * then holds the last iterate). */
hsolve_status hsolve_solve(hsolve_handle* h, hsolve_krylov krylov, double tol,
                           int maxit, const double* b, double* x, int nrhs,
                           int64_t ld, hsolve_solve_info* info);

/* Same as hsolve_solve with b and x in HOST memory: the copies to and from
 * the device are part of the call. */
hsolve_status hsolve_solve_host(hsolve_handle* h, hsolve_krylov krylov,
                                double tol, int maxit, const double* b,
                                double* x, int nrhs, int64_t ld,
                                hsolve_solve_info* info);

/* Sparse matrix-vector product y = A x with the analysed matrix, float64,
 * device pointers (column-major n x nrhs, leading dimension ld). */
hsolve_status hsolve_spmv(hsolve_handle* h, const double* x, double* y,
                          int nrhs, int64_t ld);

/* The tensor-core product behind the MIXED_TF32 / MIXED_BF16 dense top,
 * exported so that it can be tested and profiled on its own (the paper has
 * no counterpart; it is a building block of the factorization's dense
 * steps).  C = beta C + alpha A B^T on DEVICE float32 buffers: A is M x K
 * with element (r, k) at A[r * rsa + k * csa], B is N x K with element
 * (n, k) at B[n * rsb + k * csb], C is M x N column-major with leading
 * dimension ldc >= M.  mode 0 = TF32 operands (rounded to nearest), 1 =
 * 3xTF32 (each operand split into TF32 hi + lo, three products), 2 = BF16
 * operands; accumulation in float32 tensor memory (tcgen05).  lower != 0
 * writes only elements with row >= column.  Synchronises the stream.
 * Errors: HSOLVE_ERR_ARG, HSOLVE_ERR_TIMEOUT (a bounded wait of the kernel
 * expired), HSOLVE_ERR_CUDA. */
hsolve_status hsolve_tc_gemm(int mode, int M, int N, int K, const float* A,
                             int64_t rsa, int64_t csa, const float* B,
                             int64_t rsb, int64_t csb, float* C, int64_t ldc,
                             float alpha, float beta, int lower, void* stream);

/* Diagnostic of the library's bounded device waits (the paper has no
 * counterpart: every wait of the library's kernels gives up after about a
 * second and reports HSOLVE_ERR_TIMEOUT instead of hanging).  Runs one wait
 * of the given kind with a limit of limit_cycles SM clocks on something that
 * nothing signals -- kind 0: the mbarrier wait of the tensor-core kernels
 * (the only kind) -- and returns the status the kernel recorded:
 * HSOLVE_ERR_TIMEOUT when the wait gave up as designed.  The device stays
 * usable afterwards.  stream: a cudaStream_t (NULL = default stream).
 * Errors: HSOLVE_ERR_ARG (another kind, negative limit), HSOLVE_ERR_OOM,
 * HSOLVE_ERR_CUDA. */
hsolve_status hsolve_wait_selftest(int kind, int64_t limit_cycles, void* stream);

/* ---- Serving runtime (a request loop over the solver; the paper has no
 * counterpart: it is the service form of factoring once and solving many
 * right-hand sides).  Worker threads take the oldest queued request whose
 * matrix is idle, batch every queued request of that matrix behind it (up to
 * max_batch_rhs columns), make the matrix's factorization resident if needed
 * (analysis + factorization on the matrix's own CUDA stream, evicting least
 * recently used idle factorizations while the resident bytes would exceed
 * memory_budget) and solve the batch with one hsolve_solve call (one
 * host-to-device copy of the batch, one copy back).
 * Requests of different matrices run on different workers at once. */
typedef struct hsolve_server hsolve_server;

typedef struct {
  int64_t memory_budget;  /* device bytes resident factorizations may hold
                             (factors + largest level's blocks); a request
                             whose matrix does not fit waits until busy ones
                             finish (it runs alone if nothing else is
                             resident); 0 = no limit; default 60 GiB */
  int32_t max_batch_rhs;  /* most right-hand sides per batched solve (one
                             request is never split); default 256 */
  int32_t workers;        /* concurrent batches (threads); default 4 */
} hsolve_server_opts;

typedef struct {
  int32_t status;         /* hsolve_status of the request's batch */
  int32_t iterations;     /* Krylov iterations of the batch */
  double rel_residual;    /* max relative residual over the batch */
  double queue_ms;        /* submit -> batch start */
  double service_ms;      /* batch start -> done (factorization included) */
  double latency_ms;      /* submit -> done */
  int32_t batch_rhs;      /* right-hand sides solved together */
  int32_t factored;       /* 1: the batch factored the matrix first */
  char message[128];      /* the library's error text when status != OK */
} hsolve_server_result;

typedef struct {
  int64_t requests_submitted, requests_done, rhs_done, batches;
  int64_t factorizations, evictions;
  int64_t resident, resident_bytes, peak_resident_bytes, queued;
} hsolve_server_stats;

void hsolve_server_default_opts(hsolve_server_opts* opts);

/* Start the workers (opts NULL = defaults).  Errors: HSOLVE_ERR_ARG. */
hsolve_status hsolve_server_create(const hsolve_server_opts* opts,
                                   hsolve_server** out);

/* Register a matrix (host CSR and coordinates are copied; no device work
 * until its first request) with the solver settings every request of it
 * uses.  *matrix_id receives its id. */
hsolve_status hsolve_server_add_matrix(hsolve_server* s, const hsolve_csr* A,
                                       const double* coords, int dim,
                                       const hsolve_opts* opts, double eps,
                                       hsolve_precision prec,
                                       hsolve_krylov krylov, double tol,
                                       int maxit, int32_t* matrix_id);

/* Queue a request: nrhs HOST right-hand sides, column-major with leading
 * dimension ld >= n (copied).  Returns at once with *request_id. */
hsolve_status hsolve_server_submit(hsolve_server* s, int32_t matrix_id,
                                   const double* b, int32_t nrhs, int64_t ld,
                                   int64_t* request_id);

/* Wait up to timeout_s seconds for a request; on completion copy its
 * solution to x (HOST, leading dimension ld; may be NULL), its record to res
 * (may be NULL), forget the request and return its status.  Errors:
 * HSOLVE_ERR_TIMEOUT (still pending; wait again), HSOLVE_ERR_ARG (unknown
 * id). */
hsolve_status hsolve_server_wait(hsolve_server* s, int64_t request_id,
                                 double* x, int64_t ld,
                                 hsolve_server_result* res, double timeout_s);

hsolve_status hsolve_server_get_stats(hsolve_server* s,
                                      hsolve_server_stats* out);

/* Stop the workers (queued requests are dropped; running batches finish)
 * and release every factorization. */
void hsolve_server_destroy(hsolve_server* s);

/* Statistics of the analysis and the last factorization. */
hsolve_status hsolve_get_stats(const hsolve_handle* h, hsolve_stats* out);

/* Per-level detail, for tests and reports.  Copies up to cap entries of the
 * ranks (coarse unknowns kept) of level `level`'s clusters into ranks (host),
 * and writes the number of clusters of that level to *nclu.  Levels are
 * numbered from 0 (leaves); the dense top level reports zeros. */
hsolve_status hsolve_get_level(const hsolve_handle* h, int level, int32_t* nclu,
                               int32_t* sizes, int32_t* ranks, int32_t* colour,
                               int32_t cap);

/* ---- Export of a factored level (for parity tests against a reference
 * implementation of Alg. 1).  For every cluster s processed at the level,
 * the factorization keeps (Sec. 2.1, Eqs. lra, scaling, elim):
 *   T'  = [U^T A_ss^{-1}; L_F^{-1} P_F V_L^T A_ss^{-1}]   (m x m)
 *         the sparsification rows with the inverse factor of the fine block
 *         F = V_L^T A_ss^{-1} V_R folded into the fine ones; with k = 0
 *         (no fill kept) T' = L^{-1} P of A_ss = P^T L U (L^{-1} for SPD);
 *         for the dense top T' = L^{-1} of its Cholesky factor;
 *   T'_R^T (general only) = [U^T A_ss^{-T}; U_F^{-T} V_R^T A_ss^{-T}];
 *   Y   = T' A_sN (m x nw): rows 0..k are the cluster's new coarse rows
 *         U^T A_ss^{-1} A_sN, rows k..m are B_R = L_F^{-1} P_F V_L^T A_ss^{-1} A_sN;
 *   X^T (general only) = T'_R^T A_Ns^T: rows k..m are B_L^T;
 * where N are the cluster's neighbours (ascending id, width = their current
 * unknowns) and U the first k directions of the column-pivoted QR of its fill
 * block.  The pivot order of that QR is kept too: entry j is the column
 * chosen at step j, counted among the nonzero columns of the gathered fill
 * block [A_sw] (SPD) or [A_sw, A_ws^T] (general) with w ascending (among
 * the sketch columns for the randomized variant). */
typedef struct {
  int32_t m;          /* unknowns when processed; 0: not processed here */
  int32_t k;          /* coarse unknowns kept (the rank of Eq. lra) */
  int32_t nw;         /* columns of Y: sum of the neighbours' widths */
  int32_t nnb;        /* neighbours */
  int32_t colour;     /* colour class; clusters run in (colour, id) order */
  int32_t npiv;       /* pivots recorded (= k) */
  int64_t T;          /* offset of T' in the exported factor array, or -1
                         (not processed, or k = m: the cluster is untouched) */
  int64_t TR;         /* offset of T'_R^T (general), else -1 */
  int64_t Y;          /* offset of Y (column-major, ld m), or -1 */
  int64_t XT;         /* offset of X^T (general, ld m), else -1 */
  int64_t piv;        /* offset of the pivots in the pivot array */
  int64_t nb;         /* offset of the neighbours in nbr_id / nbr_w */
} hsolve_cluster_export;

typedef struct {
  int32_t nclu;       /* clusters of the level */
  int32_t dense_top;  /* 1: the level is the dense top (one cluster) */
  int32_t symmetric;  /* 1: SPD path (Cholesky, one-sided operators) */
  int32_t precision;  /* hsolve_precision of the stored blocks */
  int64_t fac_elems;  /* elements of the factor array */
  int64_t piv_total;  /* entries of the pivot array */
  int64_t nbr_total;  /* entries of nbr_id / nbr_w */
} hsolve_level_export;

/* Export level `level` (0 = leaves) of the current factorization: sizes into
 * *info (required), and, where the pointer is not NULL, nclu cluster
 * records, the factor array (fac_elems entries, converted to float64), the
 * pivots (piv_total) and the neighbour ids and widths (nbr_total each).  All
 * pointers are HOST memory owned by the caller; call once with NULLs to learn
 * the sizes.  A level that only merged clusters into the dense top reports
 * nclu clusters that were not processed.  Errors: HSOLVE_ERR_ARG (level out
 * of range), HSOLVE_ERR_STATE (no factorization), HSOLVE_ERR_CUDA. */
hsolve_status hsolve_export_level(const hsolve_handle* h, int level, hsolve_level_export* info,
                                  hsolve_cluster_export* clusters, double* fac,
                                  int32_t* pivots, int32_t* nbr_id, int32_t* nbr_w);

/* One cluster of hsolve_export_level without copying the whole level: its
 * record into *rec (offsets relative to this cluster's own arrays: T and TR
 * at 0, Y and XT at 0 when present, -1 when absent; piv and nb at 0) and,
 * where the pointer is not NULL, its blocks converted to float64 into
 * caller-owned HOST arrays -- T (m x m), TRt (m x m, general only), Y
 * (m x nw), XT (m x nw, general only), all column-major with leading
 * dimension m -- its pivots (k entries) and neighbours (nnb ids and widths).
 * Call with NULL arrays first to learn m, nw, k and nnb.  Errors:
 * HSOLVE_ERR_ARG (level or cluster out of range), HSOLVE_ERR_STATE,
 * HSOLVE_ERR_CUDA. */
hsolve_status hsolve_export_cluster(const hsolve_handle* h, int level, int cluster,
                                    hsolve_cluster_export* rec, double* T, double* TRt,
                                    double* Y, double* XT, int32_t* pivots, int32_t* nbr_id,
                                    int32_t* nbr_w);

/* Level-0 cluster of every unknown: perm[p] = global index of the unknown at
 * position p of the cluster-ordered vector (host array of n entries). */
hsolve_status hsolve_get_perm(const hsolve_handle* h, int64_t* perm);

/* Kernel timing of the last factor/apply/solve: per phase name, total device
 * milliseconds and launch count.  Writes up to cap entries; *count = number
 * of phases. */
typedef struct {
  char name[24];
  double ms;
  int32_t launches;
} hsolve_phase_time;
hsolve_status hsolve_get_phase_times(const hsolve_handle* h,
                                     hsolve_phase_time* out, int32_t cap,
                                     int32_t* count);

/* Enable (1) or disable (0) per-phase CUDA-event timing (off by default; it
 * adds a synchronisation per phase); 2 also splits every phase by level
 * (names "<phase>.L<level>"); 3 records the event pairs without any
 * synchronisation and resolves them when hsolve_get_phase_times is called
 * (timing inside a measured region).  The times of a factorization replace
 * those of the previous one; solves add to them. */
hsolve_status hsolve_set_profiling(hsolve_handle* h, int on);

/* Text of the last error on this handle (never NULL). */
const char* hsolve_last_error(const hsolve_handle* h);

/* Release the handle and all device memory it owns.  NULL is a no-op. */
void hsolve_destroy(hsolve_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* HSOLVE_H */
