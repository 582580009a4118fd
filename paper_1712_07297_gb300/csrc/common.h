// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <mutex>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hsolve.h"

namespace hs {

// Kernels launched by this process through the library (all handles).
int64_t launches_total();
// One process-wide lock around device (de)allocation and CUDA-graph capture:
// an allocation's implicit synchronisation in one thread would invalidate a
// capture running in another.
std::mutex& device_mutex();
void count_launch(int n = 1);

// ---------------------------------------------------------------------------
// Device-side error word: the first failing cluster records its code and id.
// ---------------------------------------------------------------------------
struct DevError {
  int code;     // 0 = ok, else an hsolve_status value
  int cluster;  // cluster id (level-local)
  int level;
  int pad;
};

// ---------------------------------------------------------------------------
// Host analysis (analyze.cpp): clusters, patterns, colouring.
// ---------------------------------------------------------------------------
struct LevelPattern {
  int nclu = 0;
  std::vector<int> m;          // unknowns per cluster at level start
  std::vector<int> ld;         // leading dimension of cluster i's block rows
  std::vector<int64_t> voff;   // vector slot offsets (prefix sum of m)
  // Block pattern (CSR over clusters, columns ascending): self, neighbours
  // (A_B of the level) and distance-2 clusters (where fill-in can live).
  std::vector<int> ptr, col;
  std::vector<int8_t> kind;    // 0 self, 1 neighbour, 2 distance two
  std::vector<int64_t> off;    // block offset in the level arena (elements)
  int64_t arena_elems = 0;
  std::vector<int> colour;
  std::vector<std::vector<int>> classes;  // clusters of each colour, ascending
  int64_t find(int i, int j) const;       // pattern index of (i, j) or -1
};

// Recursive coordinate bisection to a uniform depth (Alg. 1 partition step).
// Returns depth; leaves holds 2^depth sorted index lists in tree order.
int rcb_leaves(int64_t n, const double* coords, int dim, int leaf,
               std::vector<std::vector<int64_t>>& leaves);

// Fill in ld, voff, the pattern (from neighbour sets), block offsets and the
// greedy distance-2 colouring.  adj[i] = sorted neighbours (excluding i).
void build_level_pattern(LevelPattern& L, const std::vector<std::vector<int>>& adj);

int round_up(int x, int a);

// ---------------------------------------------------------------------------
// Kernel launch wrappers (kernels.cu).  `real` is float or double.
// ---------------------------------------------------------------------------

// A run of gathered columns taken from one block of the level arena.  The
// gathered matrices of a cluster (its fill columns G, its neighbour columns
// A_sN, and their transposed counterparts in the general case) are lists of
// such runs; kernels resolve a gathered column index to (offset, stride).
struct Seg {
  int64_t off;    // arena offset of the block
  int colstart;   // first gathered column index of the run
  int ld;         // leading dimension of the block
  int trans;      // 0: gathered column = block column, rows contiguous;
                  // 1: gathered column = block row (stride ld)
  int pad;
};

__host__ __device__ inline void seg_col(const Seg* sg, int nseg, int j, int64_t* p, int* st) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sg[mid].colstart <= j) lo = mid;
    else hi = mid - 1;
  }
  const Seg& g = sg[lo];
  const int q = j - g.colstart;
  if (g.trans) {
    *p = g.off + q;
    *st = g.ld;
  } else {
    *p = g.off + (int64_t)q * g.ld;
    *st = 1;
  }
}

// Per-cluster task of the dense "prep" phase.
struct PrepTask {
  int s;            // level-local cluster id
  int m;            // unknowns
  int ld;           // ld of cluster s's block rows
  int ncolG;        // fill columns gathered into G
  int64_t a_ss;     // offset of block (s,s) in the arena
  int64_t gcol;     // offset of the fill-column runs (Seg list)
  int64_t ws;       // workspace offset (elements of real)
  int64_t wsd;      // workspace offset (doubles) for norms
  int64_t T;        // factor offset of T' (m x m, ld m)
  int64_t TR;       // factor offset of T'_R (general only)
  int64_t D;        // workspace offset of D = C U^T (k x m, ld m)
  int64_t D2;       // workspace offset of D2 = C^T U^T (general only)
  int l;            // > 0: pivoted QR of the sketch Y (m x l) instead of G
  int qr;           // 2: the pivoted QR was done by the cluster kernel (k in
                    // rank[s], reflectors column-major in W_G); else in-kernel
  int64_t Y;        // workspace offset of the sketch Y (ld m)
  int ngcol;        // number of fill-column runs
  int pad2;
  int64_t pv;       // offset in the level's pivot array: the column chosen at
                    // step j of the pivoted QR goes to pv + j (index among the
                    // nonzero gathered columns, or among the sketch columns)
};

// Sketch task: Y (m x l, ld m) = G Omega for the gathered fill columns of
// one cluster, Omega[q, j] = +-1/sqrt(l) (splitmix64 sign of (q << 32) | j).
struct SketchTask {
  int m, l, ncol, nseg;
  int64_t gcol;     // offset of the fill-column runs (Seg list)
  int64_t Y;        // workspace offset of Y
};

// Grouped GEMM task: C (M x N, ldc) = A (M x K, lda) * Bg, where the columns
// of Bg are the gathered columns of a Seg list.  M, N, K may be bounded by
// the device rank array: see kernels_misc.cu.
struct GemmTask {
  int s;
  int M, N, K;         // upper bounds (rows of A, columns of Bg, inner)
  int mode;            // how M/K derive from the rank k = rank[s] (see kernels_misc.cu)
  int lda, ldc;
  int nseg;            // runs of Bg
  int64_t A, C;        // offsets (A in factor or workspace arena, C in ws/factor)
  int64_t bcol;        // offset of Bg's runs (Seg list)
};

// Schur update task: C_mapped -= P^T Q with P, Q (f x nw, ld ldy) taken
// from rows k..m of Y-type factor storage.
struct SchurTask {
  int s;
  int m;            // rows of the Y storage (ld)
  int nw;           // sum of neighbour widths
  int nb;           // neighbours
  int64_t P, Q;     // factor offsets of the P/Q storages
  int64_t map;      // offset of the neighbour runs (Seg list, nb entries)
  int64_t base;     // offset into the block-base table (nb*nb entries)
  int64_t ldn;      // offset into the neighbour-ld array (nb entries)
};

// Scatter of coarse rows/columns into the blocks after a cluster step.
struct ScatterSeg {
  int s;            // cluster
  int width;        // columns of the segment
  int ld_s, ld_o;   // lds of cluster s and of the other cluster
  int64_t src;      // offset of the segment's first column in the source (rows 0..k)
  int64_t src2;     // same for the transposed side (general) or -1 for symmetric
  int ld_src;       // leading dimension of the source
  int m;            // unknowns of s (k == m means untouched: nothing to do)
  int64_t dst_row;  // block (s, o) offset: rows 0..k receive the source
  int64_t dst_col;  // block (o, s) offset: columns 0..k receive the transpose
};

struct CopyTask {   // child block -> parent block (next-level assembly)
  int rows, cols, ld_src, ld_dst;
  int64_t src, dst;
};

struct ApplyRec {   // one cluster's factor, as the substitution sweeps use it
  int m, k, nw, sym;
  int64_t voff;     // slot offset in the level vector
  int64_t T, TR;    // T' (and T'_R) offsets in the factor arena
  int64_t Y, XT;    // B_R storage (rows k..m of Y) and B_L^T storage (XT)
  int64_t map;      // offset into the vector-index map (nw entries)
  int64_t part;     // offset of the backward partial sums (per right-hand side)
};

// Diagnostic of the bounded mbarrier wait of the tensor-core kernels: waits,
// with `limit` SM clocks, on a barrier nothing arrives at and records
// HSOLVE_ERR_TIMEOUT in *err.
void mbar_wait_probe(long long limit, int* err, cudaStream_t st);

// Tensor-core products (kernels_tc.cu).  mode 0 = TF32, 1 = 3xTF32 (hi/lo
// split), 2 = BF16 operands; float32 accumulation.  C = beta C + alpha A B^T
// with A: M x K (element (r, k) at A[r * rsa + k * csa]), B: N x K likewise,
// C column-major (ldc); lower: only tiles and elements with row >= column.
void tc_gemm(int mode, int M, int N, int K, const float* A, int64_t rsa, int64_t csa,
             const float* B, int64_t rsb, int64_t csb, float* C, int64_t ldc, float alpha,
             float beta, bool lower, DevError* err, cudaStream_t st);
// Dense top on tensor cores (float32, SPD): L into A's lower triangle, X =
// L^{-1} (ld n); W: dense_top_tc_scratch(n) floats.
size_t dense_top_tc_scratch(int n);
// Schur-complement update of a colour class (the SIMT schur launch's
// arguments) with tensor-core products in the given mode.
void schur_tc(int mode, const SchurTask* tasks, int ntask, int maxnw, const float* fac,
              float* arena, const Seg* segs, const int64_t* base, const int* ldn, const int* rank,
              DevError* err, cudaStream_t st);
void dense_top_tc(float* A, int64_t lda, int n, float* X, float* W, DevError* err, int level,
                  cudaStream_t st);

template <typename real>
struct Launch {
  static void prep(const PrepTask* tasks_dev, int ntask, real* arena, real* fac,
                   real* ws, double* wsd, const Seg* segs,
                   int* rank, int* piv, const int* fpiv, double eps, int sym, int max_rank,
                   int maxm,
                   DevError* err, int level, long long* dbg, cudaStream_t st);
  // thread-block-cluster pivoted QR: cluster size for the largest task (0 =
  // does not fit), its dynamic shared memory, and the launch
  static int qr_cluster_size(int maxm, int maxc);
  static size_t qr_cluster_smem(int maxm, int maxc, int CL);
  static void count_nz(const PrepTask* tasks_dev, int ntask, int maxc, const real* arena,
                       double* wsd, const Seg* segs, int* cnt, cudaStream_t st);
  static void qr_cluster(const PrepTask* tasks_dev, int ntask, int maxm, int maxc, int CL,
                         const real* arena, real* ws, double* wsd, const Seg* segs, int* rank,
                         int* piv, const int* fpiv, const int* cnt, double eps, int max_rank,
                         cudaStream_t st);
  static void sketch(const SketchTask* tasks_dev, int ntask, int maxm, int maxl,
                     const real* arena, real* ws, const Seg* segs,
                     cudaStream_t st);
  static void gemm_gather(const GemmTask* tasks_dev, int ntask, int maxM, int maxN,
                          const real* Abase, real* Cbase, const real* Bbase,
                          const Seg* segs, const int* rank,
                          cudaStream_t st);
  static void schur(const SchurTask* tasks_dev, int ntask, int maxnw, const real* fac,
                    real* arena, const Seg* segs, const int64_t* base, const int* ldn,
                    const int* rank, cudaStream_t st);
  static void scatter(const ScatterSeg* segs_dev, int nseg, int maxw, const real* src,
                      real* arena, const int* rank, cudaStream_t st);
  static void copy_blocks(const CopyTask* tasks_dev, int ntask, const real* src, real* dst,
                          cudaStream_t st);
  static void apply_fwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                        const real* fac, const int64_t* vmap, real* y, real* z, int64_t ldy,
                        int nrhs, cudaStream_t st);
  // largest cluster the sweeps take (one slot vector in shared memory)
  static int apply_max_m();
  static void apply_bwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                        const real* fac, const int64_t* vmap, real* y, real* z, real* part,
                        int64_t ldy, int nrhs, cudaStream_t st);
  static void scatter_csr(const int64_t* dst, const double* val, int64_t nnz, real* arena,
                          cudaStream_t st);
  static void gather_vec(const int64_t* idx, int64_t n, const real* src, int64_t lds,
                         real* dst, int64_t ldd, int nrhs, cudaStream_t st);
  static void scatter_vec(const int64_t* idx, int64_t n, const real* src, int64_t lds,
                          real* dst, int64_t ldd, int nrhs, cudaStream_t st);
  // dst[p] = S[perm[p]] src[perm[p]] and dst[perm[p]] = S[perm[p]] src[p]
  // (S = null: no scaling)
  static void perm_in(const int64_t* perm, const double* S, int64_t n, const double* src,
                      int64_t lds, real* dst, int64_t ldd, int nrhs, cudaStream_t st);
  static void perm_out(const int64_t* perm, const double* S, int64_t n, const real* src,
                       int64_t lds, double* dst, int64_t ldd, int nrhs, cudaStream_t st);
  // Dense top of an SPD factorization: A (n x n, ld lda) is overwritten by
  // its Cholesky factor L; X (n x n, ld n) receives L^{-1}.  W: scratch of
  // dense_top_scratch(n) bytes.
  static size_t dense_top_scratch(int n);
  static void dense_top(real* A, int64_t lda, int n, real* X, real* W, DevError* err, int level,
                        cudaStream_t st);
  // Dense top of a general factorization: blocked LU with partial pivoting
  // of A (n x n, ld lda, overwritten by L and U), then T = L^{-1} P and
  // TRt = U^{-T} (n x n, ld n each; A = P^T L U).  scratch: lu_top_scratch(n)
  // bytes.  n at most lu_top_max() (the tall panel of the first columns
  // must fit in the shared memory of one 16-CTA thread-block cluster);
  // false above it (nothing launched) or when a panel launch fails.
  static int lu_top_max();
  static size_t lu_top_scratch(int n);
  static bool lu_top(real* A, int64_t lda, int n, real* T, real* TRt, void* scratch,
                     DevError* err, int level, cudaStream_t st);
};

// float64 Krylov helpers (kernels.cu)
// A run of consecutive vector slots: out[dst + q] = src + q for q < w.
struct VRun {
  int64_t dst, src;
  int w, pad;
};
void expand_runs(const VRun* runs, int64_t nrun, int64_t* out, cudaStream_t st);

void spmv_csr(int64_t n, const int64_t* rp, const int* ci, const double* v, const double* x,
              int64_t ldx, double* y, int64_t ldy, int nrhs, cudaStream_t st);
void dots(int64_t n, const double* a, int64_t lda, const double* b, int64_t ldb, int nrhs,
          double* out, cudaStream_t st);
// Block Krylov helpers: nv blocks V_i of n x nrhs (ld n, block stride
// n * nrhs).  out[(nv*nrhs) * kDotBlocks + i * nrhs + c] = V_i[:, c] . w[:, c]
// (partials before it); w[:, c] += sign sum_i coef[i * nrhs + c] V_i[:, c].
void block_multi_dot(int64_t n, int nv, int nrhs, const double* V, const double* w,
                     double* out, cudaStream_t st);
void block_multi_axpy(int64_t n, int nv, int nrhs, const double* V, const double* coef,
                      double sign, double* w, int64_t ldw, cudaStream_t st);
void axpby_cols(int64_t n, int nrhs, const double* alpha, const double* x, int64_t ldx,
                const double* beta, double* y, int64_t ldy, cudaStream_t st);

}  // namespace hs
