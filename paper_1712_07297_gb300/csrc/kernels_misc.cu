// Batched products, scatters and the substitution sweeps.
//
// gemm_gather  C = A * Bg for every cluster of a colour class, where the
//              columns of Bg are gathered from the cluster's blocks (the
//              neighbour coupling A_sN for Eq. scaling's coarse rows and the
//              fine-elimination factor; the fill blocks A_sw for the
//              coarse-to-far coupling C Z).
// schur        A_nn -= B_L B_R (Eq. elim): the product of a cluster's two
//              factor panels, written straight into the neighbour blocks
//              through a row/column map (clusters of a colour touch disjoint
//              blocks, so no atomics).
// scatter      coarse rows/columns of a processed cluster into its blocks.
// float64 Krylov helpers: CSR SpMV, deterministic dot products, axpy forms.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.h"

namespace hs {

static std::atomic<int64_t> g_launches{0};
int64_t launches_total() { return g_launches.load(); }
std::mutex& device_mutex() {
  static std::mutex m;
  return m;
}
void count_launch(int n) { g_launches += n; }

namespace {

constexpr int TM = 64, TN = 64, TK = 16;
constexpr int kMaxGridYZ = 65535;  // grid y/z limit: larger task lists are split

// rows of A (M), inner K and skip rule from the rank of the cluster:
//   mode 0: M = task.M, K = task.K; skip when rank == m (untouched)
//   mode 1: M = rank; skip when rank == 0 or rank == m
template <typename real>
__global__ void __launch_bounds__(256)
gemm_gather_kernel(const GemmTask* __restrict__ tasks, const real* __restrict__ Abase,
                   real* __restrict__ Cbase, const real* __restrict__ Bbase,
                   const Seg* __restrict__ segs, const int* __restrict__ rank) {
  const GemmTask tk = tasks[blockIdx.z];
  const int r = rank[tk.s];
  int M = tk.M;
  if (tk.mode == 0) {
    if (r == tk.K) return;
  } else {
    if (r == 0 || r == tk.K) return;
    M = r;
  }
  const int N = tk.N, K = tk.K;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  if (i0 >= M || j0 >= N) return;
  __shared__ real As[TK][TM + 1];
  __shared__ real Bs[TK][TN + 1];
  __shared__ int64_t cp[TN];
  __shared__ int cst[TN];
  // this tile's gathered columns: offset and stride, resolved once
  if (threadIdx.x < TN && j0 + threadIdx.x < tk.N)
    seg_col(segs + tk.bcol, tk.nseg, j0 + threadIdx.x, &cp[threadIdx.x], &cst[threadIdx.x]);
  __syncthreads();
  const real* A = Abase + tk.A;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0;
  for (int l0 = 0; l0 < K; l0 += TK) {
    // A tile: TM x TK, consecutive threads along rows
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int i = e % TM, l = e / TM;
      int gi = i0 + i, gl = l0 + l;
      As[l][i] = (gi < M && gl < K) ? A[gi + (int64_t)gl * tk.lda] : real(0);
    }
    // B tile: TK x TN, consecutive threads along the gathered column
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int l = e % TK, j = e / TK;
      int gl = l0 + l, gj = j0 + j;
      real v = 0;
      if (gl < K && gj < N) v = Bbase[cp[j] + (int64_t)gl * cst[j]];
      Bs[l][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TK; l++) {
      real a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        a[q] = As[l][ty + 16 * q];
        b[q] = Bs[l][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
  real* C = Cbase + tk.C;
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
      if (gi < M && gj < N) C[gi + (int64_t)gj * tk.ldc] = acc[p][q];
    }
}

// SplitMix64 output function (Steele, Lea, Flood 2014; Vigna's public
// domain reference implementation).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Y (m x l) = G Omega: G's columns gathered through descriptors, Omega
// generated on the fly (Rademacher, +-1/sqrt(l)); the randomized variant of
// the compression of Eq. lra.  64 x 64 output tiles, inner chunks of 16
// gathered columns.
template <typename real>
__global__ void __launch_bounds__(256)
sketch_kernel(const SketchTask* __restrict__ tasks, const real* __restrict__ arena,
              real* __restrict__ ws, const Seg* __restrict__ segs) {
  const SketchTask tk = tasks[blockIdx.z];
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  if (i0 >= tk.m || j0 >= tk.l) return;
  __shared__ real As[TK][TM + 1];
  __shared__ real Bs[TK][TN + 1];
  const real scale = real(1) / sqrt((real)tk.l);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0;
  __shared__ int64_t cp[TK];
  __shared__ int cst[TK];
  for (int q0 = 0; q0 < tk.ncol; q0 += TK) {
    if (threadIdx.x < TK && q0 + threadIdx.x < tk.ncol)
      seg_col(segs + tk.gcol, tk.nseg, q0 + threadIdx.x, &cp[threadIdx.x], &cst[threadIdx.x]);
    __syncthreads();
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int i = e % TM, l = e / TM;
      int gi = i0 + i, q = q0 + l;
      real v = 0;
      if (gi < tk.m && q < tk.ncol) v = arena[cp[l] + (int64_t)gi * cst[l]];
      As[l][i] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int l = e % TK, j = e / TK;
      int q = q0 + l, gj = j0 + j;
      real v = 0;
      if (q < tk.ncol && gj < tk.l) {
        uint64_t z = splitmix64(((uint64_t)q << 32) | (uint64_t)gj);
        v = (z >> 63) ? -scale : scale;
      }
      Bs[l][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TK; l++) {
      real a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        a[q] = As[l][ty + 16 * q];
        b[q] = Bs[l][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
  real* Y = ws + tk.Y;
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
      if (gi < tk.m && gj < tk.l) Y[gi + (int64_t)gj * tk.m] = acc[p][q];
    }
}

// C_mapped[r, c] -= sum_i P[k+i, r] Q[k+i, c], i < f = m - rank.  For an
// SPD factorization (P = Q) the update is symmetric: only the tiles on or
// below the diagonal compute, and each writes its elements to both (r, c)
// and (c, r) -- bitwise the values the full product would give, since
// P[., r] Q[., c] and P[., c] Q[., r] are the same products summed in the
// same order.
template <typename real>
__global__ void __launch_bounds__(256)
schur_kernel(const SchurTask* __restrict__ tasks, const real* __restrict__ fac,
             real* __restrict__ arena, const Seg* __restrict__ segs,
             const int64_t* __restrict__ base, const int* __restrict__ ldn,
             const int* __restrict__ rank) {
  const SchurTask tk = tasks[blockIdx.z];
  const int k = rank[tk.s];
  const int f = tk.m - k;
  if (f <= 0) return;
  const int N = tk.nw;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  if (i0 >= N || j0 >= N) return;
  const bool sym = tk.P == tk.Q;
  if (sym && j0 > i0) return;
  // the operand tiles, then (after the products) the output tile Cs[j][i]
  __shared__ real tile[TN * (TM + 1)];
  real(*As)[TM + 1] = reinterpret_cast<real(*)[TM + 1]>(tile);
  real(*Bs)[TN + 1] = reinterpret_cast<real(*)[TN + 1]>(tile + TK * (TM + 1));
  real(*Cs)[TM + 1] = reinterpret_cast<real(*)[TM + 1]>(tile);
  const real* P = fac + tk.P + k;
  const real* Q = fac + tk.Q + k;
  const int ld = tk.m;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0;
  for (int l0 = 0; l0 < f; l0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int l = e % TK, i = e / TK;
      int gl = l0 + l, gi = i0 + i;
      As[l][i] = (gl < f && gi < N) ? P[gl + (int64_t)gi * ld] : real(0);
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int l = e % TK, j = e / TK;
      int gl = l0 + l, gj = j0 + j;
      Bs[l][j] = (gl < f && gj < N) ? Q[gl + (int64_t)gj * ld] : real(0);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TK; l++) {
      real a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        a[q] = As[l][ty + 16 * q];
        b[q] = Bs[l][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
  // neighbour (run) and local index of every row/column of the tile: the
  // runs of a cluster's neighbour columns, one per neighbour
  __shared__ int rblk[TM], rloc[TM], cblk[TN], cloc[TN];
  const Seg* sg = segs + tk.map;
  for (int e = threadIdx.x; e < TM + TN; e += blockDim.x) {
    const int r = (e < TM) ? i0 + e : j0 + (e - TM);
    int a = 0, lr = 0;
    if (r < N) {
      int lo = 0, hi = tk.nb - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sg[mid].colstart <= r) lo = mid;
        else hi = mid - 1;
      }
      a = lo;
      lr = r - sg[lo].colstart;
    }
    if (e < TM) {
      rblk[e] = a;
      rloc[e] = lr;
    } else {
      cblk[e - TM] = a;
      cloc[e - TM] = lr;
    }
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) Cs[tx + 16 * q][ty + 16 * p] = acc[p][q];
  __syncthreads();
  // read-modify-write of the target blocks from the staged tile, consecutive
  // threads on consecutive rows of a block (column-major: contiguous)
  const int64_t* bs = base + tk.base;
  const int* ldv = ldn + tk.ldn;
  for (int e = threadIdx.x; e < TM * TN; e += blockDim.x) {
    const int ii = e % TM, jj = e / TM, gi = i0 + ii, gj = j0 + jj;
    if (gi >= N || gj >= N || (sym && gj > gi)) continue;
    const int a = rblk[ii];
    arena[bs[a * tk.nb + cblk[jj]] + rloc[ii] + (int64_t)cloc[jj] * ldv[a]] -= Cs[jj][ii];
  }
  if (!sym) return;
  // the mirror elements (c, r) of the strictly lower part: row gj of block
  // (cblk, rblk), column gi; consecutive threads on consecutive rows gj
  for (int e = threadIdx.x; e < TM * TN; e += blockDim.x) {
    const int jj = e % TN, ii = e / TN, gi = i0 + ii, gj = j0 + jj;
    if (gi >= N || gj >= gi) continue;
    const int b = cblk[jj];
    arena[bs[b * tk.nb + rblk[ii]] + cloc[jj] + (int64_t)rloc[ii] * ldv[b]] -= Cs[jj][ii];
  }
}

// One segment per (cluster, other-cluster) coupling: rows 0..k of the
// source columns go to rows 0..k of block (s, o); their transpose (or the
// second source, general case) to columns 0..k of block (o, s).
template <typename real>
__global__ void scatter_kernel(const ScatterSeg* __restrict__ segs, const real* __restrict__ src,
                               real* __restrict__ arena, const int* __restrict__ rank) {
  const ScatterSeg sg = segs[blockIdx.y];
  const int k = rank[sg.s];
  if (k == 0 || k == sg.m) return;
  const int total = k * sg.width;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int i = e % k, c = e / k;
    real v = src[sg.src + i + (int64_t)c * sg.ld_src];
    arena[sg.dst_row + i + (int64_t)c * sg.ld_s] = v;
    real v2 = (sg.src2 >= 0) ? src[sg.src2 + i + (int64_t)c * sg.ld_src] : v;
    arena[sg.dst_col + c + (int64_t)i * sg.ld_o] = v2;
  }
}

template <typename real>
__global__ void copy_blocks_kernel(const CopyTask* __restrict__ tasks, const real* __restrict__ src,
                                   real* __restrict__ dst) {
  const CopyTask t = tasks[blockIdx.y];
  const int total = t.rows * t.cols;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int i = e % t.rows, j = e / t.rows;
    dst[t.dst + i + (int64_t)j * t.ld_dst] = src[t.src + i + (int64_t)j * t.ld_src];
  }
}

template <typename real>
__global__ void scatter_csr_kernel(const int64_t* __restrict__ dst, const double* __restrict__ val,
                                   int64_t nnz, real* __restrict__ arena) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    arena[dst[e]] += (real)val[e];
}

template <typename real>
__global__ void gather_vec_kernel(const int64_t* __restrict__ idx, int64_t n,
                                  const real* __restrict__ src, int64_t lds, real* __restrict__ dst,
                                  int64_t ldd, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e % n;
    int r = (int)(e / n);
    dst[p + r * ldd] = src[idx[p] + r * lds];
  }
}

template <typename real>
__global__ void scatter_vec_kernel(const int64_t* __restrict__ idx, int64_t n,
                                   const real* __restrict__ src, int64_t lds,
                                   real* __restrict__ dst, int64_t ldd, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e % n;
    int r = (int)(e / n);
    dst[idx[p] + r * ldd] = src[p + r * lds];
  }
}

template <typename real>
__global__ void perm_in_kernel(const int64_t* __restrict__ perm, const double* __restrict__ S,
                               int64_t n, const double* __restrict__ src, int64_t lds,
                               real* __restrict__ dst, int64_t ldd, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e % n;
    int r = (int)(e / n);
    const int64_t g = perm[p];
    const double v = src[g + r * lds];
    dst[p + r * ldd] = (real)(S ? S[g] * v : v);
  }
}

template <typename real>
__global__ void perm_out_kernel(const int64_t* __restrict__ perm, const double* __restrict__ S,
                                int64_t n, const real* __restrict__ src, int64_t lds,
                                double* __restrict__ dst, int64_t ldd, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = e % n;
    int r = (int)(e / n);
    const int64_t g = perm[p];
    const double v = (double)src[p + r * lds];
    dst[g + r * ldd] = S ? S[g] * v : v;
  }
}

inline int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

// ---- float64 Krylov helpers ----------------------------------------------

__global__ void spmv_kernel(int64_t n, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ x, int64_t ldx,
                            double* __restrict__ y, int64_t ldy, int nrhs) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rp[row], e = rp[row + 1];
    for (int r = 0; r < nrhs; r++) {
      double acc = 0;
      const double* xr = x + r * ldx;
      for (int64_t p = b; p < e; p++) acc += v[p] * xr[ci[p]];
      y[row + r * ldy] = acc;
    }
  }
}

constexpr int kDotBlocks = 256;

// partial[c * kDotBlocks + b] = sum over this block's rows of
// a[:,c] * b[:, c mod bmod]
__global__ void dots_partial(int64_t n, const double* __restrict__ a, int64_t lda,
                             const double* __restrict__ b, int64_t ldb, int ncol, int bmod,
                             double* __restrict__ part) {
  __shared__ double red[256];
  for (int c = 0; c < ncol; c++) {
    const double* ac = a + c * lda;
    const double* bc = b + (int64_t)(c % bmod) * ldb;
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      s += ac[i] * bc[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[c * kDotBlocks + blockIdx.x] = red[0];
    __syncthreads();
  }
}

__global__ void dots_final(const double* __restrict__ part, int ncol, double* __restrict__ out) {
  int c = blockIdx.x;
  __shared__ double red[kDotBlocks];
  red[threadIdx.x] = part[c * kDotBlocks + threadIdx.x];
  __syncthreads();
  for (int st = kDotBlocks / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// w[:, c] += sign * sum_i coef[i * nrhs + c] V_i[:, c] for the nv blocks
// V_i (n x nrhs, ld n, block stride n * nrhs)
__global__ void block_multi_axpy_kernel(int64_t n, int nv, int nrhs, const double* __restrict__ V,
                                        const double* __restrict__ coef, double sign,
                                        double* __restrict__ w, int64_t ldw) {
  const int64_t bs = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;
    const int c = (int)(e / n);
    double acc = 0;
    for (int j = 0; j < nv; j++) acc += V[j * bs + e] * coef[j * nrhs + c];
    w[i + c * ldw] += sign * acc;
  }
}

__global__ void axpby_kernel(int64_t n, int nrhs, const double* __restrict__ alpha,
                             const double* __restrict__ x, int64_t ldx,
                             const double* __restrict__ beta, double* __restrict__ y, int64_t ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int r = (int)(e / n);
    y[i + r * ldy] = alpha[r] * x[i + r * ldx] + beta[r] * y[i + r * ldy];
  }
}

}  // namespace

template <typename real>
void Launch<real>::gemm_gather(const GemmTask* tasks_dev, int ntask, int maxM, int maxN,
                               const real* Abase, real* Cbase, const real* Bbase,
                               const Seg* segs, const int* rank,
                               cudaStream_t st) {
  if (ntask <= 0 || maxM <= 0 || maxN <= 0) return;
  for (int t0 = 0; t0 < ntask; t0 += kMaxGridYZ) {
    dim3 grid((maxN + TN - 1) / TN, (maxM + TM - 1) / TM, std::min(kMaxGridYZ, ntask - t0));
    count_launch();
    gemm_gather_kernel<real><<<grid, 256, 0, st>>>(tasks_dev + t0, Abase, Cbase, Bbase, segs,
                                                    rank);
  }
}

template <typename real>
void Launch<real>::sketch(const SketchTask* tasks_dev, int ntask, int maxm, int maxl,
                          const real* arena, real* ws, const Seg* segs, cudaStream_t st) {
  if (ntask <= 0 || maxm <= 0 || maxl <= 0) return;
  for (int t0 = 0; t0 < ntask; t0 += kMaxGridYZ) {
    dim3 grid((maxl + TN - 1) / TN, (maxm + TM - 1) / TM, std::min(kMaxGridYZ, ntask - t0));
    count_launch();
    sketch_kernel<real><<<grid, 256, 0, st>>>(tasks_dev + t0, arena, ws, segs);
  }
}

template <typename real>
void Launch<real>::schur(const SchurTask* tasks_dev, int ntask, int maxnw, const real* fac,
                         real* arena, const Seg* segs, const int64_t* base, const int* ldn,
                         const int* rank, cudaStream_t st) {
  if (ntask <= 0 || maxnw <= 0) return;
  for (int t0 = 0; t0 < ntask; t0 += kMaxGridYZ) {
    dim3 grid((maxnw + TN - 1) / TN, (maxnw + TM - 1) / TM, std::min(kMaxGridYZ, ntask - t0));
    count_launch();
    schur_kernel<real><<<grid, 256, 0, st>>>(tasks_dev + t0, fac, arena, segs, base, ldn, rank);
  }
}

template <typename real>
void Launch<real>::scatter(const ScatterSeg* segs_dev, int nseg, int maxw, const real* src,
                           real* arena, const int* rank, cudaStream_t st) {
  if (nseg <= 0) return;
  for (int t0 = 0; t0 < nseg; t0 += kMaxGridYZ) {
    dim3 grid(std::max(1, std::min(64, (maxw * 64 + 255) / 256)), std::min(kMaxGridYZ, nseg - t0));
    count_launch();
    scatter_kernel<real><<<grid, 256, 0, st>>>(segs_dev + t0, src, arena, rank);
  }
}

template <typename real>
void Launch<real>::copy_blocks(const CopyTask* tasks_dev, int ntask, const real* src, real* dst,
                               cudaStream_t st) {
  if (ntask <= 0) return;
  for (int t0 = 0; t0 < ntask; t0 += kMaxGridYZ) {
    dim3 grid(8, std::min(kMaxGridYZ, ntask - t0));
    count_launch();
    copy_blocks_kernel<real><<<grid, 256, 0, st>>>(tasks_dev + t0, src, dst);
  }
}

template <typename real>
void Launch<real>::scatter_csr(const int64_t* dst, const double* val, int64_t nnz, real* arena,
                               cudaStream_t st) {
  if (nnz <= 0) return;
  count_launch();
  scatter_csr_kernel<real><<<grid_for(nnz, 256), 256, 0, st>>>(dst, val, nnz, arena);
}

template <typename real>
void Launch<real>::gather_vec(const int64_t* idx, int64_t n, const real* src, int64_t lds,
                              real* dst, int64_t ldd, int nrhs, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  gather_vec_kernel<real><<<grid_for(n * nrhs, 256), 256, 0, st>>>(idx, n, src, lds, dst, ldd, nrhs);
}

template <typename real>
void Launch<real>::scatter_vec(const int64_t* idx, int64_t n, const real* src, int64_t lds,
                               real* dst, int64_t ldd, int nrhs, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  scatter_vec_kernel<real><<<grid_for(n * nrhs, 256), 256, 0, st>>>(idx, n, src, lds, dst, ldd, nrhs);
}

template <typename real>
void Launch<real>::perm_in(const int64_t* perm, const double* S, int64_t n, const double* src,
                           int64_t lds, real* dst, int64_t ldd, int nrhs, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  perm_in_kernel<real><<<grid_for(n * nrhs, 256), 256, 0, st>>>(perm, S, n, src, lds, dst, ldd,
                                                                  nrhs);
}

template <typename real>
void Launch<real>::perm_out(const int64_t* perm, const double* S, int64_t n, const real* src,
                            int64_t lds, double* dst, int64_t ldd, int nrhs, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  perm_out_kernel<real><<<grid_for(n * nrhs, 256), 256, 0, st>>>(perm, S, n, src, lds, dst, ldd,
                                                                   nrhs);
}


template struct Launch<double>;
template struct Launch<float>;

namespace {
__global__ void expand_runs_kernel(const VRun* __restrict__ runs, int64_t nrun,
                                   int64_t* __restrict__ out) {
  for (int64_t r = blockIdx.x; r < nrun; r += gridDim.x) {
    const VRun v = runs[r];
    for (int q = threadIdx.x; q < v.w; q += blockDim.x) out[v.dst + q] = v.src + q;
  }
}
}  // namespace

void expand_runs(const VRun* runs, int64_t nrun, int64_t* out, cudaStream_t st) {
  if (nrun <= 0) return;
  count_launch();
  expand_runs_kernel<<<(int)std::min<int64_t>(nrun, 152 * 32), 128, 0, st>>>(runs, nrun, out);
}

void spmv_csr(int64_t n, const int64_t* rp, const int* ci, const double* v, const double* x,
              int64_t ldx, double* y, int64_t ldy, int nrhs, cudaStream_t st) {
  count_launch();
  spmv_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, v, x, ldx, y, ldy, nrhs);
}

// out[c] = a[:,c] . b[:,c]; partial sums in a fixed order (deterministic).
// `out` must have room for nrhs * (kDotBlocks + 1) doubles: the first
// nrhs * kDotBlocks hold partials, results go to out[nrhs*kDotBlocks + c].
void dots(int64_t n, const double* a, int64_t lda, const double* b, int64_t ldb, int nrhs,
          double* out, cudaStream_t st) {
  count_launch();
  dots_partial<<<kDotBlocks, 256, 0, st>>>(n, a, lda, b, ldb, nrhs, nrhs, out);
  count_launch();
  dots_final<<<nrhs, kDotBlocks, 0, st>>>(out, nrhs, out + (int64_t)nrhs * kDotBlocks);
}

void block_multi_dot(int64_t n, int nv, int nrhs, const double* V, const double* w,
                     double* out, cudaStream_t st) {
  // column q = i * nrhs + c of the nv blocks is V_i[:, c] (stride n); it
  // meets w[:, c] = w[:, q mod nrhs]
  const int ncol = nv * nrhs;
  count_launch();
  dots_partial<<<kDotBlocks, 256, 0, st>>>(n, V, n, w, n, ncol, nrhs, out);
  count_launch();
  dots_final<<<ncol, kDotBlocks, 0, st>>>(out, ncol, out + (int64_t)ncol * kDotBlocks);
}

void block_multi_axpy(int64_t n, int nv, int nrhs, const double* V, const double* coef,
                      double sign, double* w, int64_t ldw, cudaStream_t st) {
  count_launch();
  block_multi_axpy_kernel<<<grid_for(n * nrhs, 256), 256, 0, st>>>(n, nv, nrhs, V, coef, sign,
                                                                    w, ldw);
}

void axpby_cols(int64_t n, int nrhs, const double* alpha, const double* x, int64_t ldx,
                const double* beta, double* y, int64_t ldy, cudaStream_t st) {
  count_launch();
  axpby_kernel<<<grid_for(n * nrhs, 256), 256, 0, st>>>(n, nrhs, alpha, x, ldx, beta, y, ldy);
}

}  // namespace hs
