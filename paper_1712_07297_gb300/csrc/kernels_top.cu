// Dense top factorization (Alg. 1: "factorize A with the conventional
// Cholesky factorization" once the remaining system is small enough), for an
// SPD top block too large for one CTA: blocked right-looking Cholesky over
// 64-column panels (one CTA factors the diagonal block, a launch of CTAs
// solves the panel, a launch updates the trailing lower triangle), then the
// explicit inverse factor X = L^{-1} by block rows (one launch per block
// row, one CTA per block column), which the substitution sweeps apply as
// dense products.  Matrices are column-major in global memory.
//
// A general (nonsymmetric) top goes through a blocked right-looking LU with
// partial pivoting instead.  Each panel of nb columns (128 bytes of a row:
// 32 float32 or 16 float64 columns) is factored by one thread-block cluster
// that holds the whole tall panel in distributed shared memory: per column
// the CTAs agree on the pivot through two cluster barriers (largest |a| over
// the remaining rows, then the lowest current row among the entries within
// 1e-10 of it, the tie rule of the one-CTA LU), and row interchanges inside
// the panel are relabellings, not copies.  Then one launch applies the
// panel's interchanges to the other columns, one solves the unit-lower
// system for the block row of U, and the trailing update is a tensor-core
// 3xTF32 product (float32) or a SIMT product (float64).  The stored
// operators follow from A = P^T L U: T' = L^{-1} P (the inverse of the unit
// lower factor, columns scattered by the row order) and T'_R^T = U^{-T},
// both by block rows as for the Cholesky top.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <cooperative_groups.h>

#include "common.h"

namespace cg = cooperative_groups;

namespace hs {

namespace {

constexpr int NB = 64;

template <typename real>
__device__ __forceinline__ real tsqrt(real x);
template <>
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }

// Cholesky of the diagonal block A[j0:j0+b, j0:j0+b] in shared memory.
template <typename real>
__global__ void __launch_bounds__(256)
potrf_diag_kernel(real* A, int64_t ld, int j0, int b, DevError* err, int level) {
  __shared__ real S[NB][NB + 1];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, j = e / b;
    S[j][i] = A[(j0 + i) + (int64_t)(j0 + j) * ld];
  }
  __syncthreads();
  for (int j = 0; j < b; j++) {
    if (threadIdx.x == 0) {
      real d = S[j][j];
      if (!(d > real(0))) bad = 1;
      else S[j][j] = tsqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const real rd = real(1) / S[j][j];
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) S[j][i] *= rd;
    __syncthreads();
    const int t = b - j - 1;
    for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
      int i = j + 1 + e % t, l = j + 1 + e / t;
      if (i >= l) S[l][i] -= S[j][i] * S[j][l];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0 && atomicCAS(&err->code, 0, (int)HSOLVE_ERR_NOT_SPD) == 0) {
      err->cluster = 0;
      err->level = level;
    }
    return;
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, j = e / b;
    A[(j0 + i) + (int64_t)(j0 + j) * ld] = (i >= j) ? S[j][i] : real(0);
  }
}

// Panel solve: rows r >= j0 + b of columns j0..j0+b: X L_jj^T = B, one CTA
// per 64-row strip, each thread a row of the strip.
template <typename real>
__global__ void __launch_bounds__(64)
trsm_panel_kernel(real* A, int64_t ld, int n, int j0, int b) {
  __shared__ real L[NB][NB + 1];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, j = e / b;
    L[j][i] = A[(j0 + i) + (int64_t)(j0 + j) * ld];
  }
  __syncthreads();
  const int r = j0 + b + blockIdx.x * NB + threadIdx.x;
  if (r >= n) return;
  real x[NB];
#pragma unroll 8
  for (int j = 0; j < NB; j++) x[j] = (j < b) ? A[r + (int64_t)(j0 + j) * ld] : real(0);
  // x L^T = rhs: x_j = (rhs_j - sum_{l<j} x_l L[j][l]) / L[j][j]
  for (int j = 0; j < b; j++) {
    real v = x[j];
    for (int l = 0; l < j; l++) v -= x[l] * L[l][j];
    x[j] = v / L[j][j];
  }
#pragma unroll 8
  for (int j = 0; j < NB; j++)
    if (j < b) A[r + (int64_t)(j0 + j) * ld] = x[j];
}

// Trailing update of the lower triangle: A[I, J] -= P_I P_J^T for 64 x 64
// tiles I >= J of the trailing block, P = A[j0+b:, j0:j0+b].
template <typename real>
__global__ void __launch_bounds__(256)
syrk_update_kernel(real* A, int64_t ld, int n, int j0, int b) {
  const int t0 = j0 + b;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;
  const int i0 = t0 + ti * NB, jc0 = t0 + tj * NB;
  if (i0 >= n || jc0 >= n) return;
  __shared__ real As[16][NB + 1];
  __shared__ real Bs[16][NB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = 0;
  for (int l0 = 0; l0 < b; l0 += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      int i = e % NB, l = e / NB;
      int gi = i0 + i, gj = jc0 + i, gl = j0 + l0 + l;
      bool okl = (l0 + l) < b;
      As[l][i] = (gi < n && okl) ? A[gi + (int64_t)gl * ld] : real(0);
      Bs[l][i] = (gj < n && okl) ? A[gj + (int64_t)gl * ld] : real(0);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; l++) {
      real a[4], c[4];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        a[p] = As[l][ty + 16 * p];
        c[p] = Bs[l][tx + 16 * p];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * c[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int gi = i0 + ty + 16 * p, gj = jc0 + tx + 16 * q;
      if (gi < n && gj < n && gi >= gj) A[gi + (int64_t)gj * ld] -= acc[p][q];
    }
}

// Block row i of X = L^{-1}: for every block column j <= i (one CTA each),
// X_ij = L_ii^{-1} (delta_ij I - sum_{k=j}^{i-1} L_ik X_kj).  Only the lower
// triangle of L is read (not its diagonal if `unit`).  Column c of X is
// stored at column cmap[c] of the output (cmap = null: c).
template <typename real>
__global__ void __launch_bounds__(256)
trtri_row_kernel(const real* L, int64_t ld, real* X, int64_t ldx, int n, int i, int unit,
                 const int* __restrict__ cmap) {
  const int j = blockIdx.x;
  const int r0 = i * NB, c0 = j * NB;
  const int br = min(NB, n - r0), bc = min(NB, n - c0);
  __shared__ real S[NB][NB + 1];   // the accumulated right-hand side, S[col][row]
  __shared__ real Ld[NB][NB + 1];  // L_ii
  __shared__ real As[16][NB + 1];
  __shared__ real Bs[16][NB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = 0;
  // acc = sum_{k=j}^{i-1} L_ik X_kj over the K range [c0, r0)
  for (int l0 = c0; l0 < r0; l0 += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      int a = e % NB, l = e / NB;
      int gl = l0 + l;
      As[l][a] = (a < br) ? L[(r0 + a) + (int64_t)gl * ld] : real(0);
      Bs[l][a] = (a < bc) ? X[gl + (int64_t)(cmap ? cmap[c0 + a] : c0 + a) * ldx] : real(0);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; l++) {
      real a[4], c[4];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        a[p] = As[l][ty + 16 * p];
        c[p] = Bs[l][tx + 16 * p];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * c[q];
    }
    __syncthreads();
  }
  // S = delta_ij I - acc
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int a = ty + 16 * p, c = tx + 16 * q;
      S[c][a] = ((i == j && a == c) ? real(1) : real(0)) - acc[p][q];
    }
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    int a = e % NB, c = e / NB;
    Ld[c][a] = (a < br && c < br) ? L[(r0 + a) + (int64_t)(r0 + c) * ld] : real(0);
  }
  __syncthreads();
  // forward substitution L_ii Y = S, one thread per column of S
  if (threadIdx.x < bc) {
    const int c = threadIdx.x;
    for (int a = 0; a < br; a++) {
      real v = S[c][a];
      for (int l = 0; l < a; l++) v -= Ld[l][a] * S[c][l];
      S[c][a] = unit ? v : v / Ld[a][a];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < br * bc; e += 256) {
    int a = e % br, c = e / br;
    X[(r0 + a) + (int64_t)(cmap ? cmap[c0 + c] : c0 + c) * ldx] = S[c][a];
  }
}

template <typename real>
__global__ void zero_upper_kernel(real* X, int64_t ldx, int n, const int* __restrict__ cmap) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % n), j = (int)(e / n);
    if (i < j) X[i + (int64_t)(cmap ? cmap[j] : j) * ldx] = 0;
  }
}

// ---- LU top

constexpr int kLuThreads = 256;
constexpr int kLuMaxCl = 16;                 // CTAs per panel cluster, at most
constexpr size_t kLuSmemCap = 200 * 1024;    // dynamic shared memory per CTA, at most
constexpr double kLuTieRtol = 1e-10;         // pivot near-ties (the one-CTA LU's rule)

template <typename real>
__host__ __device__ constexpr int lu_nb() { return (int)(128 / sizeof(real)); }

__host__ __device__ inline size_t lu_al16(size_t b) { return (b + 15) / 16 * 16; }

// Dynamic shared memory of a panel CTA holding R rows: the rows (column-major,
// ld R) and their current positions.
template <typename real>
__host__ __device__ inline size_t lu_panel_smem(int R) {
  return lu_al16((size_t)R * lu_nb<real>() * sizeof(real)) + lu_al16((size_t)R * sizeof(int));
}

struct LuXch {
  double val;  // largest local |a| in the pivot column
  int cand;    // lowest current position among the local near-maximal rows
  int slot;    // panel slot of that row
};

__device__ __forceinline__ double lu_warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ unsigned long long lu_warp_min(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
    v = x < v ? x : v;
  }
  return v;
}

// LU with partial pivoting of the panel A[j0:n, j0:j0+b] on one thread-block
// cluster: CTA cr holds panel slots [cr R, cr R + R) (slot s = panel row s at
// the launch) in shared memory, with lab[s] = the row's current position in
// the panel.  Step j: pivot = the slot of largest |a_j| among positions >= j
// (ties as in the one-CTA LU: the lowest position within 1e-10 of the
// maximum); it takes position j and the slot at position j takes the pivot's
// old position (ipiv[j0 + j] = j0 + that position, the LAPACK convention);
// the rows at positions > j are then updated with l = a_j / u_jj.  The
// pivot row is read by every CTA from its owner's shared memory; it is never
// written again.  Finally every slot is written back at its position.  All
// CTAs take the same branches (their decisions use the same exchanged
// values), so the cluster barriers always match.  A column with no nonzero
// left records HSOLVE_ERR_SINGULAR and ends the panel (the remaining ipiv
// entries are identities, so later launches stay in bounds).
template <typename real>
__global__ void __launch_bounds__(kLuThreads)
lu_panel_kernel(real* A, int64_t lda, int n, int j0, int b, int R, int* __restrict__ ipiv,
                DevError* err, int level) {
  constexpr int NBL = lu_nb<real>();
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks();
  const int cr = (int)cl.block_rank();
  const int rows = n - j0;
  const int s0 = cr * R;
  const int nloc = max(0, min(R, rows - s0));
  extern __shared__ __align__(16) unsigned char lu_smem[];
  real* Ps = reinterpret_cast<real*>(lu_smem);
  int* lab = reinterpret_cast<int*>(lu_smem + lu_al16((size_t)R * NBL * sizeof(real)));
  __shared__ LuXch xch;
  __shared__ real urow[NBL];
  __shared__ int slot_of[NBL];  // slot at positions 0..b-1
  __shared__ double red_d[kLuThreads / 32];
  __shared__ unsigned long long red_u[kLuThreads / 32];
  __shared__ double s_M;
  __shared__ int s_p, s_sp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nwarp = kLuThreads / 32;

  for (int e = threadIdx.x; e < nloc * b; e += blockDim.x) {
    const int i = e % nloc, c = e / nloc;
    Ps[i + (int64_t)c * R] = A[(j0 + s0 + i) + (int64_t)(j0 + c) * lda];
  }
  for (int i = threadIdx.x; i < nloc; i += blockDim.x) lab[i] = s0 + i;
  if (threadIdx.x < NBL) slot_of[threadIdx.x] = threadIdx.x;
  __syncthreads();

  for (int j = 0; j < b; j++) {
    // 1. largest |a_j| over the remaining rows of the cluster
    double mx = 0;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x)
      if (lab[i] >= j) mx = fmax(mx, fabs((double)Ps[i + (int64_t)j * R]));
    mx = lu_warp_max(mx);
    if (lane == 0) red_d[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_d[0];
      for (int w = 1; w < nwarp; w++) v = fmax(v, red_d[w]);
      xch.val = v;
    }
    cl.sync();
    if (warp == 0) {
      double v = (lane < CL) ? cl.map_shared_rank(&xch, lane)->val : 0.0;
      v = lu_warp_max(v);
      if (lane == 0) s_M = v;
    }
    __syncthreads();
    const double M = s_M;
    if (!(M > 0.0)) {
      if (cr == 0 && threadIdx.x == 0) {
        if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_SINGULAR) == 0) {
          err->cluster = 0;
          err->level = level;
        }
        for (int jj = j; jj < b; jj++) ipiv[j0 + jj] = j0 + jj;
      }
      break;
    }
    // 2. lowest current position among the near-maximal rows
    unsigned long long key = ~0ull;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
      const int p = lab[i];
      if (p >= j && fabs((double)Ps[i + (int64_t)j * R]) >= (1.0 - kLuTieRtol) * M) {
        const unsigned long long kk = ((unsigned long long)p << 32) | (unsigned)i;
        key = kk < key ? kk : key;
      }
    }
    key = lu_warp_min(key);
    if (lane == 0) red_u[warp] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long v = red_u[0];
      for (int w = 1; w < nwarp; w++) v = red_u[w] < v ? red_u[w] : v;
      const bool any = v != ~0ull;
      xch.cand = any ? (int)(v >> 32) : INT_MAX;
      xch.slot = any ? s0 + (int)(v & 0xffffffffu) : -1;
    }
    cl.sync();
    if (warp == 0) {
      unsigned long long v = ~0ull;
      if (lane < CL)
        v = ((unsigned long long)(unsigned)cl.map_shared_rank(&xch, lane)->cand << 8) | lane;
      v = lu_warp_min(v);
      if (lane == 0) {
        const int owner = (int)(v & 0xff);
        s_p = (int)(v >> 8);
        s_sp = cl.map_shared_rank(&xch, owner)->slot;
      }
    }
    __syncthreads();
    const int p = s_p, sp = s_sp, sj = slot_of[j];
    const int cp = sp / R;
    // 3. the pivot row, from its owner's shared memory
    if (threadIdx.x < b)
      urow[threadIdx.x] = cl.map_shared_rank(Ps, cp)[(sp - cp * R) + (int64_t)threadIdx.x * R];
    // 4. interchange positions j and p (labels only)
    if (threadIdx.x == 0) {
      if (sp >= s0 && sp < s0 + nloc) lab[sp - s0] = j;
      if (sj != sp && sj >= s0 && sj < s0 + nloc) lab[sj - s0] = p;
      slot_of[j] = sp;
      if (p < b && p != j) slot_of[p] = sj;
      if (cr == 0) ipiv[j0 + j] = j0 + p;
    }
    __syncthreads();
    // 5. multipliers and the rank-1 update of the rows below position j
    const real rd = real(1) / urow[j];
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
      if (lab[i] <= j) continue;
      const real l = Ps[i + (int64_t)j * R] * rd;
      Ps[i + (int64_t)j * R] = l;
      for (int c = j + 1; c < b; c++) Ps[i + (int64_t)c * R] -= l * urow[c];
    }
  }
  // no CTA leaves (or overwrites) while another may still read its rows
  cl.sync();
  for (int e = threadIdx.x; e < nloc * b; e += blockDim.x) {
    const int i = e % nloc, c = e / nloc;
    A[(j0 + lab[i]) + (int64_t)(j0 + c) * lda] = Ps[i + (int64_t)c * R];
  }
}

// The panel's interchanges (ipiv[j0..j0+b)) applied to every column outside
// the panel, and to the row order perm (perm[i] = original row at position
// i).  Each CTA replays the swaps on the at most 2b rows they touch (one
// thread), then one warp per column moves those rows: all loads before the
// stores.  An entry outside [j0 + j, n) is taken as no interchange.
template <typename real>
__global__ void __launch_bounds__(256)
lu_swap_kernel(real* A, int64_t lda, int n, int j0, int b, const int* __restrict__ ipiv,
               int* __restrict__ perm) {
  constexpr int NBL = lu_nb<real>();
  __shared__ int pos[2 * NBL], src[2 * NBL];
  __shared__ int nmv;
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < b; j++) {
      const int a = j0 + j, q = ipiv[j0 + j];
      if (q <= a || q >= n) continue;
      int ia = -1, iq = -1;
      for (int t = 0; t < cnt; t++) {
        if (pos[t] == a) ia = t;
        if (pos[t] == q) iq = t;
      }
      if (ia < 0) { pos[cnt] = a; src[cnt] = a; ia = cnt++; }
      if (iq < 0) { pos[cnt] = q; src[cnt] = q; iq = cnt++; }
      const int t = src[ia];
      src[ia] = src[iq];
      src[iq] = t;
    }
    nmv = cnt;
  }
  __syncthreads();
  const int cnt = nmv;
  if (cnt == 0) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  if (gw == 0) {
    int v0 = 0, v1 = 0;
    if (lane < cnt) v0 = perm[src[lane]];
    if (lane + 32 < cnt) v1 = perm[src[lane + 32]];
    __syncwarp();
    if (lane < cnt) perm[pos[lane]] = v0;
    if (lane + 32 < cnt) perm[pos[lane + 32]] = v1;
  }
  for (int w = gw; w < n - b; w += nw) {
    const int c = w < j0 ? w : w + b;
    real* col = A + (int64_t)c * lda;
    real v0 = 0, v1 = 0;
    if (lane < cnt) v0 = col[src[lane]];
    if (lane + 32 < cnt) v1 = col[src[lane + 32]];
    __syncwarp();
    if (lane < cnt) col[pos[lane]] = v0;
    if (lane + 32 < cnt) col[pos[lane + 32]] = v1;
  }
}

// Block row of U: A[j0:j0+b, c] = L11^{-1} A[j0:j0+b, c] for the columns c
// right of the panel (L11 unit lower, b x b), one thread per column.
template <typename real>
__global__ void __launch_bounds__(128)
lu_trsm_kernel(real* A, int64_t lda, int n, int j0, int b) {
  constexpr int NBL = lu_nb<real>();
  __shared__ real L[NBL][NBL + 1];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    L[j][i] = A[(j0 + i) + (int64_t)(j0 + j) * lda];
  }
  __syncthreads();
  const int c = j0 + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  real* col = A + j0 + (int64_t)c * lda;
  real x[NBL];
#pragma unroll
  for (int i = 0; i < NBL; i++) x[i] = (i < b) ? col[i] : real(0);
#pragma unroll
  for (int i = 1; i < NBL; i++) {
    real v = x[i];
#pragma unroll
    for (int l = 0; l < i; l++) v -= L[l][i] * x[l];
    x[i] = v;
  }
#pragma unroll
  for (int i = 0; i < NBL; i++)
    if (i < b) col[i] = x[i];
}

// C -= A B^T on the SIMT units (the float64 trailing update): A = M x K with
// element (r, k) at A[r + k lda_a], B = N x K with element (c, k) at
// B[k + c ldb] (the block row of U), C column-major.  64 x 64 tiles, 4 x 4
// per thread, K in chunks of 16.
template <typename real>
__global__ void __launch_bounds__(256)
lu_update_kernel(int M, int N, int K, const real* A, int64_t lda_a, const real* B, int64_t ldb,
                 real* C, int64_t ldc) {
  const int i0 = blockIdx.x * NB, c0 = blockIdx.y * NB;
  __shared__ real As[16][NB + 1];
  __shared__ real Bs[16][NB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  real acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = 0;
  for (int l0 = 0; l0 < K; l0 += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      const int i = e % NB, l = e / NB;          // A: rows contiguous
      const int lb = e % 16, cb = e / 16;        // B: K contiguous
      As[l][i] = (i0 + i < M && l0 + l < K) ? A[(i0 + i) + (int64_t)(l0 + l) * lda_a] : real(0);
      Bs[lb][cb] = (c0 + cb < N && l0 + lb < K) ? B[(l0 + lb) + (int64_t)(c0 + cb) * ldb] : real(0);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; l++) {
      real a[4], c[4];
#pragma unroll
      for (int p = 0; p < 4; p++) {
        a[p] = As[l][ty + 16 * p];
        c[p] = Bs[l][tx + 16 * p];
      }
#pragma unroll
      for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] += a[p] * c[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int gi = i0 + ty + 16 * p, gj = c0 + tx + 16 * q;
      if (gi < M && gj < N) C[gi + (int64_t)gj * ldc] -= acc[p][q];
    }
}

// W = A^T for the upper triangle (W's lower triangle = U^T), 32 x 32 tiles
// through shared memory.
template <typename real>
__global__ void __launch_bounds__(256)
lu_transpose_upper_kernel(const real* A, int64_t lda, real* W, int64_t ldw, int n) {
  __shared__ real t[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // W tile rows bi.., cols bj..
  if (bj > bi + 31) return;  // strictly above W's diagonal: not read
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int r = e % 32, c = e / 32;  // A(bj + r, bi + c)
    if (bj + r < n && bi + c < n) t[c][r] = A[(bj + r) + (int64_t)(bi + c) * lda];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int r = e % 32, c = e / 32;  // W(bi + r, bj + c) = A(bj + c, bi + r)
    if (bi + r < n && bj + c < n) W[(bi + r) + (int64_t)(bj + c) * ldw] = t[r][c];
  }
}

__global__ void lu_iota_kernel(int* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

// Rows per CTA and CTAs of the panel cluster for `rows` panel rows: about one
// row per thread, at most 16 CTAs; 0 CTAs when the panel does not fit.
template <typename real>
void lu_panel_shape(int rows, int& CL, int& R) {
  CL = 1;
  while (CL < kLuMaxCl && (int64_t)CL * kLuThreads < rows) CL *= 2;
  R = (rows + CL - 1) / CL;
  if (lu_panel_smem<real>(R) > kLuSmemCap) CL = 0;
}

}  // namespace

template <typename real>
void Launch<real>::dense_top(real* A, int64_t lda, int n, real* X, DevError* err, int level,
                             cudaStream_t st) {
  if (n <= 0) return;
  const int nblk = (n + NB - 1) / NB;
  for (int p = 0; p < nblk; p++) {
    const int j0 = p * NB, b = std::min(NB, n - j0);
    count_launch();
    potrf_diag_kernel<real><<<1, 256, 0, st>>>(A, lda, j0, b, err, level);
    const int rest = n - j0 - b;
    if (rest > 0) {
      const int nt = (rest + NB - 1) / NB;
      count_launch();
      trsm_panel_kernel<real><<<nt, 64, 0, st>>>(A, lda, n, j0, b);
      count_launch();
      syrk_update_kernel<real><<<dim3(nt, nt), 256, 0, st>>>(A, lda, n, j0, b);
    }
  }
  count_launch();
  zero_upper_kernel<real><<<152 * 4, 256, 0, st>>>(X, n, n, nullptr);
  for (int i = 0; i < nblk; i++) {
    count_launch();
    trtri_row_kernel<real><<<i + 1, 256, 0, st>>>(A, lda, X, n, n, i, 0, nullptr);
  }
}

template <typename real>
int Launch<real>::lu_top_max() {
  int R = (int)(kLuSmemCap / (lu_nb<real>() * sizeof(real) + sizeof(int)));
  while (R > 0 && lu_panel_smem<real>(R) > kLuSmemCap) R--;
  return kLuMaxCl * R;
}

template <typename real>
size_t Launch<real>::lu_top_scratch(int n) {
  return sizeof(real) * (size_t)n * n + sizeof(int) * 2 * (size_t)n;
}

template <typename real>
bool Launch<real>::lu_top(real* A, int64_t lda, int n, real* T, real* TRt, void* scratch,
                          DevError* err, int level, cudaStream_t st) {
  if (n <= 0) return true;
  if (n > lu_top_max()) return false;
  constexpr int NBL = lu_nb<real>();
  real* W = static_cast<real*>(scratch);
  int* ipiv = reinterpret_cast<int*>(W + (size_t)n * n);
  int* perm = ipiv + n;
  // the limits are raised once, to the sizing cap, and never lowered
  static const bool attr_set = [] {
    cudaFuncSetAttribute(lu_panel_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kLuSmemCap);
    cudaFuncSetAttribute(lu_panel_kernel<real>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return true;
  }();
  (void)attr_set;
  count_launch();
  lu_iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(perm, n);
  for (int j0 = 0; j0 < n; j0 += NBL) {
    const int b = std::min(NBL, n - j0), rows = n - j0;
    int CL = 0, R = 0;
    lu_panel_shape<real>(rows, CL, R);
    if (CL == 0) return false;  // above lu_top_max(): nothing launched for this panel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kLuThreads);
    cfg.dynamicSmemBytes = lu_panel_smem<real>(R);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    // a cluster that cannot be launched ends the factorization here (the
    // error stays readable through cudaGetLastError)
    if (cudaLaunchKernelEx(&cfg, lu_panel_kernel<real>, A, lda, n, j0, b, R, ipiv, err, level) !=
        cudaSuccess)
      return false;
    // the interchanges (and the row order) also when no other column is left
    const int cols = std::max(1, n - b);
    count_launch();
    lu_swap_kernel<real><<<std::min(152 * 4, (cols + 7) / 8), 256, 0, st>>>(A, lda, n, j0, b,
                                                                           ipiv, perm);
    const int rest = n - j0 - b;
    if (rest <= 0) continue;
    count_launch();
    lu_trsm_kernel<real><<<(rest + 127) / 128, 128, 0, st>>>(A, lda, n, j0, b);
    const real* L21 = A + (j0 + b) + (int64_t)j0 * lda;
    const real* U12 = A + j0 + (int64_t)(j0 + b) * lda;
    real* A22 = A + (j0 + b) + (int64_t)(j0 + b) * lda;
    if constexpr (std::is_same<real, float>::value) {
      tc_gemm(1, rest, rest, b, reinterpret_cast<const float*>(L21), 1, lda,
              reinterpret_cast<const float*>(U12), lda, 1, reinterpret_cast<float*>(A22), lda,
              -1.f, 1.f, false, err, st);
    } else {
      count_launch();
      lu_update_kernel<real><<<dim3((rest + NB - 1) / NB, (rest + NB - 1) / NB), 256, 0, st>>>(
          rest, rest, b, L21, lda, U12, lda, A22, lda);
    }
  }
  const int nblk = (n + NB - 1) / NB;
  // T' = L^{-1} P: the unit lower inverse, column c stored at column perm[c]
  count_launch();
  zero_upper_kernel<real><<<152 * 4, 256, 0, st>>>(T, n, n, perm);
  for (int i = 0; i < nblk; i++) {
    count_launch();
    trtri_row_kernel<real><<<i + 1, 256, 0, st>>>(A, lda, T, n, n, i, 1, perm);
  }
  // T'_R^T = U^{-T}: U^T into the lower triangle of W, then its inverse
  count_launch();
  lu_transpose_upper_kernel<real><<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, st>>>(A, lda, W,
                                                                                      n, n);
  count_launch();
  zero_upper_kernel<real><<<152 * 4, 256, 0, st>>>(TRt, n, n, nullptr);
  for (int i = 0; i < nblk; i++) {
    count_launch();
    trtri_row_kernel<real><<<i + 1, 256, 0, st>>>(W, n, TRt, n, n, i, 0, nullptr);
  }
  return true;
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
