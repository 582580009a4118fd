// Dense top factorization (Alg. 1: the remaining system is factored with a
// conventional dense factorization once it is small enough).
//
// SPD top too large for one CTA (float64; the float32 modes use the
// tensor-core recursion of the tcgen05 kernels): blocked right-looking
// Cholesky over 64-column panels (one CTA factors the diagonal block, a
// launch of CTAs solves the panel, a launch updates the trailing lower
// triangle), then the explicit inverse factor X = L^{-1} recursively: the
// 64 x 64 diagonal blocks inverted in one launch, then X21 = -X22 (L21 X11)
// per split, as matrix products.  The substitution sweeps apply X as dense
// products.  Matrices are column-major in global memory.
//
// General (nonsymmetric) top (Sec. 6): recursive LU with partial pivoting
// over column halves -- left half, U12 = X11 A12, A22 -= L21 U12, right half
// -- that grows the inverse factors X = L^{-1} and Z = U^{-T} with it
// (X21 = -X22 (L21 X11), Z21 = -Z22 (U12^T Z11)).  A leaf is one panel of nb
// columns (128 bytes of a row: 32 float32 or 16 float64 columns) factored by
// one thread-block cluster that holds the whole tall panel in distributed
// shared memory: per column one cluster barrier, after which every CTA reads
// each CTA's largest |a| over the remaining rows and its lowest current row
// within 1e-10 of that, and takes the lowest such row within 1e-10 of the
// overall maximum (the tie rule of the one-CTA LU, applied per CTA); row
// interchanges inside the panel are relabellings, not copies, and the
// panel's diagonal blocks of X and Z come out with it; a second launch
// applies the panel's interchanges to every other column.  The products run
// on the tensor cores (3xTF32) in float32 and on the SIMT units in float64
// (skipping the zero chunks of triangular operands).  The stored operators
// follow from A = P^T L U: T' = L^{-1} P (the columns of X scattered by the
// row order) and T'_R^T = Z.
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
// the panel.  Step j: every CTA publishes its largest |a_j| over positions
// >= j and, among its rows within 1e-10 of that, the lowest position; after
// one cluster barrier every CTA reads all of them, and the pivot is the
// lowest published position among the CTAs within 1e-10 of the overall
// maximum (the tie rule of the one-CTA LU, applied per CTA).  The pivot takes
// position j and the slot at position j takes the pivot's old position
// (ipiv[j0 + j] = j0 + that position, the LAPACK convention); the rows at
// positions > j are updated with l = a_j / u_jj.  The exchange records are
// double-buffered by step parity: a CTA can only write a record again after
// the next barrier, which every CTA reaches after reading it.  The pivot row
// is read by every CTA from its owner's shared memory; it is never written
// again.  At the end CTA 0 gathers the b x b diagonal block (L_jj \ U_jj)
// through distributed shared memory and writes X_jj = L_jj^{-1} and
// Z_jj = U_jj^{-T} (b x b, zeros above the diagonal) at (j0, j0) of X and
// Z; every slot is written back at its position.  All CTAs take the same
// branches (their decisions use the same exchanged values), so the cluster
// barriers always match.  A column with no nonzero left records
// HSOLVE_ERR_SINGULAR and ends the panel (the remaining ipiv entries are
// identities, so later launches stay in bounds).
template <typename real>
__global__ void __launch_bounds__(kLuThreads)
lu_panel_kernel(real* A, int64_t lda, int n, int j0, int b, int R, int* __restrict__ ipiv,
                real* __restrict__ X, int64_t ldx, real* __restrict__ Z, int64_t ldz,
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
  __shared__ LuXch xch[2];
  __shared__ real urow[NBL];
  __shared__ int slot_of[NBL];  // slot at positions 0..b-1
  __shared__ double red_d[kLuThreads / 32];
  __shared__ unsigned long long red_u[kLuThreads / 32];
  __shared__ double s_mloc;
  __shared__ int s_p, s_sp, s_bad;
  __shared__ real D[NBL][NBL + 1];  // CTA 0: the diagonal block, D[c][q] = (q, c)
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
    LuXch& xo = xch[j & 1];
    // 1. this CTA's largest |a_j| over the remaining rows ...
    double mx = 0;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x)
      if (lab[i] >= j) mx = fmax(mx, fabs((double)Ps[i + (int64_t)j * R]));
    mx = lu_warp_max(mx);
    if (lane == 0) red_d[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_d[0];
      for (int w = 1; w < nwarp; w++) v = fmax(v, red_d[w]);
      s_mloc = v;
    }
    __syncthreads();
    // ... and its lowest position within the tie band of it
    const double ml = s_mloc;
    unsigned long long key = ~0ull;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) {
      const int p = lab[i];
      if (p >= j && fabs((double)Ps[i + (int64_t)j * R]) >= (1.0 - kLuTieRtol) * ml) {
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
      const bool any = v != ~0ull && ml > 0.0;
      xo.val = ml;
      xo.cand = any ? (int)(v >> 32) : INT_MAX;
      xo.slot = any ? s0 + (int)(v & 0xffffffffu) : -1;
    }
    cl.sync();
    // 2. the pivot from all CTAs' records (warp 0, one lane per CTA)
    if (warp == 0) {
      double v = 0.0;
      int cand = INT_MAX, slot = -1;
      if (lane < CL) {
        const LuXch* r = cl.map_shared_rank(&xo, lane);
        v = r->val;
        cand = r->cand;
        slot = r->slot;
      }
      const double M = lu_warp_max(v);
      unsigned long long kk = ~0ull;
      if (lane < CL && M > 0.0 && v >= (1.0 - kLuTieRtol) * M && cand != INT_MAX)
        kk = ((unsigned long long)(unsigned)cand << 8) | lane;
      kk = lu_warp_min(kk);
      const int win = kk == ~0ull ? 0 : (int)(kk & 0xff);
      const int wslot = __shfl_sync(0xffffffffu, slot, win);
      if (lane == 0) {
        s_bad = kk == ~0ull;
        s_p = (int)(kk >> 8);
        s_sp = wslot;
      }
    }
    __syncthreads();
    if (s_bad) {
      if (cr == 0 && threadIdx.x == 0) {
        if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_SINGULAR) == 0) {
          err->cluster = 0;
          err->level = level;
        }
        for (int jj = j; jj < b; jj++) ipiv[j0 + jj] = j0 + jj;
      }
      break;
    }
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
  // every update is done (and every read of a pivot row); CTA 0 then reads
  // the diagonal block, while no CTA leaves
  cl.sync();
  if (cr == 0)
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int q = e % b, c = e / b;
      const int sl = slot_of[q], ow = sl / R;
      D[c][q] = cl.map_shared_rank(Ps, ow)[(sl - ow * R) + (int64_t)c * R];
    }
  cl.sync();
  for (int e = threadIdx.x; e < nloc * b; e += blockDim.x) {
    const int i = e % nloc, c = e / nloc;
    A[(j0 + lab[i]) + (int64_t)(j0 + c) * lda] = Ps[i + (int64_t)c * R];
  }
  if (cr != 0) return;
  // X_jj = L_jj^{-1} (unit lower; threads 0..b-1, one column each) and
  // Z_jj = (U_jj^T)^{-1} (threads 32..32+b-1); results in registers' place
  // in the block's own column of X and Z
  if (threadIdx.x < b) {
    const int c = threadIdx.x;
    real x[NBL];
#pragma unroll
    for (int a = 0; a < NBL; a++) x[a] = real(0);
    x[c] = real(1);
    for (int a = c + 1; a < b; a++) {
      real v = 0;
      for (int l = c; l < a; l++) v -= D[l][a] * x[l];
      x[a] = v;
    }
    for (int a = 0; a < b; a++) X[(j0 + a) + (int64_t)(j0 + c) * ldx] = x[a];
  } else if (threadIdx.x >= 32 && threadIdx.x < 32 + b) {
    const int c = threadIdx.x - 32;
    real z[NBL];
#pragma unroll
    for (int a = 0; a < NBL; a++) z[a] = real(0);
    z[c] = real(1) / D[c][c];
    for (int a = c + 1; a < b; a++) {
      real v = 0;
      for (int l = c; l < a; l++) v -= D[a][l] * z[l];  // U^T(a, l) = U(l, a)
      z[a] = v / D[a][a];
    }
    for (int a = 0; a < b; a++) Z[(j0 + a) + (int64_t)(j0 + c) * ldz] = z[a];
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

// C = alpha A B^T + beta C on the SIMT units (the float64 products of the
// dense tops): A = M x K with element (r, k) at A[r rsa + k csa], B = N x K
// with element (c, k) at B[c rsb + k csb], C column-major (C is not read
// when beta = 0).  64 x 64 tiles, 4 x 4 per thread, K in chunks of 16; each
// operand is staged with its unit-stride index fastest.  Triangular operands
// skip their zero chunks: tri & 1 -- A(r, k) = 0 for k > r; tri & 2 --
// B(c, k) = 0 for k < c.
template <typename real>
__global__ void __launch_bounds__(256)
simt_gemm_kernel(int M, int N, int K, const real* __restrict__ A, int64_t rsa, int64_t csa,
                 const real* __restrict__ B, int64_t rsb, int64_t csb, real* __restrict__ C,
                 int64_t ldc, real alpha, real beta, int tri) {
  const int i0 = blockIdx.x * NB, c0 = blockIdx.y * NB;
  const int kbeg = (tri & 2) ? (c0 / 16) * 16 : 0;
  const int kend = (tri & 1) ? min(K, i0 + NB) : K;
  __shared__ real As[16][NB + 1];
  __shared__ real Bs[16][NB + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const bool a_rows = rsa == 1, b_rows = rsb == 1;
  real acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) acc[p][q] = 0;
  for (int l0 = kbeg; l0 < kend; l0 += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      int i, l;
      if (a_rows) { i = e % NB; l = e / NB; } else { l = e % 16; i = e / 16; }
      As[l][i] = (i0 + i < M && l0 + l < kend)
                     ? A[(int64_t)(i0 + i) * rsa + (int64_t)(l0 + l) * csa]
                     : real(0);
      int c, lb;
      if (b_rows) { c = e % NB; lb = e / NB; } else { lb = e % 16; c = e / 16; }
      Bs[lb][c] = (c0 + c < N && l0 + lb < kend)
                      ? B[(int64_t)(c0 + c) * rsb + (int64_t)(l0 + lb) * csb]
                      : real(0);
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
      if (gi < M && gj < N) {
        real* cp = C + gi + (int64_t)gj * ldc;
        *cp = beta == real(0) ? alpha * acc[p][q] : alpha * acc[p][q] + beta * *cp;
      }
    }
}

// dst (rows x cols, ld ldd) = src (ld lds)
template <typename real>
__global__ void copy_mat_kernel(const real* __restrict__ src, int64_t lds, real* __restrict__ dst,
                                int64_t ldd, int rows, int cols) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[i + (int64_t)j * ldd] = src[i + (int64_t)j * lds];
  }
}

// T[:, perm[c]] = X[:, c] (n x n, ld n each): the column order of L^{-1} P
template <typename real>
__global__ void scatter_cols_kernel(const real* __restrict__ X, real* __restrict__ T,
                                    const int* __restrict__ perm, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    T[i + (int64_t)perm[c] * n] = X[i + (int64_t)c * n];
  }
}

// X_bb = L_bb^{-1} for every 64 x 64 diagonal block b of the lower triangular
// L (n x n, ld ldl; unit diagonal if `unit`), one CTA per block, one thread
// per column; zeros above the diagonal inside the block.
template <typename real>
__global__ void __launch_bounds__(64)
tri_inv_diag_kernel(const real* __restrict__ L, int64_t ldl, real* __restrict__ X, int64_t ldx,
                    int n, int unit) {
  // Ld[c][a] = L(r0 + a, r0 + c), Xs[c][a] = X(r0 + a, r0 + c); dynamic
  // shared memory (66.5 KB in float64)
  extern __shared__ __align__(16) unsigned char tri_smem[];
  real(*Ld)[NB + 1] = reinterpret_cast<real(*)[NB + 1]>(tri_smem);
  real(*Xs)[NB + 1] = Ld + NB;
  const int r0 = blockIdx.x * NB, bs = min(NB, n - r0);
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int a = e % bs, c = e / bs;
    Ld[c][a] = L[(r0 + a) + (int64_t)(r0 + c) * ldl];
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < bs) {
    for (int a = 0; a < c; a++) Xs[c][a] = real(0);
    Xs[c][c] = unit ? real(1) : real(1) / Ld[c][c];
    for (int a = c + 1; a < bs; a++) {
      real v = 0;
      for (int l = c; l < a; l++) v -= Ld[l][a] * Xs[c][l];
      Xs[c][a] = unit ? v : v / Ld[a][a];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int a = e % bs, cc = e / bs;
    X[(r0 + a) + (int64_t)(r0 + cc) * ldx] = Xs[cc][a];
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

int grid_for(int64_t work) { return (int)std::min<int64_t>((work + 255) / 256, 152 * 8); }

// C = alpha A B^T + beta C (conventions of simt_gemm_kernel): float32 on the
// tensor cores (3xTF32, float32-level accuracy), float64 on the SIMT units.
// tri: the triangular structure of the operands (simt_gemm_kernel), used
// by the SIMT path to skip zero chunks.
template <typename real>
void gemm_nt(int M, int N, int K, const real* A, int64_t rsa, int64_t csa, const real* B,
             int64_t rsb, int64_t csb, real* C, int64_t ldc, real alpha, real beta, int tri,
             DevError* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  if constexpr (std::is_same<real, float>::value) {
    (void)tri;
    tc_gemm(1, M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, false, err, st);
  } else {
    (void)err;
    count_launch();
    simt_gemm_kernel<real><<<dim3((M + NB - 1) / NB, (N + NB - 1) / NB), 256, 0, st>>>(
        M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, tri);
  }
}

// X = L^{-1} for the lower triangular n x n L (unit diagonal if `unit`),
// recursively: with L = [L11 0; L21 L22] split at a multiple of 64,
// X11 = L11^{-1}, X22 = L22^{-1} and X21 = -X22 (L21 X11), so that all but
// the 64 x 64 diagonal blocks (inverted first, in one launch) are matrix
// products.  X's blocks above the diagonal are zeroed by the caller.  W:
// scratch of at least (n/2 + 64)^2 elements.
template <typename real>
void tri_inv_products(const real* L, int64_t ldl, real* X, int64_t ldx, int n, real* W,
                      DevError* err, cudaStream_t st) {
  if (n <= NB) return;
  const int n1 = std::max(NB, ((n / 2) + NB - 1) / NB * NB);
  const int n2 = n - n1;
  if (n2 <= 0) return;
  tri_inv_products(L, ldl, X, ldx, n1, W, err, st);
  tri_inv_products(L + n1 + (int64_t)n1 * ldl, ldl, X + n1 + (int64_t)n1 * ldx, ldx, n2, W, err,
                   st);
  // W = L21 X11 (n2 x n1, ld n2), X21 = -X22 W
  gemm_nt<real>(n2, n1, n1, L + n1, 1, ldl, X, ldx, 1, W, n2, real(1), real(0), 2, err, st);
  gemm_nt<real>(n2, n1, n2, X + n1 + (int64_t)n1 * ldx, 1, ldx, W, n2, 1, X + n1, ldx, real(-1),
                real(0), 1, err, st);
}

template <typename real>
void tri_inv(const real* L, int64_t ldl, real* X, int64_t ldx, int n, bool unit, real* W,
             DevError* err, cudaStream_t st) {
  const size_t smem = sizeof(real) * 2 * NB * (NB + 1);
  static const bool attr_set = [smem] {
    cudaFuncSetAttribute(tri_inv_diag_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    return true;
  }();
  (void)attr_set;
  count_launch();
  tri_inv_diag_kernel<real><<<(n + NB - 1) / NB, 64, smem, st>>>(L, ldl, X, ldx, n,
                                                                 unit ? 1 : 0);
  tri_inv_products(L, ldl, X, ldx, n, W, err, st);
}

// The recursive LU of the columns [j0, j0 + nn) over rows [j0, n) (the left
// columns' updates already applied), with the inverse factors of its
// diagonal block: X = L^{-1} (unit lower) and Z = U^{-T}, both ld n, at
// (j0, j0).  With the columns split at n1 (a multiple of the panel width):
//   left half recursively (its interchanges applied to all columns),
//   U12 = X11 A12, A22 -= L21 U12 (rows below), right half recursively,
//   X21 = -X22 (L21 X11), Z21 = -Z22 (U12^T Z11).
// A leaf is one panel on a thread-block cluster (which also writes its
// diagonal blocks of X and Z) and the launch applying its interchanges.
template <typename real>
struct LuCtx {
  real* A;
  int64_t lda;
  int n;
  real *X, *Z, *W;  // W: (n/2 + nb)^2 scratch
  int *ipiv, *perm;
  DevError* err;
  int level;
  cudaStream_t st;
};

template <typename real>
bool lu_rec(const LuCtx<real>& c, int j0, int nn) {
  constexpr int NBL = lu_nb<real>();
  const int n = c.n;
  const int64_t lda = c.lda, ld = n;
  if (nn <= NBL) {
    const int rows = n - j0;
    int CL = 0, R = 0;
    lu_panel_shape<real>(rows, CL, R);
    if (CL == 0) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kLuThreads);
    cfg.dynamicSmemBytes = lu_panel_smem<real>(R);
    cfg.stream = c.st;
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
    if (cudaLaunchKernelEx(&cfg, lu_panel_kernel<real>, c.A, lda, n, j0, nn, R, c.ipiv, c.X, ld,
                           c.Z, ld, c.err, c.level) != cudaSuccess)
      return false;
    // the interchanges (and the row order) also when no other column is left
    const int cols = std::max(1, n - nn);
    count_launch();
    lu_swap_kernel<real><<<std::min(152 * 4, (cols + 7) / 8), 256, 0, c.st>>>(c.A, lda, n, j0, nn,
                                                                             c.ipiv, c.perm);
    return true;
  }
  const int n1 = std::max(NBL, ((nn / 2) + NBL - 1) / NBL * NBL);
  const int n2 = nn - n1;
  const int j1 = j0 + n1;
  if (!lu_rec(c, j0, n1)) return false;
  real* A = c.A;
  const real* X11 = c.X + j0 + (int64_t)j0 * ld;
  const real* Z11 = c.Z + j0 + (int64_t)j0 * ld;
  // U12 = X11 A12 into W (n1 x n2, ld n1); A22 -= L21 U12; A12 = U12
  gemm_nt<real>(n1, n2, n1, X11, 1, ld, A + j0 + (int64_t)j1 * lda, lda, 1, c.W, n1, real(1),
                real(0), 1, c.err, c.st);
  gemm_nt<real>(n - j1, n2, n1, A + j1 + (int64_t)j0 * lda, 1, lda, c.W, n1, 1,
                A + j1 + (int64_t)j1 * lda, lda, real(-1), real(1), 0, c.err, c.st);
  count_launch();
  copy_mat_kernel<real><<<grid_for((int64_t)n1 * n2), 256, 0, c.st>>>(
      c.W, n1, A + j0 + (int64_t)j1 * lda, lda, n1, n2);
  if (!lu_rec(c, j1, n2)) return false;
  // X21 = -X22 (L21 X11): W = L21 X11 (n2 x n1, ld n2)
  gemm_nt<real>(n2, n1, n1, A + j1 + (int64_t)j0 * lda, 1, lda, X11, ld, 1, c.W, n2, real(1),
                real(0), 2, c.err, c.st);
  gemm_nt<real>(n2, n1, n2, c.X + j1 + (int64_t)j1 * ld, 1, ld, c.W, n2, 1,
                c.X + j1 + (int64_t)j0 * ld, ld, real(-1), real(0), 1, c.err, c.st);
  // Z21 = -Z22 (U12^T Z11): W = U12^T Z11
  gemm_nt<real>(n2, n1, n1, A + j0 + (int64_t)j1 * lda, lda, 1, Z11, ld, 1, c.W, n2, real(1),
                real(0), 2, c.err, c.st);
  gemm_nt<real>(n2, n1, n2, c.Z + j1 + (int64_t)j1 * ld, 1, ld, c.W, n2, 1,
                c.Z + j1 + (int64_t)j0 * ld, ld, real(-1), real(0), 1, c.err, c.st);
  return true;
}

}  // namespace

template <typename real>
void Launch<real>::dense_top(real* A, int64_t lda, int n, real* X, real* W, DevError* err,
                             int level, cudaStream_t st) {
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
  cudaMemsetAsync(X, 0, sizeof(real) * (size_t)n * n, st);
  tri_inv<real>(A, lda, X, n, n, false, W, err, st);
}

template <typename real>
size_t Launch<real>::dense_top_scratch(int n) {
  const size_t h = (size_t)n / 2 + NB;
  return sizeof(real) * h * h;
}

template <typename real>
int Launch<real>::lu_top_max() {
  int R = (int)(kLuSmemCap / (lu_nb<real>() * sizeof(real) + sizeof(int)));
  while (R > 0 && lu_panel_smem<real>(R) > kLuSmemCap) R--;
  return kLuMaxCl * R;
}

template <typename real>
size_t Launch<real>::lu_top_scratch(int n) {
  const size_t h = (size_t)n / 2 + lu_nb<real>();
  return sizeof(real) * ((size_t)n * n + h * h) + sizeof(int) * 2 * (size_t)n;
}

template <typename real>
bool Launch<real>::lu_top(real* A, int64_t lda, int n, real* T, real* TRt, void* scratch,
                          DevError* err, int level, cudaStream_t st) {
  if (n <= 0) return true;
  if (n > lu_top_max()) return false;
  const size_t h = (size_t)n / 2 + lu_nb<real>();
  real* X = static_cast<real*>(scratch);
  real* W = X + (size_t)n * n;
  int* ipiv = reinterpret_cast<int*>(W + h * h);
  int* perm = ipiv + n;
  // the limits are raised once, to the sizing cap, and never lowered
  static const bool attr_set = [] {
    cudaFuncSetAttribute(lu_panel_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kLuSmemCap);
    cudaFuncSetAttribute(lu_panel_kernel<real>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return true;
  }();
  (void)attr_set;
  // X and Z = T'_R^T start at zero: their blocks above the diagonal stay so
  if (cudaMemsetAsync(X, 0, sizeof(real) * (size_t)n * n, st) != cudaSuccess ||
      cudaMemsetAsync(TRt, 0, sizeof(real) * (size_t)n * n, st) != cudaSuccess)
    return false;
  count_launch();
  lu_iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(perm, n);
  LuCtx<real> c{A, lda, n, X, TRt, W, ipiv, perm, err, level, st};
  if (!lu_rec(c, 0, n)) return false;
  // T' = L^{-1} P: column c of X at column perm[c]
  count_launch();
  scatter_cols_kernel<real><<<grid_for((int64_t)n * n), 256, 0, st>>>(X, T, perm, n);
  return true;
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
