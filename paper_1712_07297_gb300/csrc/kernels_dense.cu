// Per-cluster dense work of one LowRank_Elimination step (Sec. 2.1):
// factor A_ss, form A_ss^{-1}, compress the fill block with column-pivoted
// Householder QR (Eq. lra), build the complement basis V with
// V^T A_ss^{-1} U = 0, the sparsification rows T = [U V]^T A_ss^{-1}
// (Eq. scaling), factor the fine block F = V^T A_ss^{-1} V (Eq. elim) and fold
// its inverse factor into T.  One CTA per cluster of a colour class; all
// clusters of the class run in one launch.
//
// Matrices are column-major.  `real` is the storage/compute type of the
// factorization (double in float64 mode, float in the mixed modes); squared
// column norms of the rank-revealing QR and its rank decision are always
// accumulated in double.
#include <cfloat>
#include <climits>
#include <cmath>

#include "common.h"

namespace hs {

namespace {

constexpr int kPrepThreads = 256;
constexpr double kPivotTieRtol = 1e-10;

template <typename real>
__device__ __forceinline__ real rsqrt_(real x);
template <>
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }

// C (M x N, ldc) = alpha * op(A) * op(B) + beta * C, whole CTA.
template <typename real>
__device__ void cta_gemm(int M, int N, int K, const real* A, int lda, bool ta, const real* B,
                         int ldb, bool tb, real* C, int ldc, real alpha, real beta) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    int i = idx % M, j = idx / M;
    real acc = 0;
    if (!ta && !tb) {
      for (int l = 0; l < K; l++) acc += A[i + (int64_t)l * lda] * B[l + (int64_t)j * ldb];
    } else if (ta && !tb) {
      for (int l = 0; l < K; l++) acc += A[l + (int64_t)i * lda] * B[l + (int64_t)j * ldb];
    } else if (!ta && tb) {
      for (int l = 0; l < K; l++) acc += A[i + (int64_t)l * lda] * B[j + (int64_t)l * ldb];
    } else {
      for (int l = 0; l < K; l++) acc += A[l + (int64_t)i * lda] * B[j + (int64_t)l * ldb];
    }
    real c = alpha * acc;
    if (beta != real(0)) c += beta * C[i + (int64_t)j * ldc];
    C[i + (int64_t)j * ldc] = c;
  }
  __syncthreads();
}

template <typename real>
__device__ void cta_copy(int M, int N, const real* A, int64_t lda, real* B, int64_t ldb) {
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    int i = idx % M, j = idx / M;
    B[i + j * ldb] = A[i + j * lda];
  }
  __syncthreads();
}

template <typename real>
__device__ void cta_identity(int M, int N, int diag_off, real* A, int lda) {
  // A[i, j] = (i == j + diag_off)
  for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
    int i = idx % M, j = idx / M;
    A[i + (int64_t)j * lda] = (i == j + diag_off) ? real(1) : real(0);
  }
  __syncthreads();
}

// In-place lower Cholesky A = L L^T.  Returns false (on every thread) for a
// non-positive pivot.
template <typename real>
__device__ bool cta_cholesky(int n, real* A, int lda, int* sflag) {
  for (int j = 0; j < n; j++) {
    if (threadIdx.x == 0) {
      real d = A[j + (int64_t)j * lda];
      if (!(d > real(0))) {
        *sflag = 1;
      } else {
        A[j + (int64_t)j * lda] = rsqrt_(d);
      }
    }
    __syncthreads();
    if (*sflag) return false;
    real djj = A[j + (int64_t)j * lda];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)j * lda] /= djj;
    __syncthreads();
    int t = n - j - 1;
    // trailing update of the lower triangle
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
      int i = j + 1 + idx % t, l = j + 1 + idx / t;
      if (i >= l) A[i + (int64_t)l * lda] -= A[i + (int64_t)j * lda] * A[l + (int64_t)j * lda];
    }
    __syncthreads();
  }
  return true;
}

// In-place LU with partial pivoting, P A = L U (unit lower L).  piv[j] = row
// swapped with j at step j.  Near-ties (|a| >= (1 - 1e-10) max) go to the
// lowest row.  Returns false for an exactly zero pivot column.
template <typename real>
__device__ bool cta_lu(int n, real* A, int lda, int* piv, real* red_v, int* red_i,
                       int* sflag) {
  for (int j = 0; j < n; j++) {
    // column maximum
    real mx = 0;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(A[i + (int64_t)j * lda]));
    red_v[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red_v[threadIdx.x] = fmax(red_v[threadIdx.x], red_v[threadIdx.x + s]);
      __syncthreads();
    }
    mx = red_v[0];
    __syncthreads();
    int best = n;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x)
      if (fabs(A[i + (int64_t)j * lda]) >= (real)(1.0 - kPivotTieRtol) * mx && i < best) best = i;
    red_i[threadIdx.x] = best;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red_i[threadIdx.x] = min(red_i[threadIdx.x], red_i[threadIdx.x + s]);
      __syncthreads();
    }
    int p = red_i[0];
    __syncthreads();
    if (threadIdx.x == 0) {
      piv[j] = p;
      if (!(mx > real(0))) *sflag = 1;
    }
    __syncthreads();
    if (*sflag) return false;
    if (p != j)
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        real t = A[j + (int64_t)c * lda];
        A[j + (int64_t)c * lda] = A[p + (int64_t)c * lda];
        A[p + (int64_t)c * lda] = t;
      }
    __syncthreads();
    real d = A[j + (int64_t)j * lda];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)j * lda] /= d;
    __syncthreads();
    int t = n - j - 1;
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
      int i = j + 1 + idx % t, l = j + 1 + idx / t;
      A[i + (int64_t)l * lda] -= A[i + (int64_t)j * lda] * A[j + (int64_t)l * lda];
    }
    __syncthreads();
  }
  return true;
}

// Linv = L^{-1} for lower triangular L (unit diagonal if `unit`), column
// parallel forward substitution.  Linv is n x n, upper part zeroed.
template <typename real>
__device__ void cta_tri_inv_lower(int n, const real* L, int ldl, bool unit, real* Li, int ldi) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    real* y = Li + (int64_t)c * ldi;
    for (int i = 0; i < c; i++) y[i] = 0;
    y[c] = unit ? real(1) : real(1) / L[c + (int64_t)c * ldl];
    for (int i = c + 1; i < n; i++) {
      real acc = 0;
      for (int l = c; l < i; l++) acc += L[i + (int64_t)l * ldl] * y[l];
      y[i] = unit ? -acc : -acc / L[i + (int64_t)i * ldl];
    }
  }
  __syncthreads();
}

// Ui = U^{-1} for upper triangular U, column-parallel back substitution.
template <typename real>
__device__ void cta_tri_inv_upper(int n, const real* U, int ldu, real* Ui, int ldi) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    real* y = Ui + (int64_t)c * ldi;
    for (int i = c + 1; i < n; i++) y[i] = 0;
    y[c] = real(1) / U[c + (int64_t)c * ldu];
    for (int i = c - 1; i >= 0; i--) {
      real acc = 0;
      for (int l = i + 1; l <= c; l++) acc += U[i + (int64_t)l * ldu] * y[l];
      y[i] = -acc / U[i + (int64_t)i * ldu];
    }
  }
  __syncthreads();
}

// Block reductions over the first `cnt` entries handled by all threads.
__device__ double cta_max_d(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

__device__ int cta_min_i(int v, int* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = min(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  int r = red[0];
  __syncthreads();
  return r;
}

// Householder QR of the m x c matrix G (in place, ld m).  With `pivot`,
// columns are pivoted by largest remaining norm (recomputed every step,
// near-ties to the lowest original index, orig[] tracks original indices),
// stopping at |r_jj| <= eps |r_11| (eps > 0), at |r_jj| <= floor (rounding
// noise of a block that is zero in exact arithmetic), at an all-zero
// remainder or at kmax steps.  Householder vectors stay in G below the diagonal (v_j in
// G[j:m, j]); tau[j] holds 2 / v^T v.  Returns the number of steps k.
template <typename real>
__device__ int cta_householder_qr(int m, int c, real* G, int ldg, double* nrm2, double* orig,
                                  real* tau, bool pivot, double eps, int kmax, double floor,
                                  double* red_d, int* red_i) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // initial squared norms
  for (int q = warp; q < c; q += nwarp) {
    const real* col = G + (int64_t)q * ldg;
    double s = 0;
    for (int i = lane; i < m; i += 32) s += (double)col[i] * (double)col[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      nrm2[q] = s;
      orig[q] = q;
    }
  }
  __syncthreads();
  double r11 = 0;
  int k = 0;
  const int steps = min(m, c);
  for (int j = 0; j < steps; j++) {
    int q = j;
    double r;
    if (pivot) {
      double mx = 0;
      for (int t = j + threadIdx.x; t < c; t += blockDim.x) mx = fmax(mx, nrm2[t]);
      mx = cta_max_d(mx, red_d);
      if (mx == 0.0) break;
      int best = INT_MAX;
      for (int t = j + threadIdx.x; t < c; t += blockDim.x)
        if (nrm2[t] >= (1.0 - kPivotTieRtol) * mx) best = min(best, (int)orig[t]);
      best = cta_min_i(best, red_i);
      // locate the column holding original index `best`
      for (int t = j + threadIdx.x; t < c; t += blockDim.x)
        if ((int)orig[t] == best) red_i[blockDim.x] = t;
      __syncthreads();
      q = red_i[blockDim.x];
      __syncthreads();
      r = sqrt(nrm2[q]);
      if (j == 0) r11 = r;
      if (r <= floor) break;
      if (eps > 0.0 && r <= eps * r11) break;
      if (j >= kmax) break;
      if (q != j) {
        real* a = G + (int64_t)j * ldg;
        real* b = G + (int64_t)q * ldg;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          real t = a[i];
          a[i] = b[i];
          b[i] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double t = nrm2[j];
          nrm2[j] = nrm2[q];
          nrm2[q] = t;
          t = orig[j];
          orig[j] = orig[q];
          orig[q] = t;
        }
        __syncthreads();
      }
    } else {
      if (j >= kmax) break;
      // norm of the current column over rows j..m
      double s = 0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        double x = G[i + (int64_t)j * ldg];
        s += x * x;
      }
      red_d[threadIdx.x] = s;
      __syncthreads();
      for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red_d[threadIdx.x] += red_d[threadIdx.x + st];
        __syncthreads();
      }
      r = sqrt(red_d[0]);
      __syncthreads();
    }
    // reflector v = x - beta e1, beta = -sign(x0) ||x||, tau = 2 / v^T v
    real* x = G + (int64_t)j * ldg;
    double x0 = (double)x[j];
    double beta = (x0 >= 0.0) ? -r : r;
    double tj = (r > 0.0) ? 1.0 / (r * (r + fabs(x0))) : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      x[j] = (real)(x0 - beta);
      tau[j] = (real)tj;
    }
    __syncthreads();
    // apply to the remaining columns; recompute their norms over rows j+1..m
    for (int t = j + 1 + warp; t < c; t += nwarp) {
      real* col = G + (int64_t)t * ldg;
      real w = 0;
      for (int i = j + lane; i < m; i += 32) w += x[i] * col[i];
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= (real)tj;
      double s = 0;
      for (int i = j + lane; i < m; i += 32) {
        real v = col[i] - w * x[i];
        col[i] = v;
        if (i > j) s += (double)v * (double)v;
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) nrm2[t] = s;
    }
    __syncthreads();
    k = j + 1;
  }
  __syncthreads();
  return k;
}

// Q[:, c0:c0+ncols] of Q = H_0 .. H_{k-1}: out (m x ncols, ld m) starts as
// the identity columns c0.. and receives the reflectors in reverse order.
template <typename real>
__device__ void cta_form_q(int m, int k, const real* V, int ldv, const real* tau, int c0,
                           int ncols, real* out, int ldo) {
  cta_identity<real>(m, ncols, c0, out, ldo);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = k - 1; j >= 0; j--) {
    const real* v = V + (int64_t)j * ldv;
    real tj = tau[j];
    for (int t = warp; t < ncols; t += nwarp) {
      real* col = out + (int64_t)t * ldo;
      real w = 0;
      for (int i = j + lane; i < m; i += 32) w += v[i] * col[i];
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= tj;
      for (int i = j + lane; i < m; i += 32) col[i] -= w * v[i];
    }
    __syncthreads();
  }
}

template <typename real>
__global__ void __launch_bounds__(kPrepThreads)
prep_kernel(const PrepTask* __restrict__ tasks, real* __restrict__ arena, real* __restrict__ fac,
            real* __restrict__ ws_all, double* __restrict__ wsd_all,
            const int64_t* __restrict__ gptr, const int* __restrict__ gstr, int* rank,
            double eps, double noise_rtol, int sym, int max_rank, DevError* err, int level) {
  __shared__ double red_d[kPrepThreads];
  __shared__ int red_i[kPrepThreads + 1];
  __shared__ int sflag;
  __shared__ int s_ncol;
  __shared__ double s_amax;
  const PrepTask tk = tasks[blockIdx.x];
  const int m = tk.m;
  if (threadIdx.x == 0) sflag = 0;
  __syncthreads();
  const int64_t mm = (int64_t)m * m;
  real* ws = ws_all + tk.ws;
  real* W_A = ws;                 // A_ss, then its factor
  real* W_B = W_A + mm;           // A_ss^{-1}
  real* W_U = W_B + mm;           // U (m x k)
  real* W_X = W_U + mm;           // X = B U, then its reflectors
  real* W_V = W_X + mm;           // V_L (m x f)
  real* W_T = W_V + mm;           // [U V_L]^T B
  real* W_F = W_T + mm;           // F, then its factor
  real* W_L = W_F + mm;           // inverse factor(s) of F
  real* W_C = W_L + mm;           // C = U^T B U
  real* W_R = W_C + mm;           // general: V_R, then T_R = B [U V_R]
  real* W_S = W_R + mm;           // general: scratch
  real* W_G = W_S + mm;           // G (m x ncolG)
  double* nrm2 = wsd_all + tk.wsd;
  double* orig = nrm2 + tk.ncolG;
  real* tau = reinterpret_cast<real*>(orig + tk.ncolG);
  real* tau2 = tau + m;
  int* piv = reinterpret_cast<int*>(tau2 + m);
  real* T = fac + tk.T;

  // ---- gather A_ss, its largest magnitude (scale of the noise floor), factor
  cta_copy<real>(m, m, arena + tk.a_ss, tk.ld, W_A, m);
  {
    double mx = 0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) mx = fmax(mx, fabs((double)W_A[idx]));
    mx = cta_max_d(mx, red_d);
    if (threadIdx.x == 0) s_amax = mx;
    __syncthreads();
  }
  bool ok = sym ? cta_cholesky<real>(m, W_A, m, &sflag)
                : cta_lu<real>(m, W_A, m, piv, reinterpret_cast<real*>(red_d), red_i, &sflag);
  if (!ok) {
    if (threadIdx.x == 0) {
      if (atomicCAS(&err->code, 0, sym ? (int)HSOLVE_ERR_NOT_SPD : (int)HSOLVE_ERR_SINGULAR) == 0) {
        err->cluster = tk.s;
        err->level = level;
      }
      rank[tk.s] = tk.m;  // leave the cluster untouched downstream
    }
    return;
  }

  // ---- gather the nonzero fill columns into G (Eq. lra input)
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // pass 1: flag nonzero columns (stored in nrm2 temporarily)
    for (int q = warp; q < tk.ncolG; q += nwarp) {
      const int64_t p = gptr[tk.gcol + q];
      const int st = gstr[tk.gcol + q];
      bool nz = false;
      for (int i = lane; i < m; i += 32) nz |= (arena[p + (int64_t)i * st] != real(0));
      nz = __any_sync(0xffffffffu, nz);
      if (lane == 0) nrm2[q] = nz ? 1.0 : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = 0;
      for (int q = 0; q < tk.ncolG; q++) {
        double f = nrm2[q];
        orig[q] = (f != 0.0) ? (double)c : -1.0;
        c += (f != 0.0);
      }
      s_ncol = c;
    }
    __syncthreads();
    for (int q = warp; q < tk.ncolG; q += nwarp) {
      int dst = (int)orig[q];
      if (dst < 0) continue;
      const int64_t p = gptr[tk.gcol + q];
      const int st = gstr[tk.gcol + q];
      for (int i = lane; i < m; i += 32) W_G[i + (int64_t)dst * m] = arena[p + (int64_t)i * st];
    }
    __syncthreads();
  }
  const int ncol = s_ncol;
  int k = 0;
  if (ncol > 0) {
    int kmax = m;
    if (max_rank > 0) kmax = min(kmax, max_rank);
    k = cta_householder_qr<real>(m, ncol, W_G, m, nrm2, orig, tau, true, eps, kmax,
                                 noise_rtol * s_amax, red_d, red_i);
  }
  if (threadIdx.x == 0) rank[tk.s] = k;
  if (k == m) return;  // untouched: all unknowns coarse, E_s = I
  const int f = m - k;

  if (k == 0) {
    // E_s = I: T' = L^{-1} (Cholesky) or L^{-1} P (LU); T'_R^T = U^{-T}
    if (sym) {
      cta_tri_inv_lower<real>(m, W_A, m, false, T, m);
    } else {
      cta_tri_inv_lower<real>(m, W_A, m, true, W_L, m);
      // T = L^{-1} P: column c of P is e_{perm^{-1}(c)}; apply swaps to columns
      // (L^{-1} P)[:, c] = L^{-1}[:, pos(c)], pos(c) = row of P A that
      // holds original row c after the swaps piv[0..m-1] in order
      cta_copy<real>(m, m, W_L, m, W_S, m);
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        // position of original row c after the swaps
        int pos = c;
        for (int j = 0; j < m; j++) {
          if (piv[j] == pos) pos = j;
          else if (j == pos) pos = piv[j];
        }
        for (int i = 0; i < m; i++) T[i + (int64_t)c * m] = W_S[i + (int64_t)pos * m];
      }
      __syncthreads();
      cta_tri_inv_upper<real>(m, W_A, m, W_L, m);
      // T'_R^T = (U^{-1})^T
      real* TRt = fac + tk.TR;
      for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        int i = idx % m, j = idx / m;
        TRt[i + (int64_t)j * m] = W_L[j + (int64_t)i * m];
      }
      __syncthreads();
    }
    return;
  }

  // ---- A_ss^{-1}
  if (sym) {
    cta_tri_inv_lower<real>(m, W_A, m, false, W_L, m);
    cta_gemm<real>(m, m, m, W_L, m, true, W_L, m, false, W_B, m, real(1), real(0));
  } else {
    // B = U^{-1} L^{-1} P
    cta_tri_inv_lower<real>(m, W_A, m, true, W_L, m);
    cta_tri_inv_upper<real>(m, W_A, m, W_S, m);
    cta_gemm<real>(m, m, m, W_S, m, false, W_L, m, false, W_F, m, real(1), real(0));
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      int pos = c;
      for (int j = 0; j < m; j++) {
        if (piv[j] == pos) pos = j;
        else if (j == pos) pos = piv[j];
      }
      for (int i = 0; i < m; i++) W_B[i + (int64_t)c * m] = W_F[i + (int64_t)pos * m];
    }
    __syncthreads();
  }

  // ---- U = first k columns of Q of the pivoted QR
  cta_form_q<real>(m, k, W_G, m, tau, 0, k, W_U, m);

  // ---- V_L: complement of X = B U (full QR of X, V = Q[:, k:])
  cta_gemm<real>(m, k, m, W_B, m, false, W_U, m, false, W_X, m, real(1), real(0));
  cta_householder_qr<real>(m, k, W_X, m, nrm2, orig, tau2, false, 0.0, k, 0.0, red_d, red_i);
  cta_form_q<real>(m, k, W_X, m, tau2, k, f, W_V, m);

  // ---- T = [U^T B; V_L^T B]
  cta_gemm<real>(k, m, m, W_U, m, true, W_B, m, false, W_T, m, real(1), real(0));
  cta_gemm<real>(f, m, m, W_V, m, true, W_B, m, false, W_T + k, m, real(1), real(0));
  // C = U^T B U (k x k) -> coarse (s,s) block
  cta_gemm<real>(k, k, m, W_T, m, false, W_U, m, false, W_C, m, real(1), real(0));
  real* blk_ss = arena + tk.a_ss;

  if (sym) {
    // F = V^T B V, Cholesky, T' rows k.. = L_F^{-1} V^T B
    cta_gemm<real>(f, f, m, W_T + k, m, false, W_V, m, false, W_F, m, real(1), real(0));
    if (!cta_cholesky<real>(f, W_F, m, &sflag)) {
      if (threadIdx.x == 0) {
        if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_NOT_SPD) == 0) {
          err->cluster = tk.s;
          err->level = level;
        }
        rank[tk.s] = m;
      }
      return;
    }
    cta_tri_inv_lower<real>(f, W_F, m, false, W_L, m);
    cta_copy<real>(k, m, W_T, m, T, m);
    cta_gemm<real>(f, m, f, W_L, m, false, W_T + k, m, false, T + k, m, real(1), real(0));
    // D = C U^T (k x m) for the coarse-to-far update C (U^T A_sw)
    cta_gemm<real>(k, m, k, W_C, m, false, W_U, m, true, ws_all + tk.D, m, real(1), real(0));
  } else {
    // V_R: complement of B^T U
    cta_gemm<real>(m, k, m, W_B, m, true, W_U, m, false, W_X, m, real(1), real(0));
    cta_householder_qr<real>(m, k, W_X, m, nrm2, orig, tau2, false, 0.0, k, 0.0, red_d, red_i);
    cta_form_q<real>(m, k, W_X, m, tau2, k, f, W_R, m);
    // F = V_L^T B V_R (f x f) and its LU
    cta_gemm<real>(f, f, m, W_T + k, m, false, W_R, m, false, W_F, m, real(1), real(0));
    if (!cta_lu<real>(f, W_F, m, piv, reinterpret_cast<real*>(red_d), red_i, &sflag)) {
      if (threadIdx.x == 0) {
        if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_SINGULAR) == 0) {
          err->cluster = tk.s;
          err->level = level;
        }
        rank[tk.s] = m;
      }
      return;
    }
    // T' rows k.. = L_F^{-1} P_F V_L^T B: permute rows of W_T[k:] by piv
    for (int j = 0; j < f; j++) {
      int p = piv[j];
      if (p != j)
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
          real t = W_T[k + j + (int64_t)c * m];
          W_T[k + j + (int64_t)c * m] = W_T[k + p + (int64_t)c * m];
          W_T[k + p + (int64_t)c * m] = t;
        }
      __syncthreads();
    }
    cta_tri_inv_lower<real>(f, W_F, m, true, W_L, m);
    cta_copy<real>(k, m, W_T, m, T, m);
    cta_gemm<real>(f, m, f, W_L, m, false, W_T + k, m, false, T + k, m, real(1), real(0));
    // T'_R = B [U, V_R U_F^{-1}]; store its transpose
    cta_tri_inv_upper<real>(f, W_F, m, W_L, m);
    cta_gemm<real>(m, f, f, W_R, m, false, W_L, m, false, W_S, m, real(1), real(0));  // V_R U_F^{-1}
    real* TRt = fac + tk.TR;
    // TRt rows 0..k = (B U)^T = U^T B^T ; rows k.. = (B V_R U_F^{-1})^T
    cta_gemm<real>(k, m, m, W_U, m, true, W_B, m, true, TRt, m, real(1), real(0));
    cta_gemm<real>(f, m, m, W_S, m, true, W_B, m, true, TRt + k, m, real(1), real(0));
    cta_gemm<real>(k, m, k, W_C, m, false, W_U, m, true, ws_all + tk.D, m, real(1), real(0));
    cta_gemm<real>(k, m, k, W_C, m, true, W_U, m, true, ws_all + tk.D2, m, real(1), real(0));
  }
  // write C into the (s,s) block (coarse part); done last: A_ss was copied
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    int i = idx % k, j = idx / k;
    blk_ss[i + (int64_t)j * tk.ld] = W_C[i + (int64_t)j * m];
  }
}

}  // namespace

template <typename real>
void Launch<real>::prep(const PrepTask* tasks_dev, int ntask, real* arena, real* fac, real* ws,
                        double* wsd, const int64_t* gptr, const int* gstr, int* rank, double eps,
                        int sym, int max_rank, int maxm, DevError* err, int level,
                        cudaStream_t st) {
  (void)maxm;
  if (ntask <= 0) return;
  // rounding-noise floor of the rank decision, relative to max |A_ss|: the
  // oracle's 1e-14 in float64; float32 blocks carry ~1e-7 relative noise
  const double noise_rtol = sizeof(real) == 8 ? 1e-14 : 1e-6;
  count_launch();
  prep_kernel<real><<<ntask, kPrepThreads, 0, st>>>(tasks_dev, arena, fac, ws, wsd, gptr, gstr,
                                                     rank, eps, noise_rtol, sym, max_rank, err,
                                                     level);
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
