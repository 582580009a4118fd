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
// accumulated in double.  The factor of A_ss and A_ss^{-1} live in shared
// memory when they fit (the host sizes the dynamic shared memory per class);
// everything else is in a per-cluster global workspace that stays in L2.
#include <cfloat>
#include <climits>
#include <cmath>

#include "common.h"

namespace hs {

namespace {

// threads of the per-cluster kernel: 512 in float32 (more warps share each
// barrier-separated step), 256 in float64 (register budget)
template <typename real>
struct PrepThreads {
  static constexpr int value = sizeof(real) == 4 ? 512 : 256;
};
constexpr double kPivotTieRtol = 1e-10;  // LU pivot search
// near-ties of the column-pivoted QR, relative: 1e-10 in float64; float32
// squared norms carry ~1e-7 relative rounding, so ties of exact arithmetic
// are recognised within 1e-5
template <typename real>
__device__ __forceinline__ double qr_tie_rtol() { return sizeof(real) == 8 ? 1e-10 : 1e-5; }
constexpr int GT = 64, GK = 16;  // CTA GEMM tile and inner chunk

template <typename real>
__device__ __forceinline__ real sqrt_(real x);
template <>
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

// C (M x N, ldc) = alpha * op(A) * op(B) + beta * C, whole CTA (NT =
// PrepThreads threads, 64 x 64 output tiles, GR x 4 outputs per thread with
// GR = 1024 / NT, inner chunks of 16 staged in shared memory `sh` of
// 2 * 16 * 65 reals).  C must not alias A or B.
template <typename real>
__device__ void cta_gemm(int M, int N, int K, const real* A, int lda, bool ta, const real* B,
                         int ldb, bool tb, real* C, int ldc, real alpha, real beta, real* sh) {
  constexpr int NT = PrepThreads<real>::value;
  constexpr int GR = 1024 / NT, RS = NT / 16;  // rows per thread, row stride
  real* As = sh;
  real* Bs = sh + GK * (GT + 1);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int i0 = 0; i0 < M; i0 += GT)
    for (int j0 = 0; j0 < N; j0 += GT) {
      real acc[GR][4];
#pragma unroll
      for (int p = 0; p < GR; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = 0;
      for (int l0 = 0; l0 < K; l0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
          int i, l;
          if (!ta) {
            i = e % GT;
            l = e / GT;
          } else {
            l = e % GK;
            i = e / GK;
          }
          int gi = i0 + i, gl = l0 + l;
          real v = 0;
          if (gi < M && gl < K) v = ta ? A[gl + (int64_t)gi * lda] : A[gi + (int64_t)gl * lda];
          As[l * (GT + 1) + i] = v;
        }
        for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
          int l, j;
          if (!tb) {
            l = e % GK;
            j = e / GK;
          } else {
            j = e % GT;
            l = e / GT;
          }
          int gl = l0 + l, gj = j0 + j;
          real v = 0;
          if (gl < K && gj < N) v = tb ? B[gj + (int64_t)gl * ldb] : B[gl + (int64_t)gj * ldb];
          Bs[l * (GT + 1) + j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < GK; l++) {
          real a[GR], b[4];
#pragma unroll
          for (int p = 0; p < GR; p++) a[p] = As[l * (GT + 1) + ty + RS * p];
#pragma unroll
          for (int q = 0; q < 4; q++) b[q] = Bs[l * (GT + 1) + tx + 16 * q];
#pragma unroll
          for (int p = 0; p < GR; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[p][q] += a[p] * b[q];
        }
        __syncthreads();
      }
#pragma unroll
      for (int p = 0; p < GR; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          int gi = i0 + ty + RS * p, gj = j0 + tx + 16 * q;
          if (gi < M && gj < N) {
            real c = alpha * acc[p][q];
            if (beta != real(0)) c += beta * C[gi + (int64_t)gj * ldc];
            C[gi + (int64_t)gj * ldc] = c;
          }
        }
    }
  __syncthreads();
}

// The helpers below map warps to columns and lanes to rows: column-major
// accesses are then contiguous across a warp, and no per-element index
// division is needed.
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int num_warps() { return blockDim.x >> 5; }

template <typename real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename real>
__device__ void cta_copy(int M, int N, const real* A, int64_t lda, real* B, int64_t ldb) {
  for (int j = warp_id(); j < N; j += num_warps())
    for (int i = lane_id(); i < M; i += 32) B[i + j * ldb] = A[i + j * lda];
  __syncthreads();
}

// Zero the strict upper (upper=true) or strict lower part of an n x n matrix.
template <typename real>
__device__ void cta_zero_tri(int n, real* A, int lda, bool upper) {
  for (int j = warp_id(); j < n; j += num_warps()) {
    const int i0 = upper ? 0 : j + 1, i1 = upper ? j : n;
    for (int i = i0 + lane_id(); i < i1; i += 32) A[i + (int64_t)j * lda] = 0;
  }
  __syncthreads();
}

template <typename real>
__device__ void cta_identity(int M, int N, int diag_off, real* A, int lda) {
  for (int j = warp_id(); j < N; j += num_warps())
    for (int i = lane_id(); i < M; i += 32)
      A[i + (int64_t)j * lda] = (i == j + diag_off) ? real(1) : real(0);
  __syncthreads();
}

// In-place lower Cholesky A = L L^T (lower triangle), right-looking, one
// barrier per step: step j subtracts a_ij a_lj / a_jj from the trailing lower
// triangle and, in the same phase, finishes column j-1 (scaling by
// 1/sqrt(d_{j-1})), which step j does not read.  Returns false on every
// thread for a non-positive pivot.
template <typename real>
__device__ bool cta_cholesky(int n, real* A, int lda, int* sflag) {
  (void)sflag;
  const int lane = lane_id(), warp = warp_id(), nw = num_warps();
  real rprev = 0;  // 1 / sqrt(d_{j-1})
  for (int j = 0; j < n; j++) {
    const real d = A[j + (int64_t)j * lda];
    if (!(d > real(0))) return false;  // uniform: every thread read the same d
    const real invd = real(1) / d;
    if (j > 0) {
      real* cp = A + (int64_t)(j - 1) * lda;
      for (int i = j + threadIdx.x; i < n; i += blockDim.x) cp[i] *= rprev;
    }
    const real* cj = A + (int64_t)j * lda;
    for (int l = j + 1 + warp; l < n; l += nw) {
      const real alj = cj[l] * invd;
      real* cl = A + (int64_t)l * lda;
      for (int i = l + lane; i < n; i += 32) cl[i] -= cj[i] * alj;
    }
    __syncthreads();
    // the diagonal of column j-1 was read as d in the previous step only
    if (j > 0 && threadIdx.x == 0) A[(j - 1) + (int64_t)(j - 1) * lda] = real(1) / rprev;
    rprev = real(1) / sqrt_(d);
  }
  if (n > 0 && threadIdx.x == 0) A[(n - 1) + (int64_t)(n - 1) * lda] = real(1) / rprev;
  __syncthreads();
  return true;
}

// In-place LU with partial pivoting, P A = L U (unit lower L).  piv[j] = row
// swapped with j at step j.  Near-ties (|a| >= (1 - 1e-10) max) go to the
// lowest row.  Returns false for an exactly zero pivot column.
__device__ double cta_max_d(double v, double* red);
__device__ int cta_min_i(int v, int* red);

template <typename real>
__device__ bool cta_lu(int n, real* A, int lda, int* piv, double* red_d, int* red_i,
                       int* sflag) {
  (void)sflag;
  const int lane = lane_id(), warp = warp_id(), nw = num_warps();
  for (int j = 0; j < n; j++) {
    double mx = 0;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x)
      mx = fmax(mx, fabs((double)A[i + (int64_t)j * lda]));
    mx = cta_max_d(mx, red_d);
    if (!(mx > 0.0)) return false;  // uniform
    int best = n;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x)
      if (fabs((double)A[i + (int64_t)j * lda]) >= (1.0 - kPivotTieRtol) * mx && i < best) best = i;
    const int p = cta_min_i(best, red_i);
    if (threadIdx.x == 0) piv[j] = p;
    if (p != j)
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        real t = A[j + (int64_t)c * lda];
        A[j + (int64_t)c * lda] = A[p + (int64_t)c * lda];
        A[p + (int64_t)c * lda] = t;
      }
    __syncthreads();
    // l_ij = a_ij / a_jj is formed on the fly by every column's update and
    // written back in the next phase
    const real rd = real(1) / A[j + (int64_t)j * lda];
    const real* cj = A + (int64_t)j * lda;
    for (int l = j + 1 + warp; l < n; l += nw) {
      real* cl = A + (int64_t)l * lda;
      const real ujl = cl[j];
      for (int i = j + 1 + lane; i < n; i += 32) cl[i] -= (cj[i] * rd) * ujl;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)j * lda] *= rd;
    __syncthreads();
  }
  return true;
}

// X = L^{-1} for lower triangular L (unit diagonal if `unit`), out of place:
// X (n x n, zero above the diagonal) starts as I and every step i subtracts
// l_ri x_ic for rows r > i from all columns c <= i (x_ic = x_ic / l_ii on the
// fly); row i is finished in the next phase.  One barrier per step.
template <typename real>
__device__ void cta_trtri_lower_oop(int n, const real* L, int ldl, bool unit, real* X, int ldx) {
  const int lane = lane_id(), warp = warp_id(), nw = num_warps();
  cta_identity<real>(n, n, 0, X, ldx);
  real dprev = 1;
  for (int i = 0; i < n; i++) {
    const real di = unit ? real(1) : real(1) / L[i + (int64_t)i * ldl];
    if (i > 0 && !unit)
      for (int c = threadIdx.x; c < i; c += blockDim.x) X[(i - 1) + (int64_t)c * ldx] *= dprev;
    const real* li = L + (int64_t)i * ldl;
    for (int c = warp; c <= i; c += nw) {
      real* xc = X + (int64_t)c * ldx;
      const real xic = xc[i] * di;
      for (int r = i + 1 + lane; r < n; r += 32) xc[r] -= li[r] * xic;
    }
    dprev = di;
    __syncthreads();
  }
  if (n > 0 && !unit)
    for (int c = threadIdx.x; c < n; c += blockDim.x) X[(n - 1) + (int64_t)c * ldx] *= dprev;
  __syncthreads();
}

// In-place inverse of an upper triangular matrix, column by column from the
// first.  tmp: n reals.
template <typename real>
__device__ void cta_trtri_upper(int n, real* U, int ld, real* tmp) {
  for (int j = 0; j < n; j++) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) tmp[i] = U[i + (int64_t)j * ld];
    if (threadIdx.x == 0) U[j + (int64_t)j * ld] = real(1) / U[j + (int64_t)j * ld];
    __syncthreads();
    const real d = U[j + (int64_t)j * ld];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      real acc = 0;
      for (int l = i; l < j; l++) acc += U[i + (int64_t)l * ld] * tmp[l];
      U[i + (int64_t)j * ld] = -acc * d;
    }
    __syncthreads();
  }
}

// Block reductions: shuffle within each warp, one exchange through shared
// memory (red: at least one slot per warp), two barriers.
__device__ double cta_max_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane_id() == 0) red[warp_id()] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < num_warps(); w++) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

__device__ int cta_min_i(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane_id() == 0) red[warp_id()] = v;
  __syncthreads();
  int r = red[0];
  for (int w = 1; w < num_warps(); w++) r = min(r, red[w]);
  __syncthreads();
  return r;
}

__device__ double cta_sum_d(double v, double* red) {
  v = warp_sum(v);
  if (lane_id() == 0) red[warp_id()] = v;
  __syncthreads();
  double r = 0;
  for (int w = 0; w < num_warps(); w++) r += red[w];
  __syncthreads();
  return r;
}

// Householder QR of the m x c matrix G (in place).  Element (i, q) sits at
// G[i * ldg + q] when RowMajor (one thread per column then reads coalesced
// across a warp), else at G[i + q * ldg].  With `pivot`, columns are pivoted
// by largest remaining norm (recomputed every step, near-ties to the lowest
// original index, orig[] tracks original indices), stopping at
// |r_jj| <= eps |r_11| (eps > 0), at |r_jj| <= floor (rounding noise of a
// block that is zero in exact arithmetic), at an all-zero remainder or at
// kmax steps.  Householder vectors stay in G (v_j in rows j..m of column j);
// tau[j] = 2 / v^T v.  vsh: m reals of shared memory.  Returns the number of
// steps.
template <typename real, bool RowMajor>
__device__ int cta_householder_qr(int m, int c, real* G, int ldg, double* nrm2, double* orig,
                                  real* tau, bool pivot, double eps, int kmax, double floor,
                                  double* red_d, int* red_i, real* vsh, real* rsign = nullptr,
                                  const int* fpiv = nullptr) {
  auto at = [&](int i, int q) -> real& {
    return RowMajor ? G[(int64_t)i * ldg + q] : G[i + (int64_t)q * ldg];
  };
  if (pivot) {
    for (int q = threadIdx.x; q < c; q += blockDim.x) {
      real s = 0;
      for (int i = 0; i < m; i++) {
        const real v = at(i, q);
        s += v * v;
      }
      nrm2[q] = (double)s;
      orig[q] = q;
    }
    __syncthreads();
  }
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
      if (fpiv) {
        // a given pivot order (forced-rank factorization) replaces the search
        best = j < kmax ? fpiv[j] : INT_MAX;
      } else {
        for (int t = j + threadIdx.x; t < c; t += blockDim.x)
          if (nrm2[t] >= (1.0 - qr_tie_rtol<real>()) * mx) best = min(best, (int)orig[t]);
        best = cta_min_i(best, red_i);
      }
      if (threadIdx.x == 0) red_i[blockDim.x] = -1;
      __syncthreads();
      for (int t = j + threadIdx.x; t < c; t += blockDim.x)
        if ((int)orig[t] == best) red_i[blockDim.x] = t;
      __syncthreads();
      q = red_i[blockDim.x];
      __syncthreads();
      if (q < 0) break;  // the given pivot names no remaining column
      r = sqrt(nrm2[q]);
      if (j == 0) r11 = r;
      if (r <= floor) break;
      if (eps > 0.0 && r <= eps * r11) break;
      if (j >= kmax) break;
      if (q != j) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          real t = at(i, j);
          at(i, j) = at(i, q);
          at(i, q) = t;
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
      double s = 0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        double x = at(i, j);
        s += x * x;
      }
      r = sqrt(cta_sum_d(s, red_d));
    }
    // reflector v = x - beta e1, beta = -sign(x0) ||x||, tau = 2 / v^T v
    const double x0 = (double)at(j, j);
    const double beta = (x0 >= 0.0) ? -r : r;
    const double tj = (r > 0.0) ? 1.0 / (r * (r + fabs(x0))) : 0.0;
    __syncthreads();
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) vsh[i] = (i == j) ? (real)(x0 - beta) : at(i, j);
    __syncthreads();
    if (threadIdx.x == 0) {
      at(j, j) = (real)(x0 - beta);
      tau[j] = (real)tj;
      if (rsign) rsign[j] = beta < 0.0 ? real(-1) : real(1);
    }
    const real rt = (real)tj;
    // apply to the remaining columns, CB columns per thread and RB rows per
    // batch of independent loads (memory-level parallelism); recompute the
    // squared norms over rows j+1..m
    constexpr int CB = 4, RB = 4;
    const int nth = blockDim.x;
    for (int t0 = j + 1 + threadIdx.x; t0 < c; t0 += nth * CB) {
      real w[CB];
      bool ok[CB];
#pragma unroll
      for (int g = 0; g < CB; g++) {
        w[g] = 0;
        ok[g] = (t0 + g * nth) < c;
      }
      for (int i = j; i < m; i += RB) {
        real x[RB][CB];
#pragma unroll
        for (int rr = 0; rr < RB; rr++)
#pragma unroll
          for (int g = 0; g < CB; g++)
            x[rr][g] = (ok[g] && i + rr < m) ? at(i + rr, t0 + g * nth) : real(0);
#pragma unroll
        for (int rr = 0; rr < RB; rr++) {
          const real vi = (i + rr < m) ? vsh[i + rr] : real(0);
#pragma unroll
          for (int g = 0; g < CB; g++) w[g] += vi * x[rr][g];
        }
      }
      // squared norms in the working precision: a float64 FMA per element
      // here would bound the float32 path by the float64 rate
      real sq[CB];
#pragma unroll
      for (int g = 0; g < CB; g++) {
        w[g] *= rt;
        sq[g] = 0;
      }
      for (int i = j; i < m; i += RB) {
        real x[RB][CB];
#pragma unroll
        for (int rr = 0; rr < RB; rr++)
#pragma unroll
          for (int g = 0; g < CB; g++)
            x[rr][g] = (ok[g] && i + rr < m) ? at(i + rr, t0 + g * nth) : real(0);
#pragma unroll
        for (int rr = 0; rr < RB; rr++) {
          if (i + rr >= m) break;
          const real vi = vsh[i + rr];
#pragma unroll
          for (int g = 0; g < CB; g++) {
            if (!ok[g]) continue;
            const real v = x[rr][g] - w[g] * vi;
            at(i + rr, t0 + g * nth) = v;
            if (i + rr > j) sq[g] += v * v;
          }
        }
      }
      if (pivot)
#pragma unroll
        for (int g = 0; g < CB; g++)
          if (ok[g]) nrm2[t0 + g * nth] = (double)sq[g];
    }
    __syncthreads();
    k = j + 1;
  }
  __syncthreads();
  return k;
}

// Q[:, c0:c0+ncols] of Q = H_0 .. H_{k-1} (H_j = I - tau_j v_j v_j^T, v_j in
// rows j..m of column j of V): out (m x ncols) starts as the identity columns
// c0.. and receives the reflectors in reverse order.  One warp per group of
// four columns; lane l owns rows l, l + 32, ... of them (held in registers
// when m <= 256), so the warps never wait for one another and the lanes only
// exchange the four dot products of each reflector (shuffles).
template <typename real, bool RowMajor>
__device__ void cta_form_q(int m, int k, const real* V, int ldv, const real* tau, int c0,
                           int ncols, real* out, int ldo, real* vsh) {
  (void)vsh;
  constexpr int CW = 4, R = 8;
  const int lane = lane_id(), warp = warp_id(), nw = num_warps();
  auto vat = [&](int i, int j) -> real {
    return RowMajor ? V[(int64_t)i * ldv + j] : V[i + (int64_t)j * ldv];
  };
  for (int g0 = warp * CW; g0 < ncols; g0 += nw * CW) {
    const int ng = min(CW, ncols - g0);
    if (m <= 32 * R) {
      real x[R][CW];
#pragma unroll
      for (int r = 0; r < R; r++)
#pragma unroll
        for (int g = 0; g < CW; g++) x[r][g] = (lane + 32 * r == c0 + g0 + g) ? real(1) : real(0);
      for (int j = k - 1; j >= 0; j--) {
        const real tj = tau[j];
        real v[R], d[CW];
#pragma unroll
        for (int g = 0; g < CW; g++) d[g] = 0;
#pragma unroll
        for (int r = 0; r < R; r++) {
          const int i = lane + 32 * r;
          v[r] = (i >= j && i < m) ? vat(i, j) : real(0);
#pragma unroll
          for (int g = 0; g < CW; g++) d[g] += v[r] * x[r][g];
        }
#pragma unroll
        for (int g = 0; g < CW; g++) d[g] = warp_sum(d[g]) * tj;
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
          for (int g = 0; g < CW; g++) x[r][g] -= d[g] * v[r];
      }
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int i = lane + 32 * r;
        if (i < m)
#pragma unroll
          for (int g = 0; g < CW; g++)
            if (g < ng) out[i + (int64_t)(g0 + g) * ldo] = x[r][g];
      }
    } else {
      for (int g = 0; g < ng; g++)
        for (int i = lane; i < m; i += 32)
          out[i + (int64_t)(g0 + g) * ldo] = (i == c0 + g0 + g) ? real(1) : real(0);
      for (int j = k - 1; j >= 0; j--) {
        const real tj = tau[j];
        real d[CW];
#pragma unroll
        for (int g = 0; g < CW; g++) d[g] = 0;
        for (int i = lane; i < m; i += 32) {
          if (i < j) continue;
          const real v = vat(i, j);
#pragma unroll
          for (int g = 0; g < CW; g++)
            if (g < ng) d[g] += v * out[i + (int64_t)(g0 + g) * ldo];
        }
#pragma unroll
        for (int g = 0; g < CW; g++) d[g] = warp_sum(d[g]) * tj;
        for (int i = lane; i < m; i += 32) {
          if (i < j) continue;
          const real v = vat(i, j);
#pragma unroll
          for (int g = 0; g < CW; g++)
            if (g < ng) out[i + (int64_t)(g0 + g) * ldo] -= d[g] * v;
        }
      }
    }
  }
  __syncthreads();
}

// Householder QR without pivoting of the m x k matrix X (column-major, in
// place): v_j in rows j..m of column j (its head x_jj - beta, beta =
// -sign(x_jj) ||x_j||), tau[j] = 1 / (r (r + |x_jj|)).  Step j: the warp
// owning column j forms the reflector; after a barrier every warp applies it
// to its columns t > j, four at a time (lanes over rows, shuffled dots).
template <typename real>
__device__ void cta_qr_np(int m, int k, real* X, int ldx, real* tau) {
  constexpr int CW = 4;
  const int lane = lane_id(), warp = warp_id(), nw = num_warps();
  for (int j = 0; j < k; j++) {
    if (warp == j % nw) {
      real* xj = X + (int64_t)j * ldx;
      real sq = 0;
      for (int i = j + lane; i < m; i += 32) sq += xj[i] * xj[i];
      sq = warp_sum(sq);
      const double r = sqrt((double)sq);
      const double x0 = (double)xj[j];
      const double beta = (x0 >= 0.0) ? -r : r;
      const double tj = (r > 0.0) ? 1.0 / (r * (r + fabs(x0))) : 0.0;
      __syncwarp();
      if (lane == 0) {
        xj[j] = (real)(x0 - beta);
        tau[j] = (real)tj;
      }
    }
    __syncthreads();
    const real* vj = X + (int64_t)j * ldx;
    const real tj = tau[j];
    for (int t0 = j + 1 + warp; t0 < k; t0 += nw * CW) {
      real d[CW];
#pragma unroll
      for (int g = 0; g < CW; g++) d[g] = 0;
      for (int i = j + lane; i < m; i += 32) {
        const real v = vj[i];
#pragma unroll
        for (int g = 0; g < CW; g++) {
          const int t = t0 + g * nw;
          if (t < k) d[g] += v * X[i + (int64_t)t * ldx];
        }
      }
#pragma unroll
      for (int g = 0; g < CW; g++) d[g] = warp_sum(d[g]) * tj;
      for (int i = j + lane; i < m; i += 32) {
        const real v = vj[i];
#pragma unroll
        for (int g = 0; g < CW; g++) {
          const int t = t0 + g * nw;
          if (t < k) X[i + (int64_t)t * ldx] -= d[g] * v;
        }
      }
    }
    __syncthreads();
  }
}

// Column permutation of the LU inverse: (X P)[:, c] = X[:, pos(c)], pos(c) =
// row of P A holding original row c after the swaps piv[0..n-1] in order.
template <typename real>
__device__ void cta_permute_cols(int n, const int* piv, const real* X, int ldx, real* Y, int ldy) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    int pos = c;
    for (int j = 0; j < n; j++) {
      if (piv[j] == pos) pos = j;
      else if (j == pos) pos = piv[j];
    }
    for (int i = 0; i < n; i++) Y[i + (int64_t)c * ldy] = X[i + (int64_t)pos * ldx];
  }
  __syncthreads();
}

template <typename real>
__device__ void report(DevError* err, int code, int s, int level, int* rank, int m) {
  if (threadIdx.x == 0) {
    if (atomicCAS(&err->code, 0, code) == 0) {
      err->cluster = s;
      err->level = level;
    }
    rank[s] = m;  // leave the cluster untouched downstream
  }
}

template <typename real>
__global__ void __launch_bounds__(PrepThreads<real>::value)
prep_kernel(const PrepTask* __restrict__ tasks, real* __restrict__ arena, real* __restrict__ fac,
            real* __restrict__ ws_all, double* __restrict__ wsd_all,
            const Seg* __restrict__ segs, int* rank, int* __restrict__ piv_all,
            const int* __restrict__ fpiv, double eps, double noise_rtol, int sym, int max_rank,
            int smem_mats, int smem_m,
            DevError* err, int level, long long* dbg) {
  __shared__ double red_d[PrepThreads<real>::value];
  __shared__ int red_i[PrepThreads<real>::value + 1];
  __shared__ int sflag;
  __shared__ int s_ncol;
  __shared__ double s_amax;
  __shared__ real gsh[2 * GK * (GT + 1)];
  extern __shared__ unsigned char dsm[];
  const PrepTask tk = tasks[blockIdx.x];
  const int m = tk.m;
  // optional per-phase clock stamps (profiling): dbg[task * 8 + checkpoint]
  long long* stamp = dbg ? dbg + (int64_t)blockIdx.x * 8 : nullptr;
  auto mark = [&](int i) {
    if (stamp && threadIdx.x == 0) stamp[i] = clock64();
  };
  mark(0);
  if (threadIdx.x == 0) sflag = 0;
  __syncthreads();
  const int64_t mm = (int64_t)m * m;
  real* ws = ws_all + tk.ws;
  real* smat = reinterpret_cast<real*>(dsm);
  real* vsh = smat + (int64_t)smem_mats * (smem_m | 1) * smem_m;  // m reals
  real* tsh = vsh + smem_m;                                  // m reals
  // shared-memory matrices get an odd leading dimension: loops that give one
  // column to each thread then touch 32 different banks
  const int64_t reg = (int64_t)(smem_m | 1) * smem_m;  // one shared region
  int ldA = smem_mats >= 1 ? (m | 1) : m;
  int ldB = smem_mats >= 2 ? (m | 1) : m;
  const int ldU = smem_mats >= 3 ? (m | 1) : m;
  real* W_A = smem_mats >= 1 ? smat : ws;                  // A_ss -> factor -> inverse factor
  real* W_B = smem_mats >= 2 ? smat + reg : ws + mm;       // A_ss^{-1}
  // [U V_L] as one m x m matrix: U in columns 0..k, V_L in columns k..m
  real* W_U = smem_mats >= 3 ? smat + 2 * reg : ws + 2 * mm;
  real* W_X = ws + 3 * mm;   // X = B U, then its reflectors
  real* W_V = W_U + (int64_t)0;  // V_L = columns k..m of W_U (set below)
  real* W_T = ws + 4 * mm;   // [U V_L]^T B
  real* W_F = W_T + mm;      // F, then its factor / inverse factor (general)
  real* W_L = W_F + mm;      // general: L^{-1} P, (U_F^{-1})
  real* W_C = W_L + mm;      // C = U^T B U
  real* W_R = W_C + mm;      // general: V_R
  real* W_S = W_R + mm;      // general: scratch
  real* W_G = W_S + mm;      // G (m x ncolG)
  double* nrm2 = wsd_all + tk.wsd;
  double* orig = nrm2 + tk.ncolG;
  real* tau = reinterpret_cast<real*>(orig + tk.ncolG);
  real* tau2 = tau + m;
  real* rsign = tau2 + m;  // sign of R's diagonal in the pivoted QR
  int* piv = reinterpret_cast<int*>(rsign + m);
  real* T = fac + tk.T;

  // ---- A_ss, its largest magnitude (scale of the noise floor), its factor
  cta_copy<real>(m, m, arena + tk.a_ss, tk.ld, W_A, ldA);
  {
    double mx = 0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x)
      mx = fmax(mx, fabs((double)W_A[idx % m + (int64_t)(idx / m) * ldA]));
    mx = cta_max_d(mx, red_d);
    if (threadIdx.x == 0) s_amax = mx;
    __syncthreads();
  }
  const bool ok = sym ? cta_cholesky<real>(m, W_A, ldA, &sflag)
                      : cta_lu<real>(m, W_A, ldA, piv, red_d, red_i, &sflag);
  if (!ok) {
    report<real>(err, sym ? (int)HSOLVE_ERR_NOT_SPD : (int)HSOLVE_ERR_SINGULAR, tk.s, level, rank, m);
    return;
  }

  mark(1);
  const bool sketched = tk.l > 0;
  const bool qr_done = tk.qr == 2;  // done by the thread-block-cluster kernel
  // ---- gather the nonzero fill columns into G (Eq. lra input), row-major
  // (not needed when the pivoted QR runs on the sketch Y = G Omega or was
  // done by the cluster kernel)
  if (!sketched && !qr_done) {
    const int nc = tk.ncolG;
    // flag nonzero columns: one thread per column, batched independent loads
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      int64_t p;
      int st;
      seg_col(segs + tk.gcol, tk.ngcol, q, &p, &st);
      bool nz = false;
      for (int i = 0; i < m; i += 8) {
        real x[8];
#pragma unroll
        for (int rr = 0; rr < 8; rr++) x[rr] = (i + rr < m) ? arena[p + (int64_t)(i + rr) * st] : real(0);
#pragma unroll
        for (int rr = 0; rr < 8; rr++) nz |= (x[rr] != real(0));
      }
      orig[q] = nz ? 1.0 : 0.0;
    }
    __syncthreads();
    // exclusive scan of the flags: contiguous chunk per thread
    const int per = (nc + blockDim.x - 1) / blockDim.x;
    const int c0 = min(nc, (int)threadIdx.x * per), c1 = min(nc, c0 + per);
    int cnt = 0;
    for (int q = c0; q < c1; q++) cnt += (orig[q] != 0.0);
    red_i[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int t = 0; t < (int)blockDim.x; t++) {
        int v = red_i[t];
        red_i[t] = acc;
        acc += v;
      }
      s_ncol = acc;
    }
    __syncthreads();
    int dst = red_i[threadIdx.x];
    for (int q = c0; q < c1; q++) orig[q] = (orig[q] != 0.0) ? (double)(dst++) : -1.0;
    __syncthreads();
    const int ncomp = s_ncol;
    // copy: one thread per column; consecutive threads write consecutive
    // entries of a row of the row-major G
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      const int d = (int)orig[q];
      if (d < 0) continue;
      int64_t p;
      int st;
      seg_col(segs + tk.gcol, tk.ngcol, q, &p, &st);
      for (int i = 0; i < m; i += 8) {
        real x[8];
#pragma unroll
        for (int rr = 0; rr < 8; rr++) x[rr] = (i + rr < m) ? arena[p + (int64_t)(i + rr) * st] : real(0);
#pragma unroll
        for (int rr = 0; rr < 8; rr++)
          if (i + rr < m) W_G[(int64_t)(i + rr) * ncomp + d] = x[rr];
      }
    }
    __syncthreads();
  }
  mark(2);
  const int ncol = sketched ? tk.l : s_ncol;
  int k = 0;
  int kmax = m;
  if (max_rank > 0) kmax = min(kmax, max_rank);
  if (max_rank < 0) {  // forced rank (set by the host in rank[s]): no eps, no floor
    kmax = min(kmax, rank[tk.s]);
    eps = 0.0;
    noise_rtol = 0.0;
  }
  if (qr_done) {
    k = rank[tk.s];
  } else if (sketched) {
    // pivoted QR of the sketch (column-major m x l), in the shared memory of
    // the not yet used A_ss^{-1} and [U V] buffers when it fits; the kept
    // reflectors then move to W_G (column-major, ld m) for U
    real* Ysrc = ws_all + tk.Y;
    const bool ysm = smem_mats >= 3 && (int64_t)(m | 1) * tk.l <= 2 * reg;
    real* Yq = ysm ? W_B : Ysrc;
    const int ldY = ysm ? (m | 1) : m;
    if (ysm) cta_copy<real>(m, tk.l, Ysrc, m, Yq, ldY);
    k = cta_householder_qr<real, false>(m, tk.l, Yq, ldY, nrm2, orig, tau, true, eps, kmax,
                                        noise_rtol * s_amax, red_d, red_i, vsh, rsign,
                                        fpiv ? fpiv + tk.pv : nullptr);
    cta_copy<real>(m, k, Yq, ldY, W_G, m);
  } else if (ncol > 0) {
    k = cta_householder_qr<real, true>(m, ncol, W_G, ncol, nrm2, orig, tau, true, eps, kmax,
                                       noise_rtol * s_amax, red_d, red_i, vsh, rsign,
                                       fpiv ? fpiv + tk.pv : nullptr);
  }
  __syncthreads();
  if (threadIdx.x == 0) rank[tk.s] = k;
  // pivot order (the cluster kernel recorded its own): orig[j] is the
  // compacted (or sketch) column chosen at step j
  if (!qr_done)
    for (int j = threadIdx.x; j < k; j += blockDim.x) piv_all[tk.pv + j] = (int)orig[j];
  mark(3);
  if (k == m) return;  // untouched: all unknowns coarse, E_s = I
  const int f = m - k;

  if (sym) {
    // L^{-1} into the home of A_ss^{-1}, then B = L^{-T} L^{-1} into the
    // home of the (spent) factor; the two buffers then trade names
    cta_trtri_lower_oop<real>(m, W_A, ldA, false, W_B, ldB);
    if (k == 0) {  // E_s = I: T' = L^{-1}
      cta_copy<real>(m, m, W_B, ldB, T, m);
      return;
    }
    cta_gemm<real>(m, m, m, W_B, ldB, true, W_B, ldB, false, W_A, ldA, real(1), real(0), gsh);
    real* tp = W_A;
    W_A = W_B;
    W_B = tp;
    const int tl = ldA;
    ldA = ldB;
    ldB = tl;
  } else {
    // L^{-1} (unit lower) into W_L, U^{-1} into W_S
    cta_trtri_lower_oop<real>(m, W_A, ldA, true, W_L, m);
    cta_copy<real>(m, m, W_A, ldA, W_S, m);
    cta_trtri_upper<real>(m, W_S, m, tsh);
    cta_zero_tri<real>(m, W_S, m, false);
    if (k == 0) {
      // E_s = I: T' = L^{-1} P, T'_R^T = (U^{-1})^T
      cta_permute_cols<real>(m, piv, W_L, m, T, m);
      real* TRt = fac + tk.TR;
      for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        int i = idx % m, j = idx / m;
        TRt[i + (int64_t)j * m] = W_S[j + (int64_t)i * m];
      }
      __syncthreads();
      return;
    }
    // B = U^{-1} L^{-1} P
    cta_gemm<real>(m, m, m, W_S, m, false, W_L, m, false, W_F, m, real(1), real(0), gsh);
    cta_permute_cols<real>(m, piv, W_F, m, W_B, ldB);
  }

  mark(4);
  // ---- U = first k columns of Q of the pivoted QR
  if (sketched || qr_done)
    cta_form_q<real, false>(m, k, W_G, m, tau, 0, k, W_U, ldU, vsh);
  else
    cta_form_q<real, true>(m, k, W_G, ncol, tau, 0, k, W_U, ldU, vsh);
  // orient U so that R has a positive diagonal (Gram-Schmidt directions)
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
    int i = idx % m, j = idx / m;
    W_U[i + (int64_t)j * ldU] *= rsign[j];
  }
  __syncthreads();

  // ---- V_L: complement of X = B U (full QR of X, V = Q[:, k:]); in the SPD
  // case X takes the (spent) shared-memory home of the factor of A_ss
  int ldX = m;
  if (sym) {
    W_X = W_A;
    ldX = ldA;
  }
  cta_gemm<real>(m, k, m, W_B, ldB, false, W_U, ldU, false, W_X, ldX, real(1), real(0), gsh);
  cta_qr_np<real>(m, k, W_X, ldX, tau2);
  W_V = W_U + (int64_t)k * ldU;
  cta_form_q<real, false>(m, k, W_X, ldX, tau2, k, f, W_V, ldU, vsh);

  mark(5);
  // ---- T = [U V_L]^T B (one product); C = U^T B U -> coarse (s,s) block
  cta_gemm<real>(m, m, m, W_U, ldU, true, W_B, ldB, false, W_T, m, real(1), real(0), gsh);
  cta_gemm<real>(k, k, m, W_T, m, false, W_U, ldU, false, W_C, m, real(1), real(0), gsh);

  if (sym) {
    // F = V^T B V; L_F^{-1}; T' rows k.. = L_F^{-1} V^T B.  F lives where the
    // factor of A_ss was (shared memory when it fits): that factor is spent.
    W_F = W_A;
    const int ldF = ldA;
    mark(6);
    cta_gemm<real>(f, f, m, W_T + k, m, false, W_V, ldU, false, W_F, ldF, real(1), real(0), gsh);
    if (!cta_cholesky<real>(f, W_F, ldF, &sflag)) {
      report<real>(err, (int)HSOLVE_ERR_NOT_SPD, tk.s, level, rank, m);
      return;
    }
    cta_trtri_lower_oop<real>(f, W_F, ldF, false, W_L, m);
    cta_copy<real>(k, m, W_T, m, T, m);
    cta_gemm<real>(f, m, f, W_L, m, false, W_T + k, m, false, T + k, m, real(1), real(0), gsh);
    // D = C U^T (k x m) for the coarse-to-far update C (U^T A_sw)
    cta_gemm<real>(k, m, k, W_C, m, false, W_U, ldU, true, ws_all + tk.D, m, real(1), real(0),
                   gsh);
  } else {
    // V_R: complement of B^T U
    cta_gemm<real>(m, k, m, W_B, ldB, true, W_U, ldU, false, W_X, m, real(1), real(0), gsh);
    cta_qr_np<real>(m, k, W_X, m, tau2);
    cta_form_q<real, false>(m, k, W_X, m, tau2, k, f, W_R, m, vsh);
    // F = V_L^T B V_R (f x f) and its LU
    cta_gemm<real>(f, f, m, W_T + k, m, false, W_R, m, false, W_F, m, real(1), real(0), gsh);
    if (!cta_lu<real>(f, W_F, m, piv, red_d, red_i, &sflag)) {
      report<real>(err, (int)HSOLVE_ERR_SINGULAR, tk.s, level, rank, m);
      return;
    }
    // T' rows k.. = L_F^{-1} P_F V_L^T B: permute rows of W_T[k:] by piv
    for (int j = 0; j < f; j++) {
      const int p = piv[j];
      if (p != j)
        for (int c = threadIdx.x; c < m; c += blockDim.x) {
          real t = W_T[k + j + (int64_t)c * m];
          W_T[k + j + (int64_t)c * m] = W_T[k + p + (int64_t)c * m];
          W_T[k + p + (int64_t)c * m] = t;
        }
      __syncthreads();
    }
    cta_trtri_lower_oop<real>(f, W_F, m, true, W_L, m);
    cta_copy<real>(k, m, W_T, m, T, m);
    cta_gemm<real>(f, m, f, W_L, m, false, W_T + k, m, false, T + k, m, real(1), real(0), gsh);
    // T'_R = B [U, V_R U_F^{-1}]; store its transpose
    cta_trtri_upper<real>(f, W_F, m, tsh);
    cta_zero_tri<real>(f, W_F, m, false);
    cta_gemm<real>(m, f, f, W_R, m, false, W_F, m, false, W_S, m, real(1), real(0), gsh);
    real* TRt = fac + tk.TR;
    cta_gemm<real>(k, m, m, W_U, ldU, true, W_B, ldB, true, TRt, m, real(1), real(0), gsh);
    cta_gemm<real>(f, m, m, W_S, m, true, W_B, ldB, true, TRt + k, m, real(1), real(0), gsh);
    cta_gemm<real>(k, m, k, W_C, m, false, W_U, ldU, true, ws_all + tk.D, m, real(1), real(0),
                   gsh);
    cta_gemm<real>(k, m, k, W_C, m, true, W_U, ldU, true, ws_all + tk.D2, m, real(1), real(0),
                   gsh);
  }
  // write C into the (s,s) block (coarse part); done last: A_ss was copied
  real* blk_ss = arena + tk.a_ss;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    int i = idx % k, j = idx / k;
    blk_ss[i + (int64_t)j * tk.ld] = W_C[i + (int64_t)j * m];
  }
  mark(7);
}

}  // namespace

template <typename real>
void Launch<real>::prep(const PrepTask* tasks_dev, int ntask, real* arena, real* fac, real* ws,
                        double* wsd, const Seg* segs, int* rank, int* piv, const int* fpiv,
                        double eps,
                        int sym, int max_rank, int maxm, DevError* err, int level,
                        long long* dbg, cudaStream_t st) {
  if (ntask <= 0) return;
  // rounding-noise floor of the rank decision, relative to max |A_ss|: the
  // oracle's 1e-14 in float64; float32 blocks carry ~1e-7 relative noise
  const double noise_rtol = sizeof(real) == 8 ? 1e-14 : 1e-6;
  // the factor of A_ss and A_ss^{-1} in shared memory when they fit
  const size_t budget = 220 * 1024 - 2 * GK * (GT + 1) * sizeof(real) - 4 * 1024;
  const size_t one = sizeof(real) * (size_t)(maxm | 1) * maxm;
  const size_t vec = sizeof(real) * 2 * (size_t)maxm;
  int mats = 0;
  if (3 * one + vec <= budget) mats = 3;
  else if (2 * one + vec <= budget) mats = 2;
  else if (one + vec <= budget) mats = 1;
  const size_t smem = mats * one + vec;
  // the limit is raised once to the budget and never lowered: host threads
  // factoring different matrices launch this kernel concurrently
  static const bool limit_set = [budget] {
    cudaFuncSetAttribute(prep_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)budget);
    return true;
  }();
  (void)limit_set;
  count_launch();
  prep_kernel<real><<<ntask, PrepThreads<real>::value, smem, st>>>(tasks_dev, arena, fac, ws, wsd, segs,
                                                        rank, piv, fpiv, eps, noise_rtol, sym, max_rank, mats,
                                                        maxm, err, level, dbg);
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
