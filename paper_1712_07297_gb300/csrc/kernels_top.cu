// Dense top factorization (Alg. 1: "factorize A with the conventional
// Cholesky factorization" once the remaining system is small enough), for an
// SPD top block too large for one CTA: blocked right-looking Cholesky over
// 64-column panels (one CTA factors the diagonal block, a launch of CTAs
// solves the panel, a launch updates the trailing lower triangle), then the
// explicit inverse factor X = L^{-1} by block rows (one launch per block
// row, one CTA per block column), which the substitution sweeps apply as
// dense products.  Matrices are column-major in global memory.
#include <algorithm>

#include "common.h"

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
// X_ij = L_ii^{-1} (delta_ij I - sum_{k=j}^{i-1} L_ik X_kj).
template <typename real>
__global__ void __launch_bounds__(256)
trtri_row_kernel(const real* L, int64_t ld, real* X, int64_t ldx, int n, int i) {
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
      Bs[l][a] = (a < bc) ? X[gl + (int64_t)(c0 + a) * ldx] : real(0);
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
      S[c][a] = v / Ld[a][a];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < br * bc; e += 256) {
    int a = e % br, c = e / br;
    X[(r0 + a) + (int64_t)(c0 + c) * ldx] = S[c][a];
  }
}

template <typename real>
__global__ void zero_upper_kernel(real* X, int64_t ldx, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % n), j = (int)(e / n);
    if (i < j) X[i + (int64_t)j * ldx] = 0;
  }
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
  zero_upper_kernel<real><<<152 * 4, 256, 0, st>>>(X, n, n);
  for (int i = 0; i < nblk; i++) {
    count_launch();
    trtri_row_kernel<real><<<i + 1, 256, 0, st>>>(A, lda, X, n, n, i);
  }
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
