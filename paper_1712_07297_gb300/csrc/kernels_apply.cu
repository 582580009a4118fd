// Substitution sweeps of Alg. 2, one colour class per group of launches.
//
// Forward (y <- W_s y for the clusters of a class):
//   fwd_t    z_s = T' y_s, T' = diag(I, L_F^{-1} [P_F]) [U V_L]^T A_ss^{-1}
//            (rows split over CTAs)
//   fwd_nbr  y_N -= B_L z_f (columns split over CTAs), and y_s = z_s
// Backward (x <- W_s^T x):
//   bwd_part partial sums of B_R x_N over column chunks (deterministic order)
//   bwd_z    z_s = [x_c; x_f - sum of partials]
//   bwd_t    x_s = T_R'^T z_s (rows split over CTAs)
// Clusters of one class touch disjoint slots (their neighbour sets are
// disjoint, Sec. 3.2), so no atomics are needed.  z and the partial sums are
// level-sized scratch vectors owned by the factorization.
#include <algorithm>

#include "common.h"

namespace hs {

namespace {

constexpr int kRows = 64;   // output rows per CTA in the T' products
constexpr int kCols = 64;   // neighbour columns per CTA

template <typename real>
__global__ void __launch_bounds__(256)
fwd_t_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ fac, const real* __restrict__ y, real* __restrict__ z,
             int64_t ldy, int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  real* ys = reinterpret_cast<real*>(smem_raw);
  __shared__ real red[256];
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m;
  if (rc.k == m) return;
  const int i0 = blockIdx.x * kRows;
  if (i0 >= m) return;
  const real* T = fac + rc.T;
  const int ii = threadIdx.x % kRows, part = threadIdx.x / kRows;  // 4 parts over l
  const int i = i0 + ii;
  for (int r = 0; r < nrhs; r++) {
    const real* yr = y + rc.voff + (int64_t)r * ldy;
    for (int l = threadIdx.x; l < m; l += blockDim.x) ys[l] = yr[l];
    __syncthreads();
    real acc = 0;
    if (i < m)
      for (int l = part; l < m; l += 4) acc += T[i + (int64_t)l * m] * ys[l];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (part == 0 && i < m)
      z[rc.voff + i + (int64_t)r * ldy] = red[ii] + red[ii + 64] + red[ii + 128] + red[ii + 192];
    __syncthreads();
  }
}

template <typename real>
__global__ void __launch_bounds__(256)
fwd_nbr_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
               const real* __restrict__ fac, const int64_t* __restrict__ vmap,
               real* __restrict__ y, const real* __restrict__ z, int64_t ldy, int nrhs) {
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  if (blockIdx.x == 0)
    for (int r = 0; r < nrhs; r++)
      for (int i = threadIdx.x; i < m; i += blockDim.x)
        y[rc.voff + i + (int64_t)r * ldy] = z[rc.voff + i + (int64_t)r * ldy];
  const int c0 = blockIdx.x * kCols;
  if (c0 >= rc.nw) return;
  const int c1 = min(rc.nw, c0 + kCols);
  const real* BL = fac + (rc.sym ? rc.Y : rc.XT) + k;  // column c: B_L[c, :]
  const int64_t* vm = vmap + rc.map;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int r = 0; r < nrhs; r++) {
    const real* zf = z + rc.voff + k + (int64_t)r * ldy;
    for (int c = c0 + warp; c < c1; c += nwarp) {
      const real* col = BL + (int64_t)c * m;
      real acc = 0;
      for (int i = lane; i < f; i += 32) acc += col[i] * zf[i];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) y[vm[c] + (int64_t)r * ldy] -= acc;
    }
  }
}

template <typename real>
__global__ void __launch_bounds__(256)
bwd_part_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
                const real* __restrict__ fac, const int64_t* __restrict__ vmap,
                const real* __restrict__ y, real* __restrict__ part, int64_t ldy, int nrhs) {
  __shared__ real xn[kCols];
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const int c0 = blockIdx.x * kCols;
  if (c0 >= rc.nw) return;
  const int nc = min(rc.nw, c0 + kCols) - c0;
  const int nchunk = (rc.nw + kCols - 1) / kCols;
  const real* BR = fac + rc.Y + k;
  const int64_t* vm = vmap + rc.map;
  real* pr = part + rc.part * nrhs;
  for (int r = 0; r < nrhs; r++) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) xn[c] = y[vm[c0 + c] + (int64_t)r * ldy];
    __syncthreads();
    for (int i = threadIdx.x; i < f; i += blockDim.x) {
      real acc = 0;
      for (int c = 0; c < nc; c++) acc += BR[i + (int64_t)(c0 + c) * m] * xn[c];
      pr[((int64_t)r * nchunk + blockIdx.x) * f + i] = acc;
    }
    __syncthreads();
  }
}

template <typename real>
__global__ void __launch_bounds__(256)
bwd_z_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ y, real* __restrict__ z, const real* __restrict__ part,
             int64_t ldy, int nrhs) {
  const ApplyRec rc = recs[ids[blockIdx.x]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const int nchunk = (rc.nw + kCols - 1) / kCols;
  const real* pr = part + rc.part * nrhs;
  for (int r = 0; r < nrhs; r++) {
    const real* ys = y + rc.voff + (int64_t)r * ldy;
    real* zs = z + rc.voff + (int64_t)r * ldy;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      real v = ys[i];
      if (i >= k)
        for (int q = 0; q < nchunk; q++) v -= pr[((int64_t)r * nchunk + q) * f + (i - k)];
      zs[i] = v;
    }
  }
}

template <typename real>
__global__ void __launch_bounds__(256)
bwd_t_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ fac, real* __restrict__ y, const real* __restrict__ z,
             int64_t ldy, int nrhs) {
  extern __shared__ unsigned char smem_raw[];
  real* zsm = reinterpret_cast<real*>(smem_raw);
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m;
  if (rc.k == m) return;
  const int i0 = blockIdx.x * kRows;
  if (i0 >= m) return;
  const int i1 = min(m, i0 + kRows);
  const real* TRt = fac + (rc.sym ? rc.T : rc.TR);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int r = 0; r < nrhs; r++) {
    const real* zs = z + rc.voff + (int64_t)r * ldy;
    for (int l = threadIdx.x; l < m; l += blockDim.x) zsm[l] = zs[l];
    __syncthreads();
    for (int i = i0 + warp; i < i1; i += nwarp) {
      const real* col = TRt + (int64_t)i * m;
      real acc = 0;
      for (int l = lane; l < m; l += 32) acc += col[l] * zsm[l];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) y[rc.voff + i + (int64_t)r * ldy] = acc;
    }
    __syncthreads();
  }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename real>
void Launch<real>::apply_fwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                             const real* fac, const int64_t* vmap, real* y, real* z, int64_t ldy,
                             int nrhs, cudaStream_t st) {
  if (nids <= 0) return;
  const size_t sm = sizeof(real) * (size_t)std::max(maxm, 1);
  set_smem(fwd_t_kernel<real>, sm);
  dim3 g1((maxm + kRows - 1) / kRows, nids);
  count_launch();
  fwd_t_kernel<real><<<g1, 256, sm, st>>>(recs, ids, fac, y, z, ldy, nrhs);
  dim3 g2(std::max(1, (maxnw + kCols - 1) / kCols), nids);
  count_launch();
  fwd_nbr_kernel<real><<<g2, 256, 0, st>>>(recs, ids, fac, vmap, y, z, ldy, nrhs);
}

template <typename real>
void Launch<real>::apply_bwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                             const real* fac, const int64_t* vmap, real* y, real* z, real* part,
                             int64_t ldy, int nrhs, cudaStream_t st) {
  if (nids <= 0) return;
  if (maxnw > 0) {
    dim3 g1((maxnw + kCols - 1) / kCols, nids);
    count_launch();
    bwd_part_kernel<real><<<g1, 256, 0, st>>>(recs, ids, fac, vmap, y, part, ldy, nrhs);
  }
  count_launch();
  bwd_z_kernel<real><<<nids, 256, 0, st>>>(recs, ids, y, z, part, ldy, nrhs);
  const size_t sm = sizeof(real) * (size_t)std::max(maxm, 1);
  set_smem(bwd_t_kernel<real>, sm);
  dim3 g3((maxm + kRows - 1) / kRows, nids);
  count_launch();
  bwd_t_kernel<real><<<g3, 256, sm, st>>>(recs, ids, fac, y, z, ldy, nrhs);
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
