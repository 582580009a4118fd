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
//   (classes of clusters of at most 256 unknowns: bwd_zt does bwd_z and
//   bwd_t on one CTA per cluster)
// Clusters of one class touch disjoint slots (their neighbour sets are
// disjoint, Sec. 3.2), so no atomics are needed.  z and the partial sums are
// level-sized scratch vectors owned by the factorization.  Every kernel takes
// a group of up to 8 right-hand sides per CTA (grid z over the groups): each
// operator element read serves the whole group.
#include <algorithm>

#include "common.h"

namespace hs {

namespace {

constexpr int kRows = 64;   // output rows per CTA in the T' products
constexpr int kCols = 64;   // neighbour columns per CTA
// right-hand sides per CTA (grid z runs over the groups): 8 when there are
// several, 1 for a single one (a wider group's predicated-off products would
// still be issued, which the float64 pipe cannot afford)
constexpr int kRbWide = 8;

// The right-hand-side group of this CTA: columns r0 .. r0 + nr, groups of
// rb <= RB columns (rb is smaller when RB slot vectors would not fit in
// shared memory).
struct RhsGroup {
  int r0, nr;
  __device__ RhsGroup(int nrhs, int rb)
      : r0(blockIdx.z * rb), nr(min(rb, nrhs - (int)blockIdx.z * rb)) {}
};

// Sums of RB values over a warp.  RB = 8: a reduce-scatter butterfly (9
// shuffles instead of 8 x 5): each exchange halves the set of values a lane
// carries, lane l ending with the total of value rs_index(l); lanes 0..7
// hold the 8 totals once each.  RB = 1: the plain butterfly in every lane.
__device__ __forceinline__ int rs_index(int lane) {
  return ((lane & 1) << 2) | (lane & 2) | ((lane & 4) >> 2);
}

template <typename real>
__device__ __forceinline__ real warp_sum8(const real (&v)[8]) {
  const int lane = threadIdx.x & 31;
  real a[4], b[2];
  const bool h1 = lane & 1, h2 = lane & 2, h4 = lane & 4;
#pragma unroll
  for (int j = 0; j < 4; j++)
    a[j] = (h1 ? v[4 + j] : v[j]) + __shfl_xor_sync(0xffffffffu, h1 ? v[j] : v[4 + j], 1);
#pragma unroll
  for (int j = 0; j < 2; j++)
    b[j] = (h2 ? a[2 + j] : a[j]) + __shfl_xor_sync(0xffffffffu, h2 ? a[j] : a[2 + j], 2);
  real c = (h4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b[0] : b[1], 4);
  c += __shfl_xor_sync(0xffffffffu, c, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 16);
  return c;
}

// Reduce acc[0..RB) over the warp; returns the total that this lane reports
// and sets *r to its right-hand side (-1: this lane reports nothing).
template <typename real, int RB>
__device__ __forceinline__ real warp_sums(real (&acc)[RB], int* r) {
  const int lane = threadIdx.x & 31;
  if constexpr (RB == 8) {
    const real t = warp_sum8<real>(acc);
    *r = lane < 8 ? rs_index(lane) : -1;
    return t;
  } else {
    real t = acc[0];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    *r = lane == 0 ? 0 : -1;
    return t;
  }
}

template <typename real, int RB>
__global__ void __launch_bounds__(256)
fwd_t_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ fac, const real* __restrict__ y, real* __restrict__ z,
             int64_t ldy, int nrhs, int rb) {
  extern __shared__ unsigned char smem_raw[];
  real* ys = reinterpret_cast<real*>(smem_raw);  // RB x m
  __shared__ real red[RB][256];
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m;
  if (rc.k == m) return;
  const int i0 = blockIdx.x * kRows;
  if (i0 >= m) return;
  const RhsGroup g(nrhs, rb);
  const real* T = fac + rc.T;
  const int ii = threadIdx.x % kRows, part = threadIdx.x / kRows;  // 4 parts over l
  const int i = i0 + ii;
  for (int r = 0; r < g.nr; r++)
    for (int l = threadIdx.x; l < m; l += blockDim.x)
      ys[r * m + l] = y[rc.voff + l + (int64_t)(g.r0 + r) * ldy];
  __syncthreads();
  real acc[RB];
#pragma unroll
  for (int r = 0; r < RB; r++) acc[r] = 0;
  if (i < m) {
    // four independent loads in flight per step
    int l = part;
    for (; l + 12 < m; l += 16) {
      const real t0 = __ldg(T + i + (int64_t)l * m);
      const real t1 = __ldg(T + i + (int64_t)(l + 4) * m);
      const real t2 = __ldg(T + i + (int64_t)(l + 8) * m);
      const real t3 = __ldg(T + i + (int64_t)(l + 12) * m);
#pragma unroll
      for (int r = 0; r < RB; r++)
        if (r < g.nr)
          acc[r] += t0 * ys[r * m + l] + t1 * ys[r * m + l + 4] + t2 * ys[r * m + l + 8] +
                    t3 * ys[r * m + l + 12];
    }
    for (; l < m; l += 4) {
      const real t = __ldg(T + i + (int64_t)l * m);
#pragma unroll
      for (int r = 0; r < RB; r++)
        if (r < g.nr) acc[r] += t * ys[r * m + l];
    }
  }
#pragma unroll
  for (int r = 0; r < RB; r++) red[r][threadIdx.x] = acc[r];
  __syncthreads();
  if (part == 0 && i < m)
    for (int r = 0; r < g.nr; r++)
      z[rc.voff + i + (int64_t)(g.r0 + r) * ldy] =
          red[r][ii] + red[r][ii + 64] + red[r][ii + 128] + red[r][ii + 192];
}

template <typename real, int RB>
__global__ void __launch_bounds__(256)
fwd_nbr_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
               const real* __restrict__ fac, const int64_t* __restrict__ vmap,
               real* __restrict__ y, const real* __restrict__ z, int64_t ldy, int nrhs, int rb) {
  extern __shared__ unsigned char smem_raw[];
  real* zsh = reinterpret_cast<real*>(smem_raw);  // RB x f: z_f, read once per CTA
  __shared__ real dsh[RB][kCols];                 // the column sums of this CTA
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const RhsGroup g(nrhs, rb);
  if (blockIdx.x == 0)
    for (int r = 0; r < g.nr; r++)
      for (int i = threadIdx.x; i < m; i += blockDim.x)
        y[rc.voff + i + (int64_t)(g.r0 + r) * ldy] = z[rc.voff + i + (int64_t)(g.r0 + r) * ldy];
  const int c0 = blockIdx.x * kCols;
  if (c0 >= rc.nw) return;
  const int c1 = min(rc.nw, c0 + kCols);
  for (int r = 0; r < g.nr; r++)
    for (int i = threadIdx.x; i < f; i += blockDim.x)
      zsh[r * f + i] = z[rc.voff + k + i + (int64_t)(g.r0 + r) * ldy];
  __syncthreads();
  const real* BL = fac + (rc.sym ? rc.Y : rc.XT) + k;  // column c: B_L[c, :]
  const int64_t* vm = vmap + rc.map;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = c0 + warp; c < c1; c += nwarp) {
    const real* col = BL + (int64_t)c * m;
    real acc[RB];
#pragma unroll
    for (int r = 0; r < RB; r++) acc[r] = 0;
    for (int i = lane; i < f; i += 32) {
      const real b = col[i];
#pragma unroll
      for (int r = 0; r < RB; r++)
        if (r < g.nr) acc[r] += b * zsh[r * f + i];
    }
    int rr;
    const real t = warp_sums<real, RB>(acc, &rr);
    if (rr >= 0) dsh[rr][c - c0] = t;
  }
  __syncthreads();
  // y_N -= B_L z_f: every thread one (column, right-hand side) of the CTA;
  // the neighbour slots of a column range are contiguous runs
  const int nc = c1 - c0;
  for (int e = threadIdx.x; e < nc * g.nr; e += blockDim.x) {
    const int c = e % nc, r = e / nc;
    y[vm[c0 + c] + (int64_t)(g.r0 + r) * ldy] -= dsh[r][c];
  }
}

template <typename real, int RB>
__global__ void __launch_bounds__(256)
bwd_part_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
                const real* __restrict__ fac, const int64_t* __restrict__ vmap,
                const real* __restrict__ y, real* __restrict__ part, int64_t ldy, int nrhs, int rb) {
  __shared__ real xn[RB][kCols];
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const int c0 = blockIdx.x * kCols;
  if (c0 >= rc.nw) return;
  const RhsGroup g(nrhs, rb);
  const int nc = min(rc.nw, c0 + kCols) - c0;
  const int nchunk = (rc.nw + kCols - 1) / kCols;
  const real* BR = fac + rc.Y + k;
  const int64_t* vm = vmap + rc.map;
  real* pr = part + rc.part * nrhs;
  for (int r = 0; r < g.nr; r++)
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
      xn[r][c] = y[vm[c0 + c] + (int64_t)(g.r0 + r) * ldy];
  __syncthreads();
  for (int i = threadIdx.x; i < f; i += blockDim.x) {
    real acc[RB];
#pragma unroll
    for (int r = 0; r < RB; r++) acc[r] = 0;
    const real* Bi = BR + i + (int64_t)c0 * m;
    int c = 0;
    // four independent loads in flight per step
    for (; c + 3 < nc; c += 4) {
      const real b0 = __ldg(Bi + (int64_t)c * m), b1 = __ldg(Bi + (int64_t)(c + 1) * m);
      const real b2 = __ldg(Bi + (int64_t)(c + 2) * m), b3 = __ldg(Bi + (int64_t)(c + 3) * m);
#pragma unroll
      for (int r = 0; r < RB; r++)
        acc[r] += b0 * xn[r][c] + b1 * xn[r][c + 1] + b2 * xn[r][c + 2] + b3 * xn[r][c + 3];
    }
    for (; c < nc; c++) {
      const real b = __ldg(Bi + (int64_t)c * m);
#pragma unroll
      for (int r = 0; r < RB; r++) acc[r] += b * xn[r][c];
    }
#pragma unroll
    for (int r = 0; r < RB; r++)
      if (r < g.nr) pr[((int64_t)(g.r0 + r) * nchunk + blockIdx.x) * f + i] = acc[r];
  }
}

template <typename real, int RB>
__global__ void __launch_bounds__(256)
bwd_z_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ y, real* __restrict__ z, const real* __restrict__ part,
             int64_t ldy, int nrhs, int rb) {
  const ApplyRec rc = recs[ids[blockIdx.x]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const RhsGroup g(nrhs, rb);
  const int nchunk = (rc.nw + kCols - 1) / kCols;
  const real* pr = part + rc.part * nrhs;
  for (int r = g.r0; r < g.r0 + g.nr; r++) {
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

template <typename real, int RB>
__global__ void __launch_bounds__(256)
bwd_t_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
             const real* __restrict__ fac, real* __restrict__ y, const real* __restrict__ z,
             int64_t ldy, int nrhs, int rb) {
  extern __shared__ unsigned char smem_raw[];
  real* zsm = reinterpret_cast<real*>(smem_raw);  // RB x m
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m;
  if (rc.k == m) return;
  const int i0 = blockIdx.x * kRows;
  if (i0 >= m) return;
  const RhsGroup g(nrhs, rb);
  const int i1 = min(m, i0 + kRows);
  const real* TRt = fac + (rc.sym ? rc.T : rc.TR);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int r = 0; r < g.nr; r++)
    for (int l = threadIdx.x; l < m; l += blockDim.x)
      zsm[r * m + l] = z[rc.voff + l + (int64_t)(g.r0 + r) * ldy];
  __syncthreads();
  for (int i = i0 + warp; i < i1; i += nwarp) {
    const real* col = TRt + (int64_t)i * m;
    real acc[RB];
#pragma unroll
    for (int r = 0; r < RB; r++) acc[r] = 0;
    for (int l = lane; l < m; l += 32) {
      const real t = col[l];
#pragma unroll
      for (int r = 0; r < RB; r++)
        if (r < g.nr) acc[r] += t * zsm[r * m + l];
    }
    int rr;
    const real tot = warp_sums<real, RB>(acc, &rr);
    if (rr >= 0 && rr < g.nr) y[rc.voff + i + (int64_t)(g.r0 + rr) * ldy] = tot;
  }
}

// Backward step of a cluster on one CTA (clusters of at most kZtMax
// unknowns): z = [x_c; x_f - sum of the partials of B_R x_N] in shared
// memory, then x_s = T_R'^T z written over the cluster's slots.  The CTA
// reads every slot of its cluster before any is written, so no separate z
// pass is needed.
constexpr int kZtMax = 256;
// output rows a warp of bwd_zt works on at once: 8 in float32, 4 in float64
// (8 float64 rows x 8 right-hand sides of accumulators cost occupancy)
template <typename real>
__host__ __device__ constexpr int rows_in_flight() { return sizeof(real) == 4 ? 8 : 4; }

template <typename real, int RB>
__global__ void __launch_bounds__(256)
bwd_zt_kernel(const ApplyRec* __restrict__ recs, const int* __restrict__ ids,
              const real* __restrict__ fac, real* __restrict__ y, const real* __restrict__ part,
              int64_t ldy, int nrhs, int rb) {
  extern __shared__ unsigned char smem_raw[];
  real* zsm = reinterpret_cast<real*>(smem_raw);  // rb x m
  const ApplyRec rc = recs[ids[blockIdx.y]];
  const int m = rc.m, k = rc.k, f = m - k;
  if (k == m) return;
  const RhsGroup g(nrhs, rb);
  const int nchunk = (rc.nw + kCols - 1) / kCols;
  const real* pr = part + rc.part * nrhs;
  for (int r = 0; r < g.nr; r++) {
    const int rr = g.r0 + r;
    for (int l = threadIdx.x; l < m; l += blockDim.x) {
      real v = y[rc.voff + l + (int64_t)rr * ldy];
      if (l >= k)
        for (int q = 0; q < nchunk; q++) v -= pr[((int64_t)rr * nchunk + q) * f + (l - k)];
      zsm[r * m + l] = v;
    }
  }
  __syncthreads();
  const real* TRt = fac + (rc.sym ? rc.T : rc.TR);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // several output rows per warp at a time (rows i0 + w nwarp), so
  // that their operator loads overlap; every row's sum runs in the same
  // order as one row at a time
  constexpr int kRowsInFlight = rows_in_flight<real>();
  for (int i0 = warp; i0 < m; i0 += nwarp * kRowsInFlight) {
    real acc[kRowsInFlight][RB];
#pragma unroll
    for (int w = 0; w < kRowsInFlight; w++)
#pragma unroll
      for (int r = 0; r < RB; r++) acc[w][r] = 0;
    for (int l = lane; l < m; l += 32) {
      real t[kRowsInFlight];
#pragma unroll
      for (int w = 0; w < kRowsInFlight; w++) {
        const int i = i0 + w * nwarp;
        t[w] = i < m ? TRt[(int64_t)i * m + l] : real(0);
      }
#pragma unroll
      for (int r = 0; r < RB; r++)
        if (r < g.nr) {
          const real zv = zsm[r * m + l];
#pragma unroll
          for (int w = 0; w < kRowsInFlight; w++) acc[w][r] += t[w] * zv;
        }
    }
#pragma unroll
    for (int w = 0; w < kRowsInFlight; w++) {
      const int i = i0 + w * nwarp;
      int rr;
      const real tot = warp_sums<real, RB>(acc[w], &rr);
      if (i < m && rr >= 0 && rr < g.nr) y[rc.voff + i + (int64_t)(g.r0 + rr) * ldy] = tot;
    }
  }
}

// Right-hand sides per CTA: rbmax, fewer when rbmax slot vectors of maxm
// entries would exceed 160 KB of shared memory (the dense top's long
// vectors).
template <typename real>
int group_size(int maxm, int rbmax) {
  const size_t per = sizeof(real) * (size_t)std::max(maxm, 1);
  return (int)std::max<size_t>(1, std::min<size_t>(rbmax, (160u * 1024u) / per));
}

// The dynamic shared-memory limit of a kernel is raised once, to a ceiling
// above every request (at most 160 KB of slot vectors) plus its static arrays,
// and never lowered: a CUDA graph captured earlier may hold a launch of the
// same kernel with a larger request than the current one.
constexpr int kSmemCeiling = 192 * 1024;
template <auto Kernel>
void set_smem() {
  static const bool once = [] {
    cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCeiling);
    return true;
  }();
  (void)once;
}

template <typename real, int RB>
void launch_fwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                const real* fac, const int64_t* vmap, real* y, real* z, int64_t ldy, int nrhs,
                cudaStream_t st) {
  const int rb = group_size<real>(maxm, RB);
  const int nz = (nrhs + rb - 1) / rb;
  const size_t sm = sizeof(real) * (size_t)rb * std::max(maxm, 1);
  set_smem<fwd_t_kernel<real, RB>>();
  dim3 g1((maxm + kRows - 1) / kRows, nids, nz);
  count_launch();
  fwd_t_kernel<real, RB><<<g1, 256, sm, st>>>(recs, ids, fac, y, z, ldy, nrhs, rb);
  dim3 g2(std::max(1, (maxnw + kCols - 1) / kCols), nids, nz);
  set_smem<fwd_nbr_kernel<real, RB>>();
  count_launch();
  fwd_nbr_kernel<real, RB><<<g2, 256, sm, st>>>(recs, ids, fac, vmap, y, z, ldy, nrhs, rb);
}

template <typename real, int RB>
void launch_bwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                const real* fac, const int64_t* vmap, real* y, real* z, real* part, int64_t ldy,
                int nrhs, cudaStream_t st) {
  const int rb = group_size<real>(maxm, RB);
  const int nz = (nrhs + rb - 1) / rb;
  if (maxnw > 0) {
    dim3 g1((maxnw + kCols - 1) / kCols, nids, nz);
    count_launch();
    bwd_part_kernel<real, RB><<<g1, 256, 0, st>>>(recs, ids, fac, vmap, y, part, ldy, nrhs, rb);
  }
  if (maxm <= kZtMax) {
    const size_t sm = sizeof(real) * (size_t)rb * std::max(maxm, 1);
    set_smem<bwd_zt_kernel<real, RB>>();
    count_launch();
    bwd_zt_kernel<real, RB><<<dim3(1, nids, nz), 256, sm, st>>>(recs, ids, fac, y, part, ldy,
                                                                nrhs, rb);
    return;
  }
  count_launch();
  bwd_z_kernel<real, RB><<<dim3(nids, 1, nz), 256, 0, st>>>(recs, ids, y, z, part, ldy, nrhs,
                                                             rb);
  const size_t sm = sizeof(real) * (size_t)rb * std::max(maxm, 1);
  set_smem<bwd_t_kernel<real, RB>>();
  dim3 g3((maxm + kRows - 1) / kRows, nids, nz);
  count_launch();
  bwd_t_kernel<real, RB><<<g3, 256, sm, st>>>(recs, ids, fac, y, z, ldy, nrhs, rb);
}

}  // namespace

template <typename real>
int Launch<real>::apply_max_m() {
  return (int)(kSmemCeiling / sizeof(real));
}

template <typename real>
void Launch<real>::apply_fwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                             const real* fac, const int64_t* vmap, real* y, real* z, int64_t ldy,
                             int nrhs, cudaStream_t st) {
  if (nids <= 0) return;
  if (nrhs == 1)
    launch_fwd<real, 1>(recs, ids, nids, maxm, maxnw, fac, vmap, y, z, ldy, nrhs, st);
  else
    launch_fwd<real, kRbWide>(recs, ids, nids, maxm, maxnw, fac, vmap, y, z, ldy, nrhs, st);
}

template <typename real>
void Launch<real>::apply_bwd(const ApplyRec* recs, const int* ids, int nids, int maxm, int maxnw,
                             const real* fac, const int64_t* vmap, real* y, real* z, real* part,
                             int64_t ldy, int nrhs, cudaStream_t st) {
  if (nids <= 0) return;
  if (nrhs == 1)
    launch_bwd<real, 1>(recs, ids, nids, maxm, maxnw, fac, vmap, y, z, part, ldy, nrhs, st);
  else
    launch_bwd<real, kRbWide>(recs, ids, nids, maxm, maxnw, fac, vmap, y, z, part, ldy, nrhs,
                              st);
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
