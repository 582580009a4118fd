// Truncated column-pivoted Householder QR of a cluster's fill block (Eq. lra)
// spread over a thread-block cluster.
//
// The fill block G (m x c, c often in the thousands) is split by columns over
// the CL CTAs of a cluster; each CTA keeps its nonzero columns in its own
// shared memory for the whole factorization, so every step streams shared
// memory instead of L2.  Per step the CTAs agree on the pivot through
// distributed shared memory: the largest remaining column norm over the
// cluster, then the lowest original column index among the columns within
// 1e-10 of it (the tie rule of the single-CTA path); every CTA forms the
// reflector from the pivot column in the owner's shared memory and updates
// its columns.  Two cluster barriers per step; every CTA takes the same
// branches (its decisions use the same exchanged values), so the barriers
// always match.
//
// A count pass first flags and counts the nonzero gathered columns, so that
// each CTA holds an equal share of the nonzero ones and the cluster size and
// shared memory are chosen for the compacted block.
//
// Outputs, in the layout the per-cluster kernel expects: the rank k in
// rank[s], the reflectors v_j as column j of W_G (column-major, ld m, rows
// j..m), tau_j and the sign of R's diagonal in the per-cluster double
// workspace.
#include <climits>
#include <cooperative_groups.h>

#include "common.h"

namespace cg = cooperative_groups;

namespace hs {

namespace {

// near-ties of the pivot search, relative: 1e-10 in float64; in float32 the
// squared norms carry ~1e-7 relative rounding, so ties of exact arithmetic
// are recognised within 1e-5
template <typename real>
__device__ __forceinline__ double tie_rtol() { return sizeof(real) == 8 ? 1e-10 : 1e-5; }
constexpr size_t kQrSmemCap = 200 * 1024;  // dynamic shared memory per CTA, at most
constexpr int kQrThreads = 256;  // threads per CTA of the cluster QR (more only add barrier cost)
constexpr int kMaxGrid = 1 << 20;

// Dynamic shared memory of one CTA: every array starts on a 16-byte boundary
// (the same computation sizes the launch and carves the buffer).
struct QrSmem {
  size_t G, nrm, oidx, tpos, vloc, total;
  __host__ __device__ static size_t al(size_t b) { return (b + 15) / 16 * 16; }
  __host__ __device__ QrSmem(int ldsm, int cc, int sz) {
    G = 0;
    nrm = G + al((size_t)ldsm * cc * sz);
    oidx = nrm + al((size_t)cc * sizeof(double));
    tpos = oidx + al((size_t)cc * sizeof(int));
    vloc = tpos + al((size_t)kQrThreads * sizeof(int));
    total = vloc + al((size_t)ldsm * sz);
  }
};

struct Exchange {
  double val;      // largest local squared norm
  double candnrm;  // squared norm of the local candidate
  int cand;        // lowest original index among the local candidates
  int loc;         // local column of the candidate
};

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
    v = x < v ? x : v;
  }
  return v;
}

__device__ double block_max(double v, double* red) {
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

template <typename real>
__global__ void __launch_bounds__(kQrThreads)
qr_cluster_kernel(const PrepTask* __restrict__ tasks, const real* __restrict__ arena,
                  real* __restrict__ ws_all, double* __restrict__ wsd_all,
                  const Seg* __restrict__ segs, int* rank, int* __restrict__ piv,
                  const int* __restrict__ fpiv, const int* __restrict__ cnt, double eps,
                  double noise_rtol, int max_rank, int ldsm, int ccmax) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks();
  const int cr = (int)cl.block_rank();
  const PrepTask tk = tasks[blockIdx.x / CL];
  const int m = tk.m, c = tk.ncolG;
  __shared__ double red_d[kQrThreads];
  __shared__ Exchange xch;
  extern __shared__ __align__(16) unsigned char dsm[];
  const QrSmem lay(ldsm, ccmax, (int)sizeof(real));
  real* Gs = reinterpret_cast<real*>(dsm + lay.G);  // ldsm x ccmax, column-major
  double* nrm = reinterpret_cast<double*>(dsm + lay.nrm);
  int* oidx = reinterpret_cast<int*>(dsm + lay.oidx);
  int* tpos = reinterpret_cast<int*>(dsm + lay.tpos);
  real* vloc = reinterpret_cast<real*>(dsm + lay.vloc);  // the step's reflector

  // per-cluster outputs (same layout as the per-cluster kernel)
  double* nrm2_g = wsd_all + tk.wsd;
  real* tau_g = reinterpret_cast<real*>(nrm2_g + 2 * (int64_t)tk.ncolG);
  real* rsign_g = tau_g + 2 * m;
  real* W_G = ws_all + tk.ws + 10 * (int64_t)m * m;

  // scale of the rounding-noise floor: max |A_ss|
  double amx = 0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x)
    amx = fmax(amx, fabs((double)arena[tk.a_ss + idx % m + (int64_t)(idx / m) * tk.ld]));
  // forced ranks keep every direction up to the forced count (no floor)
  const double floor = max_rank < 0 ? 0.0 : noise_rtol * block_max(amx, red_d);

  // The count pass flagged the nonzero gathered columns (flags[q] != 0) and
  // counted them (nz); CTA cr keeps nonzero columns cr*cz .. (cr+1)*cz - 1
  // in gathered order, so every CTA holds at most cz columns.
  const double* flags = nrm2_g + tk.ncolG;
  const int nz = cnt[blockIdx.x / CL];
  const int cz = (nz + CL - 1) / CL;
  const int z0 = cr * cz, z1 = min(nz, z0 + cz);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  {
    const int per = (c + blockDim.x - 1) / blockDim.x;
    const int a0 = min(c, (int)threadIdx.x * per), a1 = min(c, a0 + per);
    int n = 0;
    for (int q = a0; q < a1; q++) n += (flags[q] != 0.0);
    tpos[threadIdx.x] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int t = 0; t < (int)blockDim.x; t++) {
        const int v = tpos[t];
        tpos[t] = acc;
        acc += v;
      }
    }
    __syncthreads();
    int zq = tpos[threadIdx.x];
    // the gathered column of each of this CTA's slots
    for (int q = a0; q < a1; q++) {
      if (flags[q] == 0.0) continue;
      if (zq >= z0 && zq < z1) oidx[zq - z0] = q;
      zq++;
    }
    __syncthreads();
  }
  const int nloc = max(0, z1 - z0);
  for (int d = warp; d < nloc; d += nwarp) {
    int64_t p;
    int st;
    seg_col(segs + tk.gcol, tk.ngcol, oidx[d], &p, &st);
    for (int i = lane; i < m; i += 32) Gs[i + (int64_t)d * ldsm] = arena[p + (int64_t)i * st];
  }
  __syncthreads();
  // squared norms in the working precision (float64 arithmetic per element
  // would bound the float32 path by the float64 rate); compared in float64
  for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
    real s = 0;
    for (int i = 0; i < m; i++) {
      const real x = Gs[i + (int64_t)t * ldsm];
      s += x * x;
    }
    nrm[t] = (double)s;
  }
  __syncthreads();

  // max_rank < 0: the rank of every cluster is forced to rank[s] (set by the
  // host before the launch, read before any CTA of the cluster can write it)
  const int kmax = max_rank > 0 ? min(m, max_rank) : (max_rank < 0 ? min(m, rank[tk.s]) : m);
  if (max_rank < 0) eps = 0.0;
  const int steps = min(m, c);
  double r11 = 0;
  int k = 0;
  __shared__ unsigned long long red_u[kQrThreads / 32];
  __shared__ double s_M, s_r;
  __shared__ int s_owner;
  for (int j = 0; j < steps; j++) {
    // 1. largest remaining norm over the cluster
    double lmx = 0;
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) lmx = fmax(lmx, nrm[t]);
    lmx = warp_max(lmx);
    if (lane == 0) red_d[warp] = lmx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_d[0];
      for (int w = 1; w < nwarp; w++) v = fmax(v, red_d[w]);
      xch.val = v;
    }
    cl.sync();
    if (warp == 0) {
      double v = (lane < CL) ? cl.map_shared_rank(&xch, lane)->val : 0.0;
      v = warp_max(v);
      if (lane == 0) s_M = v;
    }
    __syncthreads();
    const double M = s_M;
    if (M <= 0.0) break;
    // 2. lowest original index among the near-maximal columns: one key
    //    (original index, local slot) per candidate, the smallest wins; a
    //    given pivot order (fpiv) makes its column the only candidate
    unsigned long long key = ~0ull;
    const int fq = fpiv ? fpiv[tk.pv + j] : -1;
    for (int t = threadIdx.x; t < nloc; t += blockDim.x)
      if (fpiv ? (z0 + t == fq && nrm[t] >= 0.0) : (nrm[t] >= (1.0 - tie_rtol<real>()) * M)) {
        const unsigned long long kk = ((unsigned long long)oidx[t] << 32) | (unsigned)t;
        key = kk < key ? kk : key;
      }
    key = warp_min_u64(key);
    if (lane == 0) red_u[warp] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long v = red_u[0];
      for (int w = 1; w < nwarp; w++) v = red_u[w] < v ? red_u[w] : v;
      const bool any = v != ~0ull;
      xch.cand = any ? (int)(v >> 32) : INT_MAX;
      xch.loc = any ? (int)(v & 0xffffffffu) : -1;
      xch.candnrm = any ? nrm[(int)(v & 0xffffffffu)] : -1.0;
    }
    cl.sync();
    if (warp == 0) {
      unsigned long long v = ~0ull;
      if (lane < CL)
        v = ((unsigned long long)(unsigned)cl.map_shared_rank(&xch, lane)->cand << 8) | lane;
      v = warp_min_u64(v);
      if (lane == 0) {
        s_owner = (int)(v & 0xff);
        s_r = sqrt(cl.map_shared_rank(&xch, (int)(v & 0xff))->candnrm);
      }
    }
    __syncthreads();
    const int owner = s_owner;
    const double r = s_r;
    if (!(r >= 0.0)) break;  // a given pivot that names no remaining column
    if (j == 0) r11 = r;
    if (r <= floor || (eps > 0.0 && r <= eps * r11) || j >= kmax) break;
    // 3. every CTA forms the reflector v = x - beta e1, beta = -sign(x0) ||x||
    //    from the pivot column in the owner's shared memory (read through
    //    distributed shared memory; that column is never written again, so
    //    no further cluster barrier is needed); the owner also stores it
    const int oloc = cl.map_shared_rank(&xch, owner)->loc;
    const real* ocol = cl.map_shared_rank(Gs, owner) + (int64_t)oloc * ldsm;
    const double x0 = (double)ocol[j];
    const double beta = (x0 >= 0.0) ? -r : r;
    const real tj = (real)((r > 0.0) ? 1.0 / (r * (r + fabs(x0))) : 0.0);
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const real v = (i == j) ? (real)(x0 - beta) : ocol[i];
      vloc[i] = v;
      if (cr == owner) W_G[i + (int64_t)j * m] = v;
    }
    if (cr == owner && threadIdx.x == 0) {
      tau_g[j] = tj;
      rsign_g[j] = beta < 0.0 ? real(-1) : real(1);
      nrm[oloc] = -1.0;  // used: out of every later step
      // the pivot as an index among the nonzero gathered columns: slot t of
      // CTA cr holds nonzero column z0 + t
      piv[tk.pv + j] = z0 + oloc;
    }
    __syncthreads();
    // 4. every CTA applies the reflector to its remaining columns and
    //    recomputes their squared norms over rows j+1..m
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
      if (nrm[t] < 0.0) continue;
      real* col = Gs + (int64_t)t * ldsm;
      // four independent partial sums (combined in a fixed order) keep four
      // products in flight instead of one dependent chain
      real w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      int i = j;
      for (; i + 3 < m; i += 4) {
        w0 += vloc[i] * col[i];
        w1 += vloc[i + 1] * col[i + 1];
        w2 += vloc[i + 2] * col[i + 2];
        w3 += vloc[i + 3] * col[i + 3];
      }
      for (; i < m; i++) w0 += vloc[i] * col[i];
      const real w = ((w0 + w1) + (w2 + w3)) * tj;
      col[j] -= w * vloc[j];
      real s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      i = j + 1;
      for (; i + 3 < m; i += 4) {
        const real a0 = col[i] - w * vloc[i], a1 = col[i + 1] - w * vloc[i + 1];
        const real a2 = col[i + 2] - w * vloc[i + 2], a3 = col[i + 3] - w * vloc[i + 3];
        col[i] = a0;
        col[i + 1] = a1;
        col[i + 2] = a2;
        col[i + 3] = a3;
        s0 += a0 * a0;
        s1 += a1 * a1;
        s2 += a2 * a2;
        s3 += a3 * a3;
      }
      for (; i < m; i++) {
        const real a = col[i] - w * vloc[i];
        col[i] = a;
        s0 += a * a;
      }
      nrm[t] = (double)((s0 + s1) + (s2 + s3));
    }
    __syncthreads();
    k = j + 1;
  }
  if (cr == 0 && threadIdx.x == 0) rank[tk.s] = k;
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

// Count pass: flag the nonzero gathered columns of every task (flags in the
// task's double workspace after the norms) and count them.  Grid (task,
// chunk of 256 columns), one thread per column with eight loads in flight;
// the counts are accumulated atomically into cnt (zeroed by the caller).
template <typename real>
__global__ void __launch_bounds__(256)
count_nz_kernel(const PrepTask* __restrict__ tasks, const real* __restrict__ arena,
                double* __restrict__ wsd_all, const Seg* __restrict__ segs, int* cnt) {
  const PrepTask tk = tasks[blockIdx.x];
  double* flags = wsd_all + tk.wsd + tk.ncolG;
  __shared__ int red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int n = 0;
  for (int q = blockIdx.y * blockDim.x + threadIdx.x; q < tk.ncolG;
       q += gridDim.y * blockDim.x) {
    int64_t p;
    int st;
    seg_col(segs + tk.gcol, tk.ngcol, q, &p, &st);
    bool nz = false;
    for (int i = 0; i < tk.m; i += 8) {
      real x[8];
#pragma unroll
      for (int r = 0; r < 8; r++) x[r] = (i + r < tk.m) ? arena[p + (int64_t)(i + r) * st] : real(0);
#pragma unroll
      for (int r = 0; r < 8; r++) nz |= (x[r] != real(0));
    }
    flags[q] = nz ? 1.0 : 0.0;
    n += nz;
  }
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if (lane == 0) red[warp] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < nwarp; w++) t += red[w];
    if (t) atomicAdd(cnt + blockIdx.x, t);
  }
}

}  // namespace

template <typename real>
void Launch<real>::count_nz(const PrepTask* tasks_dev, int ntask, int maxc, const real* arena,
                            double* wsd, const Seg* segs, int* cnt, cudaStream_t st) {
  if (ntask <= 0) return;
  cudaMemsetAsync(cnt, 0, sizeof(int) * ntask, st);
  const int chunks = std::max(1, std::min((maxc + 255) / 256, 64));
  for (int t0 = 0; t0 < ntask; t0 += kMaxGrid) {
    const int nt = std::min(kMaxGrid, ntask - t0);
    count_launch();
    count_nz_kernel<real><<<dim3(nt, chunks), 256, 0, st>>>(tasks_dev + t0, arena, wsd, segs,
                                                            cnt + t0);
  }
}

template <typename real>
int Launch<real>::qr_cluster_size(int maxm, int maxc) {
  for (int CL = 1; CL <= 16; CL *= 2) {
    if (qr_cluster_smem(maxm, maxc, CL) <= kQrSmemCap) return CL;
  }
  return 0;
}

template <typename real>
size_t Launch<real>::qr_cluster_smem(int maxm, int maxc, int CL) {
  const int cc = (maxc + CL - 1) / CL;
  return QrSmem((maxm + 1) | 1, cc, (int)sizeof(real)).total;
}

template <typename real>
void Launch<real>::qr_cluster(const PrepTask* tasks_dev, int ntask, int maxm, int maxc, int CL,
                              const real* arena, real* ws, double* wsd, const Seg* segs,
                              int* rank, int* piv, const int* fpiv, const int* cnt, double eps,
                              int max_rank, cudaStream_t st) {
  if (ntask <= 0) return;
  const double noise_rtol = sizeof(real) == 8 ? 1e-14 : 1e-6;
  const size_t smem = qr_cluster_smem(maxm, maxc, CL);
  const int cc = (maxc + CL - 1) / CL;
  // the limit is raised once to the sizing cap (qr_cluster_size keeps every
  // launch at or below it) and never lowered: host threads factoring
  // different matrices launch this kernel concurrently
  static const bool limit_set = [] {
    cudaFuncSetAttribute(qr_cluster_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kQrSmemCap);
    // clusters of 16 CTAs (the largest qr_cluster_size picks) are non-portable
    cudaFuncSetAttribute(qr_cluster_kernel<real>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return true;
  }();
  (void)limit_set;
  for (int t0 = 0; t0 < ntask; t0 += 4096) {
    const int nt = std::min(4096, ntask - t0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nt * CL);
    cfg.blockDim = dim3(kQrThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    cudaLaunchKernelEx(&cfg, qr_cluster_kernel<real>, tasks_dev + t0, arena, ws, wsd, segs, rank,
                       piv, fpiv, cnt + t0, eps, noise_rtol, max_rank, (maxm + 1) | 1, cc);
  }
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace hs
