// Dense contractions on the 5th-generation tensor cores (tcgen05), and the
// dense top factorization built on them (Alg. 1: the remaining system is
// factored with a conventional Cholesky once it is small enough).
//
// tc_gemm computes C = beta C + alpha A B^T for float32 matrices with
// arbitrary element strides (A: M x K, B: N x K, C: M x N column-major).
// One CTA of 128 threads per 128 x 128 output tile: the threads stage K-chunks
// of A and B into shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix), converting on the way (TF32 rounding,
// the hi/lo split of 3xTF32, or BF16); one thread issues tcgen05.mma
// (accumulator 128 lanes x 128 float32 columns in tensor memory) and commits
// to an mbarrier per stage, so the staging of chunk c+1 overlaps the MMAs of
// chunk c; the four warps finally read their 32 accumulator lanes with
// tcgen05.ld and apply the epilogue.  Every mbarrier wait is bounded: on
// expiry the kernel records HSOLVE_ERR_TIMEOUT and returns after freeing its
// tensor memory.
//
// The dense top (SPD, float32) uses the recursive blocked form
//   L11 = chol(A11), X11 = L11^{-1}   (recursively; 128-wide leaves on one CTA)
//   L21 = A21 X11^T,  A22 -= L21 L21^T,  L22 = chol(A22), X22 = L22^{-1}
//   X21 = -X22 (L21 X11)
// so that all but the leaves are tensor-core products.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.h"

namespace hs {

namespace {

constexpr int TM = 128, TN = 128;  // output tile
constexpr int TKB = 128;           // bytes of K per row per stage
constexpr int kTcThreads = 128;
constexpr int kTileBytes = TM * TKB;  // one operand tile (16 KB)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle, K-major: start address, the
// byte offset between core matrices adjacent in K (leading) and in M/N
// (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: float32 accumulator, K-major A and B, M = 128,
// N = 128; a/b format 2 = TF32 (kind::tf32) or 1 = BF16 (kind::f16).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(TN >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Wait for the phase with the given parity; false after `limit` SM clocks
// (about a second by default).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = 2000000000ll) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int KIND>  // 0: kind::tf32, 1: kind::f16 (bf16 operands)
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  if (KIND == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, byte b of its K-chunk) in a no-swizzle
// K-major tile: core matrix (r / 8, b / 16) at (r / 8) * SBO + (b / 16) * LBO,
// row r % 8 at 16 bytes each.  LBO = 128 (core matrices adjacent in K are
// contiguous), SBO = 1024 (eight of them per 8-row group).
constexpr uint32_t kLBO = 128, kSBO = 1024;
__device__ __forceinline__ uint32_t core_off(int r, int b) {
  return (uint32_t)((r >> 3) * kSBO + (b >> 4) * kLBO + (r & 7) * 16 + (b & 15));
}

// Operand modes: 0 = TF32 (rounded), 1 = 3xTF32 (hi/lo split, three
// products), 2 = BF16.
template <int MODE>
struct TcMode {
  static constexpr int kTiles = MODE == 1 ? 2 : 1;          // tiles per operand per stage
  static constexpr int kElem = MODE == 2 ? 2 : 4;           // bytes per element
  static constexpr int kKChunk = TKB / kElem;               // K elements per stage
  static constexpr int kKMma = 32 / kElem;                  // K per MMA instruction
  static constexpr int kKind = MODE == 2 ? 1 : 0;
  static constexpr uint32_t kIdesc = instr_desc(MODE == 2 ? 1u : 2u);
  static constexpr int kStageBytes = 2 * kTiles * kTileBytes;  // A and B tiles
};

// Stage rows [r0, r0 + 128) x K-chunk [k0, k0 + kKChunk) of an operand
// (element (r, k) at P[r * rs + k * cs]) into tile(s) at `dst`.  Thread t
// takes row t: 128 bytes of K per row, written as 16-byte vectors.
// Convert and store the EQ consecutive K-elements x[0..EQ) of row r at
// 16-byte core row (r, q) (and the lo part for 3xTF32).
template <int MODE, int EQ>
__device__ __forceinline__ void store_quad(const float* x, int r, int q, unsigned char* dst) {
  if (MODE == 2) {
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
      w[t] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(dst + core_off(r, q * 16)) = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    float hi[4], lo[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
      hi[t] = tf32_round(x[t]);
      lo[t] = tf32_round(x[t] - hi[t]);
    }
    *reinterpret_cast<float4*>(dst + core_off(r, q * 16)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    if (MODE == 1)
      *reinterpret_cast<float4*>(dst + kTileBytes + core_off(r, q * 16)) =
          make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// Staging of an operand whose K elements are contiguous (cs == 1): the
// tile's (row, 16-byte quad) items go 8 rows x 4 quads per warp and
// instruction, so a load touches 8 lines (not 32) and the 16-byte shared
// stores of 8 consecutive lanes fill 8 different rows of one core matrix
// (no bank conflicts).
template <int MODE>
__device__ __forceinline__ void stage_operand_kc(const float* __restrict__ P, int64_t rs, int rows,
                                                 int K, int r0, int k0, unsigned char* dst) {
  constexpr int EQ = TcMode<MODE>::kKChunk / 8;  // elements per 16-byte quad
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rr = lane & 7, qa = lane >> 3;
#pragma unroll 2
  for (int it = 0; it < 8; it++) {
    const int pi = it * 4 + warp;  // (row group of 8, half of the 8 quads)
    const int r = (pi >> 1) * 8 + rr, q = (pi & 1) * 4 + qa;
    const int gr = r0 + r;
    float x[EQ];
#pragma unroll
    for (int t = 0; t < EQ; t++) {
      const int gk = k0 + q * EQ + t;
      x[t] = (gr < rows && gk < K) ? P[(int64_t)gr * rs + gk] : 0.0f;
    }
    store_quad<MODE, EQ>(x, r, q, dst);
  }
}

template <int MODE>
__device__ __forceinline__ void stage_operand(const float* __restrict__ P, int64_t rs, int64_t cs,
                                              int rows, int K, int r0, int k0, unsigned char* dst) {
  using M = TcMode<MODE>;
  if (cs == 1 && rs != 1) {
    stage_operand_kc<MODE>(P, rs, rows, K, r0, k0, dst);
    return;
  }
  const int r = threadIdx.x;
  const int gr = r0 + r;
  float x[M::kKChunk];
#pragma unroll
  for (int k = 0; k < M::kKChunk; k++) {
    const int gk = k0 + k;
    x[k] = (gr < rows && gk < K) ? P[(int64_t)gr * rs + (int64_t)gk * cs] : 0.0f;
  }
  if (MODE == 2) {
#pragma unroll
    for (int b = 0; b < TKB; b += 16) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int k = b / 2 + 2 * q;
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[k], x[k + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(dst + core_off(r, b)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
#pragma unroll
    for (int b = 0; b < TKB; b += 16) {
      float hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float v = x[b / 4 + q];
        hi[q] = tf32_round(v);
        lo[q] = tf32_round(v - hi[q]);
      }
      *reinterpret_cast<float4*>(dst + core_off(r, b)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      if (MODE == 1)
        *reinterpret_cast<float4*>(dst + kTileBytes + core_off(r, b)) =
            make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads)
tc_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int64_t rsa, int64_t csa,
               const float* __restrict__ B, int64_t rsb, int64_t csb, float* __restrict__ C,
               int64_t ldc, float alpha, float beta, int lower, DevError* err) {
  using MD = TcMode<MODE>;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (lower && n0 > m0 + TM - 1) return;  // tile strictly above the diagonal
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 1024-byte aligned start of the two stages
  unsigned char* stages = tc_smem + ((1024 - (smem_u32(tc_smem) & 1023)) & 1023);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  const int nchunk = (K + MD::kKChunk - 1) / MD::kKChunk;
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    unsigned char* st = stages + s * MD::kStageBytes;
    if (c >= 2 && !mbar_wait(&bar[s], ((c - 2) >> 1) & 1)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    stage_operand<MODE>(A, rsa, csa, M, K, m0, c * MD::kKChunk, st);
    stage_operand<MODE>(B, rsb, csb, N, K, n0, c * MD::kKChunk, st + MD::kTiles * kTileBytes);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + MD::kTiles * kTileBytes);
#pragma unroll
      for (int kk = 0; kk < MD::kKChunk / MD::kKMma; kk++) {
        const uint32_t off = kk * 2 * kLBO;  // two core matrices of K per MMA
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        tc_mma<MD::kKind>(tmem, smem_desc(a0 + off, kLBO, kSBO), smem_desc(b0 + off, kLBO, kSBO),
                          MD::kIdesc, acc);
        if (MODE == 1) {  // hi*lo + lo*hi
          tc_mma<MD::kKind>(tmem, smem_desc(a0 + off, kLBO, kSBO),
                            smem_desc(b0 + kTileBytes + off, kLBO, kSBO), MD::kIdesc, 1u);
          tc_mma<MD::kKind>(tmem, smem_desc(a0 + kTileBytes + off, kLBO, kSBO),
                            smem_desc(b0 + off, kLBO, kSBO), MD::kIdesc, 1u);
        }
      }
      tc_commit(&bar[s]);
    }
  }
  if (!abort_flag && nchunk > 0) {
    const int cl = nchunk - 1;
    if (!mbar_wait(&bar[cl & 1], (cl >> 1) & 1)) abort_flag = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!abort_flag) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    for (int j0 = 0; j0 < TN; j0 += 32) {
      float v[32];
      if (nchunk > 0) {
        tmem_ld32(tl + j0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      }
      if (row < M) {
#pragma unroll 4
        for (int i = 0; i < 32; i++) {
          const int col = n0 + j0 + i;
          if (col < N && (!lower || row >= col)) {
            float* cp = C + (int64_t)row + (int64_t)col * ldc;
            *cp = alpha * v[i] + (beta != 0.f ? beta * *cp : 0.f);
          }
        }
      }
    }
  } else if (threadIdx.x == 0 && err) {
    if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_TIMEOUT) == 0) {
      err->cluster = -1;
      err->level = -1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// ---- Schur-complement update of a colour class on the tensor cores
// (Eq. elim): for every task, A_NN -= P^T Q with P = B_L^T, Q = B_R stored as
// f x nw (rows k.. of the cluster's Y storage, ld m, f = m - rank).  Grid
// (column tile, row tile, task); the 128 x 128 accumulator tile is
// subtracted from the neighbour blocks it maps to (runs of the neighbour
// columns, block bases and leading dimensions as in the SIMT update).  The
// blocks of one colour class are disjoint, so no two CTAs write the same
// element.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads)
schur_tc_kernel(const SchurTask* __restrict__ tasks, const float* __restrict__ fac,
                float* __restrict__ arena, const Seg* __restrict__ segs,
                const int64_t* __restrict__ base, const int* __restrict__ ldn,
                const int* __restrict__ rank, DevError* err) {
  using MD = TcMode<MODE>;
  const SchurTask tk = tasks[blockIdx.z];
  const int k = rank[tk.s];
  const int f = tk.m - k;
  const int N = tk.nw;
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  if (f <= 0 || i0 >= N || j0 >= N) return;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int rblk[TM], rloc[TM], cblk[TN], cloc[TN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* stages = tc_smem + ((1024 - (smem_u32(tc_smem) & 1023)) & 1023);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // neighbour run and local index of every row / column of the tile
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
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const float* P = fac + tk.P + k;
  const float* Q = fac + tk.Q + k;
  const int64_t ld = tk.m;
  const int nchunk = (f + MD::kKChunk - 1) / MD::kKChunk;
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    unsigned char* st = stages + s * MD::kStageBytes;
    if (c >= 2 && !mbar_wait(&bar[s], ((c - 2) >> 1) & 1)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    stage_operand<MODE>(P, ld, 1, N, f, i0, c * MD::kKChunk, st);
    stage_operand<MODE>(Q, ld, 1, N, f, j0, c * MD::kKChunk, st + MD::kTiles * kTileBytes);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + MD::kTiles * kTileBytes);
#pragma unroll
      for (int kk = 0; kk < MD::kKChunk / MD::kKMma; kk++) {
        const uint32_t off = kk * 2 * kLBO;
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        tc_mma<MD::kKind>(tmem, smem_desc(a0 + off, kLBO, kSBO), smem_desc(b0 + off, kLBO, kSBO),
                          MD::kIdesc, acc);
        if (MODE == 1) {
          tc_mma<MD::kKind>(tmem, smem_desc(a0 + off, kLBO, kSBO),
                            smem_desc(b0 + kTileBytes + off, kLBO, kSBO), MD::kIdesc, 1u);
          tc_mma<MD::kKind>(tmem, smem_desc(a0 + kTileBytes + off, kLBO, kSBO),
                            smem_desc(b0 + off, kLBO, kSBO), MD::kIdesc, 1u);
        }
      }
      tc_commit(&bar[s]);
    }
  }
  if (!abort_flag) {
    const int cl = nchunk - 1;
    if (!mbar_wait(&bar[cl & 1], (cl >> 1) & 1)) abort_flag = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (!abort_flag) {
    const int ii = warp * 32 + lane, gi = i0 + ii;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const int64_t* bs = base + tk.base;
    const int* ldv = ldn + tk.ldn;
    const int a = rblk[ii], lr = rloc[ii];
    const int64_t lda = ldv[a];
    for (int jc = 0; jc < TN; jc += 32) {
      float v[32];
      tmem_ld32(tl + jc, v);
      if (gi < N) {
#pragma unroll 4
        for (int q = 0; q < 32; q++) {
          const int jj = jc + q;
          if (j0 + jj < N) arena[bs[a * tk.nb + cblk[jj]] + lr + cloc[jj] * lda] -= v[q];
        }
      }
    }
  } else if (threadIdx.x == 0 && err) {
    if (atomicCAS(&err->code, 0, (int)HSOLVE_ERR_TIMEOUT) == 0) {
      err->cluster = tk.s;
      err->level = -1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// ---- dense top leaves: Cholesky and inverse factor of an n <= 128 block on
// one CTA (lower triangle of A in, L into A's lower triangle, X = L^{-1}
// into X with zeros above the diagonal)
constexpr int kLeaf = 128;

// 256 threads as a 16 x 16 grid; thread (tr, tc) keeps the elements (tr +
// 16 a, tc + 16 b), a, b < 8, of the factor (and then of the inverse) in
// registers, so a step reads 16 broadcast values from shared memory and
// updates up to 64 registers; two barriers per step.  The pivots come from a
// shared copy of the trailing diagonal updated alongside.
__global__ void __launch_bounds__(256, 1)
chol_inv_leaf_kernel(float* A, int64_t lda, float* X, int64_t ldx, int n, DevError* err,
                     int level) {
  constexpr int G = 16, R8 = kLeaf / G;
  extern __shared__ float leaf_smem[];
  const int ld = kLeaf + 1;
  float* Ls = leaf_smem;                // L, column-major (for the inverse)
  float* vec = leaf_smem + ld * kLeaf;  // the step's column / row
  __shared__ float diag[kLeaf];         // the trailing diagonal (the pivots)
  const int tr = threadIdx.x % G, tc = threadIdx.x / G;
  float R[R8][R8];
#pragma unroll
  for (int a = 0; a < R8; a++)
#pragma unroll
    for (int b = 0; b < R8; b++) {
      const int i = tr + G * a, l = tc + G * b;
      R[a][b] = (i < n && l < n && i >= l) ? A[i + (int64_t)l * lda] : 0.f;
    }
  for (int t = threadIdx.x; t < n; t += blockDim.x) diag[t] = A[t + (int64_t)t * lda];
  __syncthreads();
  // ---- Cholesky, right-looking: scale column j, then update the trailing part
  for (int j = 0; j < n; j++) {
    const float d = diag[j];
    if (!(d > 0.f)) {
      if (threadIdx.x == 0 && atomicCAS(&err->code, 0, (int)HSOLVE_ERR_NOT_SPD) == 0) {
        err->cluster = 0;
        err->level = level;
      }
      return;  // uniform
    }
    const float rs = rsqrtf(d);
    const int jb = j / G;
    if (tc == j % G) {
#pragma unroll
      for (int a = 0; a < R8; a++) {
        const int i = tr + G * a;
#pragma unroll
        for (int b = 0; b < R8; b++)
          if (b == jb && i >= j && i < n) {
            R[a][b] = (i == j) ? d * rs : R[a][b] * rs;
            vec[i] = R[a][b];
          }
      }
    }
    __syncthreads();
    float ci[R8], cl[R8];
#pragma unroll
    for (int a = 0; a < R8; a++) {
      const int i = tr + G * a;
      ci[a] = (i > j && i < n) ? vec[i] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < R8; b++) {
      const int l = tc + G * b;
      cl[b] = (l > j && l < n) ? vec[l] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < R8; a++)
#pragma unroll
      for (int b = 0; b < R8; b++) {
        const int i = tr + G * a, l = tc + G * b;
        if (i >= l) R[a][b] -= ci[a] * cl[b];
      }
    // the pivots of the later steps
    for (int t = j + 1 + threadIdx.x; t < n; t += blockDim.x) diag[t] -= vec[t] * vec[t];
    __syncthreads();
  }
  // ---- L to shared memory and global; R becomes Y = L^{-1}, from I
#pragma unroll
  for (int a = 0; a < R8; a++)
#pragma unroll
    for (int b = 0; b < R8; b++) {
      const int i = tr + G * a, l = tc + G * b;
      if (i < n && l < n) {
        Ls[i + l * ld] = (i >= l) ? R[a][b] : 0.f;
        if (i >= l) A[i + (int64_t)l * lda] = R[a][b];
      }
      R[a][b] = (i == l && i < n) ? 1.f : 0.f;
    }
  __syncthreads();
  // forward substitution on all columns at once: step i scales row i by
  // 1 / l_ii, then y_rc -= l_ri y_ic for r > i, c <= i
  for (int i = 0; i < n; i++) {
    const float di = 1.f / Ls[i + i * ld];
    const int ib = i / G;
    if (tr == i % G) {
#pragma unroll
      for (int a = 0; a < R8; a++)
#pragma unroll
        for (int b = 0; b < R8; b++) {
          const int c = tc + G * b;
          if (a == ib && c <= i) {
            R[a][b] *= di;
            vec[c] = R[a][b];
          }
        }
    }
    __syncthreads();
    float lr[R8], yc[R8];
#pragma unroll
    for (int a = 0; a < R8; a++) {
      const int r = tr + G * a;
      lr[a] = (r > i && r < n) ? Ls[r + i * ld] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < R8; b++) {
      const int c = tc + G * b;
      yc[b] = (c <= i) ? vec[c] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < R8; a++)
#pragma unroll
      for (int b = 0; b < R8; b++) R[a][b] -= lr[a] * yc[b];
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < R8; a++)
#pragma unroll
    for (int b = 0; b < R8; b++) {
      const int i = tr + G * a, c = tc + G * b;
      if (i < n && c < n) X[i + (int64_t)c * ldx] = (i >= c) ? R[a][b] : 0.f;
    }
}

__global__ void copy_block_kernel(const float* __restrict__ src, int64_t lds, float* dst,
                                  int64_t ldd, int rows, int cols) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[i + j * ldd] = src[i + j * lds];
  }
}

__global__ void zero_block_kernel(float* dst, int64_t ldd, int rows, int cols) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[i + j * ldd] = 0.f;
  }
}

template <int MODE>
void launch_gemm(int M, int N, int K, const float* A, int64_t rsa, int64_t csa, const float* B,
                 int64_t rsb, int64_t csb, float* C, int64_t ldc, float alpha, float beta,
                 bool lower, DevError* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  const size_t smem = 2 * TcMode<MODE>::kStageBytes + 1024;
  static const bool attr_set = [smem] {
    cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    return true;
  }();
  (void)attr_set;
  dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN);
  count_launch();
  tc_gemm_kernel<MODE><<<grid, kTcThreads, smem, st>>>(M, N, K, A, rsa, csa, B, rsb, csb, C, ldc,
                                                       alpha, beta, lower ? 1 : 0, err);
}

int grid1(int64_t work) { return (int)std::min<int64_t>((work + 255) / 256, 152 * 8); }

// Recursive Cholesky + inverse factor of the n x n SPD block at A (lower part),
// X = L^{-1} (ld ldx).  W: scratch of at least n * n / 4 floats.
void top_rec(float* A, int64_t lda, float* X, int64_t ldx, int n, float* W, DevError* err,
             int level, cudaStream_t st) {
  if (n <= kLeaf) {
    const size_t smem = ((size_t)(kLeaf + 1) * kLeaf + kLeaf) * sizeof(float);
    static const bool attr_set = [smem] {
      cudaFuncSetAttribute(chol_inv_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      return true;
    }();
    (void)attr_set;
    count_launch();
    chol_inv_leaf_kernel<<<1, 256, smem, st>>>(A, lda, X, ldx, n, err, level);
    return;
  }
  // split at a multiple of the leaf size near the middle
  const int n1 = std::max(kLeaf, ((n / 2) + kLeaf - 1) / kLeaf * kLeaf);
  const int n2 = n - n1;
  float* A21 = A + n1;
  float* A22 = A + n1 + (int64_t)n1 * lda;
  float* X21 = X + n1;
  float* X22 = X + n1 + (int64_t)n1 * ldx;
  top_rec(A, lda, X, ldx, n1, W, err, level, st);
  // L21 = A21 X11^T into the (not yet used) X21 block
  launch_gemm<1>(n2, n1, n1, A21, 1, lda, X, 1, ldx, X21, ldx, 1.f, 0.f, false, err, st);
  // A22 -= L21 L21^T (lower triangle)
  launch_gemm<1>(n2, n2, n1, X21, 1, ldx, X21, 1, ldx, A22, lda, -1.f, 1.f, true, err, st);
  // L21 into its place in A
  count_launch();
  copy_block_kernel<<<grid1((int64_t)n2 * n1), 256, 0, st>>>(X21, ldx, A21, lda, n2, n1);
  top_rec(A22, lda, X22, ldx, n2, W, err, level, st);
  // W = L21 X11  (n2 x n1, ld n2), then X21 = -X22 W
  launch_gemm<1>(n2, n1, n1, A21, 1, lda, X, ldx, 1, W, n2, 1.f, 0.f, false, err, st);
  launch_gemm<1>(n2, n1, n2, X22, 1, ldx, W, n2, 1, X21, ldx, -1.f, 0.f, false, err, st);
  // the upper block X12 is zero
  count_launch();
  zero_block_kernel<<<grid1((int64_t)n1 * n2), 256, 0, st>>>(X + (int64_t)n1 * ldx, ldx, n1, n2);
}

}  // namespace

void tc_gemm(int mode, int M, int N, int K, const float* A, int64_t rsa, int64_t csa,
             const float* B, int64_t rsb, int64_t csb, float* C, int64_t ldc, float alpha,
             float beta, bool lower, DevError* err, cudaStream_t st) {
  if (mode == 0)
    launch_gemm<0>(M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, lower, err, st);
  else if (mode == 1)
    launch_gemm<1>(M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, lower, err, st);
  else
    launch_gemm<2>(M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, lower, err, st);
}

template <int MODE>
void launch_schur(const SchurTask* tasks, int ntask, int maxnw, const float* fac, float* arena,
                  const Seg* segs, const int64_t* base, const int* ldn, const int* rank,
                  DevError* err, cudaStream_t st) {
  const size_t smem = 2 * TcMode<MODE>::kStageBytes + 1024;
  static const bool attr_set = [smem] {
    cudaFuncSetAttribute(schur_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    return true;
  }();
  (void)attr_set;
  for (int t0 = 0; t0 < ntask; t0 += 65535) {
    dim3 grid((maxnw + TN - 1) / TN, (maxnw + TM - 1) / TM, std::min(65535, ntask - t0));
    count_launch();
    schur_tc_kernel<MODE><<<grid, kTcThreads, smem, st>>>(tasks + t0, fac, arena, segs, base, ldn,
                                                          rank, err);
  }
}

void schur_tc(int mode, const SchurTask* tasks, int ntask, int maxnw, const float* fac,
              float* arena, const Seg* segs, const int64_t* base, const int* ldn, const int* rank,
              DevError* err, cudaStream_t st) {
  if (ntask <= 0 || maxnw <= 0) return;
  if (mode == 0)
    launch_schur<0>(tasks, ntask, maxnw, fac, arena, segs, base, ldn, rank, err, st);
  else if (mode == 1)
    launch_schur<1>(tasks, ntask, maxnw, fac, arena, segs, base, ldn, rank, err, st);
  else
    launch_schur<2>(tasks, ntask, maxnw, fac, arena, segs, base, ldn, rank, err, st);
}

size_t dense_top_tc_scratch(int n) { return (size_t)(n / 2 + kLeaf) * (size_t)(n / 2 + kLeaf); }

void dense_top_tc(float* A, int64_t lda, int n, float* X, float* W, DevError* err, int level,
                  cudaStream_t st) {
  if (n <= 0) return;
  top_rec(A, lda, X, n, n, W, err, level, st);
}

// Diagnostic of the bounded mbarrier wait: one thread waits, with the given
// limit, on a barrier nothing arrives at; the expired wait records
// HSOLVE_ERR_TIMEOUT.  No asynchronous copy or tensor-core operation is in
// flight, so the early return leaves nothing behind.
__global__ void mbar_wait_probe_kernel(long long limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) *err = (int)HSOLVE_ERR_TIMEOUT;
}

void mbar_wait_probe(long long limit, int* err, cudaStream_t st) {
  count_launch();
  mbar_wait_probe_kernel<<<1, 32, 0, st>>>(limit, err);
}

}  // namespace hs
