// C-ABI entry points and the host-side driver of the hierarchical solver.
//
// hsolve_analyze  Alg. 1 partition step (recursive coordinate bisection),
//                 Eq. quotient block pattern, distance-2 colouring (Sec. 3.2).
// hsolve_factor   Alg. 1: per level, per colour class, one batched launch per
//                 phase of LowRank_Elimination (Eqs. lra, scaling, elim, perm);
//                 sibling clusters' coarse unknowns form the next level.
// hsolve_apply    Alg. 2 forward/backward substitution.
// hsolve_solve    Sec. 5 usage: preconditioned CG / flexible GMRES in float64.
#include <algorithm>
#include <condition_variable>
#include <functional>
#include <type_traits>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.h"

using namespace hs;

namespace {

constexpr int kSketchOversample = 8;  // sketch width m + 8 (randomized Eq. lra)
constexpr int kTopOneCta = 256;       // larger single SPD clusters: blocked dense top

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

struct Status {
  hsolve_status code = HSOLVE_OK;
  std::string msg;
};

#define HS_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      throw Fail(e_ == cudaErrorMemoryAllocation ? HSOLVE_ERR_OOM : HSOLVE_ERR_CUDA, \
                 std::string(#call) + ": " + cudaGetErrorString(e_));              \
    }                                                                              \
  } while (0)

struct Fail {
  hsolve_status code;
  std::string msg;
  Fail(hsolve_status c, std::string m) : code(c), msg(std::move(m)) {}
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      std::lock_guard<std::mutex> lk(device_mutex());
      cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    cudaError_t e;
    {
      std::lock_guard<std::mutex> lk(device_mutex());
      e = cudaMalloc(&p, b);
    }
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Fail(HSOLVE_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed");
    }
    bytes = b;
  }
  void ensure(size_t b) {
    if (b > bytes) alloc(b);
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Host blob of several arrays uploaded with one copy.
struct Blob {
  std::vector<char> h;
  size_t add_raw(const void* src, size_t bytes) {
    size_t o = (h.size() + 15) & ~size_t(15);
    h.resize(o + bytes);
    if (bytes) std::memcpy(h.data() + o, src, bytes);
    return o;
  }
  template <typename T>
  size_t add(const std::vector<T>& v) { return add_raw(v.data(), v.size() * sizeof(T)); }
};

struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinnedBuf() {
    if (p) {
      std::lock_guard<std::mutex> lk(device_mutex());
      cudaFreeHost(p);
    }
  }
  void ensure(size_t b) {
    if (b <= bytes) return;
    if (p) {
      std::lock_guard<std::mutex> lk(device_mutex());
      cudaFreeHost(p);
    }
    p = nullptr;
    bytes = 0;
    cudaError_t e;
    {
      std::lock_guard<std::mutex> lk(device_mutex());
      e = cudaMallocHost(&p, b);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail(HSOLVE_ERR_OOM, "cudaMallocHost failed");
    }
    bytes = b;
  }
};

struct ApplyGraph {
  int nrhs = 0;
  int nodes = 0;
  cudaGraphExec_t exec = nullptr;
};

struct PhaseTimer {
  std::string name;
  double ms = 0;
  int launches = 0;
};

// One factored level.
struct FLevel {
  LevelPattern P;
  std::vector<int> k;                 // coarse unknowns kept per cluster
  std::vector<std::vector<int>> cls;  // processed clusters per colour class
  DevBuf fac;                         // factor arena (real)
  DevBuf recs;                        // ApplyRec per cluster
  DevBuf vmap;                        // int64 vector index maps
  DevBuf ids;                         // int cluster ids, class by class
  std::vector<int> cls_off;           // offsets of each class in ids
  std::vector<int> cls_maxm;          // largest m per class
  std::vector<int> cls_maxnw;         // largest neighbour width per class
  int64_t part_elems = 0;             // backward partial sums per right-hand side
  DevBuf next_idx;                    // int64 gather map to the next level
  int64_t next_n = 0;
  DevBuf vec, zvec, part;             // level vector, scratch vector, partial sums
  int vec_nrhs = 0;
  bool top = false;
  // kept for hsolve_export_level: the pivot order of every cluster's
  // pivoted QR (int, at the cluster's slot offset), the host copy of the
  // apply records, and each cluster's neighbours (id, width) in the column
  // order of its neighbour blocks
  DevBuf piv;
  std::vector<ApplyRec> hrecs;
  std::vector<int> nb_ptr, nb_id, nb_w;
};

}  // namespace

struct hsolve_handle {
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int> col;
  std::vector<double> val;
  DevBuf d_rowptr, d_col, d_val;
  DevBuf d_fval, d_scale;  // equilibrate: values of S A S, and S by original index
  int symmetric = 1;
  hsolve_opts opts{};
  cudaStream_t st = nullptr;
  std::vector<int64_t> perm;
  std::vector<double> scale;
  DevBuf d_perm;
  LevelPattern L0;
  std::vector<std::vector<int>> adj0;
  std::vector<int64_t> csr_dst;  // arena destination of every nonzero at level 0
  DevBuf d_csr_dst;
  // factorization
  std::vector<std::unique_ptr<FLevel>> F;
  int prec = -1;
  bool factored = false;
  double factor_ms = 0;
  double factor_flops = 0, schur_flops = 0, prep_flops = 0, gemm_flops = 0, qr_flops = 0;
  int64_t apply_bytes = 0, factor_bytes = 0, block_bytes = 0;
  int launches = 0;
  int colours_total = 0;
  int64_t coarse_total = 0;
  // scratch
  DevBuf d_err;
  DevBuf ws, wsd, blob_dev, blob2, blob3, cnt;
  DevBuf top_w;  // scratch of the tensor-core dense top
  PinnedBuf pin, pin2, pin3;
  PinnedBuf pin_rank;  // ranks and error words copied back class by class
  // CUDA graphs of the substitution sweeps, one per nrhs (dropped whenever
  // the factorization or the level buffers change)
  bool use_graphs = true;
  std::vector<ApplyGraph> graphs;
  cudaStream_t cap_stream = nullptr;
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  ~hsolve_handle() {
    for (auto& q : pending) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
  DevBuf kry;  // Krylov vectors
  DevBuf dbg;  // per-phase clock stamps of the prep kernel (profiling)
  DevBuf dots;
  PinnedBuf pin_small;
  bool profiling = false;
  bool profile_levels = false;
  // deferred timing: event pairs recorded without synchronising, resolved
  // into phases when the phase times are read or the next factor starts
  bool profile_deferred = false;
  struct Pending {
    std::string name;
    int launches;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<PhaseTimer> phases;
  // next-level patterns of earlier factorizations, keyed by the pattern they
  // were built from and the children's unknown counts
  struct PatCache {
    bool to_top;
    std::vector<int> kin, m, ptr, col;
    LevelPattern Q;
  };
  std::vector<PatCache> pcache;
  // hsolve_factor_forced: per level, the rank of every cluster and (when
  // given) the pivot order of every cluster's pivoted QR, concatenated in
  // cluster order (rank entries each)
  bool force_ranks = false;
  std::vector<std::vector<int>> forced;
  std::vector<std::vector<int>> forced_piv;
  std::string err;
};

namespace {
// tensor-core operand mode of the Schur products (tc_gemm modes), -1: SIMT
int tc_schur_mode(int prec) {
  switch (prec) {
    case HSOLVE_MIXED_TF32: return 0;
    case HSOLVE_MIXED_3XTF32: return 1;
    case HSOLVE_MIXED_BF16: return 2;
    default: return -1;
  }
}
constexpr int kNumSMs = 152;  // SMs of one GB300 (2 dies x 76)
// the equilibration S by original index, or null when A is factored itself
const double* hscale(const hsolve_handle* h) {
  return h->opts.equilibrate ? h->d_scale.as<double>() : nullptr;
}
}  // namespace

namespace {

hsolve_status set_err(hsolve_handle* h, hsolve_status c, const std::string& m) {
  if (h) h->err = m;
  return c;
}

void phase_add(hsolve_handle* h, const char* name, double ms, int launches) {
  for (auto& p : h->phases)
    if (p.name == name) {
      p.ms += ms;
      p.launches += launches;
      return;
    }
  PhaseTimer t;
  t.name = name;
  t.ms = ms;
  t.launches = launches;
  h->phases.push_back(t);
}

// Upload a host blob to the handle's device blob buffer; returns the base.
char* upload_blob(hsolve_handle* h, const Blob& b) {
  size_t bytes = std::max<size_t>(b.h.size(), 16);
  h->pin.ensure(bytes);
  // the previous upload's kernels have completed: every user syncs first
  std::memcpy(h->pin.p, b.h.data(), b.h.size());
  h->blob_dev.ensure(bytes);
  HS_CUDA(cudaMemcpyAsync(h->blob_dev.p, h->pin.p, b.h.size(), cudaMemcpyHostToDevice, h->st));
  return h->blob_dev.as<char>();
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  EventPair(bool enable) : on(enable) {
    if (on) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
    }
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Per-phase timing helper: records an event pair around a lambda when
// profiling is on, otherwise just runs it.
template <typename Fn>
void timed(hsolve_handle* h, const char* name, int launches, Fn&& fn);

// Per-level variant: phases are reported as "<name>.L<level>" when the
// handle records per-level detail.
template <typename Fn>
void timed_lv(hsolve_handle* h, const char* name, int level, int launches, Fn&& fn) {
  if (h->profiling && h->profile_levels) {
    std::string nm = std::string(name) + ".L" + std::to_string(level);
    timed(h, nm.c_str(), launches, fn);
  } else {
    timed(h, name, launches, fn);
  }
}

template <typename Fn>
void timed(hsolve_handle* h, const char* name, int launches, Fn&& fn) {
  h->launches += launches;
  if (!h->profiling) {
    fn();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      throw Fail(HSOLVE_ERR_CUDA, std::string(name) + " launch: " + cudaGetErrorString(e));
    return;
  }
  if (h->profile_deferred) {
    cudaEvent_t ev[2];
    for (auto& e : ev) {
      if (!h->event_pool.empty()) {
        e = h->event_pool.back();
        h->event_pool.pop_back();
      } else {
        cudaEventCreate(&e);
      }
    }
    cudaEventRecord(ev[0], h->st);
    fn();
    cudaEventRecord(ev[1], h->st);
    cudaError_t e = cudaGetLastError();
    h->pending.push_back({name, launches, ev[0], ev[1]});
    if (e != cudaSuccess)
      throw Fail(HSOLVE_ERR_CUDA, std::string(name) + " launch: " + cudaGetErrorString(e));
    return;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, h->st);
  fn();
  cudaEventRecord(b, h->st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw Fail(HSOLVE_ERR_CUDA, std::string(name) + " launch: " + cudaGetErrorString(e));
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  phase_add(h, name, ms, launches);
}

// Resolve deferred event pairs into phase times (waits for the last one).
void resolve_pending(hsolve_handle* h) {
  for (auto& q : h->pending) {
    float ms = 0;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess)
      phase_add(h, q.name.c_str(), ms, q.launches);
    h->event_pool.push_back(q.a);
    h->event_pool.push_back(q.b);
  }
  h->pending.clear();
}

// A process-wide pool of host worker threads for the factorization's
// parallel loops (started on first use, never stopped: the threads wait on a
// condition variable and touch no CUDA state).  One loop runs on it at a
// time; a loop that finds it busy (another handle factoring in another
// thread) runs on its caller alone.
class WorkerPool {
 public:
  explicit WorkerPool(int nt) {
    for (int t = 0; t < nt; t++)
      th_.emplace_back([this] {
        uint64_t seen = 0;
        while (true) {
          std::function<void(int)>* job;
          int n;
          {
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            job = job_;
            n = n_;
          }
          drain(job, n);
          {
            std::lock_guard<std::mutex> lk(mu_);
            if (--active_ == 0) done_.notify_all();
          }
        }
      });
  }
  int size() const { return (int)th_.size(); }
  // Run f(i) for i in [0, n) on the pool and the caller; false if busy.
  bool run(int n, std::function<void(int)>& f) {
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      n_ = n;
      next_.store(0);
      active_ = (int)th_.size();
      gen_++;
    }
    cv_.notify_all();
    drain(&f, n);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return active_ == 0; });
    return true;
  }

 private:
  void drain(std::function<void(int)>* f, int n) {
    for (int i0; (i0 = next_.fetch_add(16)) < n;)
      for (int i = i0; i < std::min(n, i0 + 16); i++) (*f)(i);
  }
  std::vector<std::thread> th_;
  std::mutex mu_, busy_;
  std::condition_variable cv_, done_;
  std::function<void(int)>* job_ = nullptr;
  int n_ = 0, active_ = 0;
  uint64_t gen_ = 0;
  std::atomic<int> next_{0};
};

WorkerPool& worker_pool() {
  static WorkerPool* pool = new WorkerPool(
      (int)std::min(15u, std::max(1u, std::thread::hardware_concurrency()) - 1));
  return *pool;
}

// Run f(i) for i in [0, n) on the worker pool (chunks of 16 indices); small
// loops, or a busy pool, run on the caller.  f must not throw.
template <typename F>
void parallel_for(int n, F&& f) {
  if (n >= 48 && worker_pool().size() > 0) {
    std::function<void(int)> fn = [&f](int i) { f(i); };
    if (worker_pool().run(n, fn)) return;
  }
  for (int i = 0; i < n; i++) f(i);
}

// Host wall time of a section, added to the phase table as "host.<name>"
// when profiling (device phases are CUDA-event times; these are not).
struct HostTimer {
  hsolve_handle* h;
  const char* name;
  std::chrono::steady_clock::time_point t0;
  HostTimer(hsolve_handle* hh, const char* n) : h(hh), name(n), t0(std::chrono::steady_clock::now()) {}
  ~HostTimer() {
    if (!h->profiling) return;
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    phase_add(h, name, ms, 0);
  }
};

void check_dev_error(hsolve_handle* h) {
  DevError e{};
  HS_CUDA(cudaMemcpyAsync(&e, h->d_err.p, sizeof(DevError), cudaMemcpyDeviceToHost, h->st));
  HS_CUDA(cudaStreamSynchronize(h->st));
  if (e.code != 0) {
    throw Fail((hsolve_status)e.code, std::string(e.code == HSOLVE_ERR_NOT_SPD
                                                      ? "Cholesky pivot not positive"
                                                      : "zero pivot in LU") +
                                          " at level " + std::to_string(e.level) +
                                          ", cluster " + std::to_string(e.cluster));
  }
}

// A copy of the device error word taken behind a class's kernels.
void check_err_copy(const DevError& e) {
  if (e.code != 0)
    throw Fail((hsolve_status)e.code, std::string(e.code == HSOLVE_ERR_NOT_SPD
                                                      ? "Cholesky pivot not positive"
                                                      : "zero pivot in LU") +
                                          " at level " + std::to_string(e.level) +
                                          ", cluster " + std::to_string(e.cluster));
}

// ---------------------------------------------------------------------------
// Factorization of one level (all colour classes) -- Alg. 1 inner loop.
// ---------------------------------------------------------------------------
template <typename real>
void factor_level(hsolve_handle* h, FLevel& FL, real* arena, int level, double eps) {
  const LevelPattern& P = FL.P;
  const int nc = P.nclu;
  const bool sym = h->symmetric != 0;
  std::vector<int> cur(P.m);
  FL.k.assign(nc, 0);
  // factor arena: T' (m^2), T'_R^T (m^2, general), Y and XT (m x sum of
  // neighbour sizes) per cluster, upper bounds from the level-start sizes
  std::vector<int64_t> oT(nc), oTR(nc, -1), oY(nc), oXT(nc, -1);
  std::vector<int> wmax(nc, 0);
  int64_t fe = 0;
  for (int s = 0; s < nc; s++) {
    int w = 0;
    for (int p = P.ptr[s]; p < P.ptr[s + 1]; p++)
      if (P.kind[p] == 1) w += P.m[P.col[p]];
    wmax[s] = w;
    int64_t m = P.m[s];
    oT[s] = fe;
    fe += m * m;
    if (!sym) {
      oTR[s] = fe;
      fe += m * m;
    }
    oY[s] = fe;
    fe += m * std::max(w, 1);
    if (!sym) {
      oXT[s] = fe;
      fe += m * std::max(w, 1);
    }
    fe = (fe + 3) / 4 * 4;
  }
  {
    HostTimer ht(h, "host.fac_alloc");
    FL.fac.alloc(std::max<int64_t>(fe, 4) * sizeof(real));
  }
  h->factor_bytes += FL.fac.bytes;
  real* fac = FL.fac.as<real>();
  DevBuf d_rank;
  d_rank.alloc(sizeof(int) * std::max(nc, 1));
  // forced ranks (hsolve_factor_forced): the kernels take rank[s] as the
  // rank of cluster s (max_rank < 0 tells them so)
  const bool forced = h->force_ranks && level < (int)h->forced.size();
  if (forced && (int)h->forced[level].size() != nc)
    throw Fail(HSOLVE_ERR_ARG, "forced ranks: level " + std::to_string(level) + " has " +
                                   std::to_string(nc) + " clusters");
  const int max_rank_arg = forced ? -1 : h->opts.max_rank;
  if (forced) {
    HS_CUDA(cudaMemcpyAsync(d_rank.p, h->forced[level].data(), sizeof(int) * nc,
                            cudaMemcpyHostToDevice, h->st));
    HS_CUDA(cudaStreamSynchronize(h->st));  // the host vector is pageable
  } else {
    // clusters never processed (m = 0) report rank 0
    HS_CUDA(cudaMemsetAsync(d_rank.p, 0, sizeof(int) * std::max(nc, 1), h->st));
  }
  int* rank = d_rank.as<int>();
  FL.piv.alloc(sizeof(int) * std::max<int64_t>(P.voff[nc], 1));
  int* pivd = FL.piv.as<int>();
  // forced pivot orders: cluster s's list at its slot offset
  DevBuf d_fpiv;
  const int* fpiv = nullptr;
  if (forced && level < (int)h->forced_piv.size()) {
    std::vector<int> fp((size_t)std::max<int64_t>(P.voff[nc], 1), -1);
    const std::vector<int>& src = h->forced_piv[level];
    size_t o = 0;
    for (int s = 0; s < nc; s++) {
      const int k = h->forced[level][s];
      if (k < 0 || k > P.m[s] || o + k > src.size())
        throw Fail(HSOLVE_ERR_ARG, "forced pivots: level " + std::to_string(level) +
                                       " has fewer entries than its ranks");
      for (int j = 0; j < k; j++) fp[P.voff[s] + j] = src[o + j];
      o += k;
    }
    if (o != src.size())
      throw Fail(HSOLVE_ERR_ARG, "forced pivots: level " + std::to_string(level) +
                                     " has more entries than its ranks");
    d_fpiv.alloc(sizeof(int) * fp.size());
    HS_CUDA(cudaMemcpyAsync(d_fpiv.p, fp.data(), sizeof(int) * fp.size(), cudaMemcpyHostToDevice,
                            h->st));
    HS_CUDA(cudaStreamSynchronize(h->st));  // the host vector is pageable
    fpiv = d_fpiv.as<int>();
  }
  std::vector<ApplyRec> recs(nc);
  FL.nb_ptr.assign(nc + 1, 0);
  std::vector<std::vector<std::pair<int, int>>> nbl(nc);
  // the level's neighbour-slot map as runs (one per neighbour block of a
  // cluster), expanded on the device at the end of the level
  std::vector<VRun> vruns;
  int64_t vmap_n = 0;
  std::vector<int> fillcols(nc, 0), fillw(nc, 0), nzcols(nc, -1);
  FL.cls.clear();
  // rank-independent part of every cluster's tasks, built in parallel for
  // the whole level: its pattern row without the diagonal (neighbour or fill
  // block, both block offsets) and, for every ordered pair of its
  // neighbours, the offset of their block (the Schur-complement targets)
  struct NbPre {
    int j, kind;
    int64_t p_sj, p_js;
  };
  std::vector<std::vector<NbPre>> pre_nb(nc);
  std::vector<std::vector<int64_t>> pre_sb(nc);
  // The pair table walks each neighbour's pattern row once against a
  // per-thread map cluster -> neighbour index (reset after every cluster)
  // instead of searching the row for every pair.
  auto prepass = [&](int s) {
    thread_local std::vector<int> pos;
    if ((int)pos.size() < nc) pos.assign(nc, -1);
    auto& L = pre_nb[s];
    L.clear();
    L.reserve(P.ptr[s + 1] - P.ptr[s]);
    int nn = 0;
    for (int p = P.ptr[s]; p < P.ptr[s + 1]; p++) {
      const int j = P.col[p];
      if (j == s) continue;
      L.push_back({j, (int)P.kind[p], P.off[p], P.off[P.find(j, s)]});
      if (P.kind[p] == 1) pos[j] = nn++;
    }
    auto& sb = pre_sb[s];
    sb.assign((size_t)nn * nn, -1);
    for (auto& ea : L) {
      if (ea.kind != 1) continue;
      int64_t* row = sb.data() + (size_t)pos[ea.j] * nn;
      for (int q = P.ptr[ea.j]; q < P.ptr[ea.j + 1]; q++) {
        const int b = pos[P.col[q]];
        if (b >= 0) row[b] = P.off[q];
      }
    }
    for (auto& ea : L)
      if (ea.kind == 1) pos[ea.j] = -1;
  };
  {
    HostTimer ht(h, "host.prepass");
    parallel_for(nc, [&](int s) {
      if (P.m[s] > 0) prepass(s);
    });
  }
  // a single large cluster (the dense top of Alg. 1) goes to the blocked
  // multi-CTA Cholesky (SPD) or LU with partial pivoting (general) and the
  // inverse factors: E_s = I, k = 0, no neighbours
  const bool dense_top = (nc == 1 && cur[0] > kTopOneCta &&
                          (sym || cur[0] <= Launch<real>::lu_top_max()));
  if (dense_top) {
    const int n = cur[0];
    if (!sym) {
      h->top_w.ensure(Launch<real>::lu_top_scratch(n));
      bool ok = true;
      timed_lv(h, "dense_top", level, 0, [&] {
        ok = Launch<real>::lu_top(arena + P.off[P.find(0, 0)], P.ld[0], n, fac + oT[0],
                                  fac + oTR[0], h->top_w.p, h->d_err.as<DevError>(), level,
                                  h->st);
      });
      if (!ok) {
        const cudaError_t e = cudaGetLastError();
        throw Fail(e == cudaSuccess ? HSOLVE_ERR_ARG : HSOLVE_ERR_CUDA,
                   std::string("LU top: ") + (e == cudaSuccess ? "above its size limit"
                                                              : cudaGetErrorString(e)));
      }
    } else if (std::is_same<real, float>::value) {
      // float32 modes: recursive Cholesky + inverse factor with tcgen05
      // 3xTF32 products (float32-level accuracy)
      h->top_w.ensure(sizeof(float) * dense_top_tc_scratch(n));
      timed_lv(h, "dense_top", level, 0, [&] {
        dense_top_tc(reinterpret_cast<float*>(arena + P.off[P.find(0, 0)]), P.ld[0], n,
                     reinterpret_cast<float*>(fac + oT[0]), h->top_w.as<float>(),
                     h->d_err.as<DevError>(), level, h->st);
      });
    } else {
      h->top_w.ensure(Launch<real>::dense_top_scratch(n));
      timed_lv(h, "dense_top", level, 0, [&] {
        Launch<real>::dense_top(arena + P.off[P.find(0, 0)], P.ld[0], n, fac + oT[0],
                                h->top_w.as<real>(), h->d_err.as<DevError>(), level, h->st);
      });
    }
    check_dev_error(h);
    FL.cls.push_back({0});
    FL.k[0] = 0;
    cur[0] = 0;
    ApplyRec& r = recs[0];
    r.m = n; r.k = 0; r.nw = 0; r.sym = sym ? 1 : 0; r.voff = 0;
    r.T = oT[0]; r.TR = sym ? oT[0] : oTR[0];
    r.Y = oY[0]; r.XT = sym ? oY[0] : oXT[0]; r.map = 0;
    // Cholesky n^3/3 + inverse n^3/3; LU 2n^3/3 + two inverses n^3/3 each
    const double nf = n, fl = (sym ? 2.0 / 3.0 : 4.0 / 3.0) * nf * nf * nf;
    h->prep_flops += fl;
    h->factor_flops += fl;
    h->apply_bytes += (int64_t)sizeof(real) * 2 * ((int64_t)n * n + 2 * (int64_t)n);
  }
  struct Nb { int j, w; int64_t p_sj, p_js; int ia; };
  // Every cluster's tasks are built in parallel with offsets relative to the
  // cluster (its gathered-column runs, workspace, norms workspace, Schur
  // block bases and neighbour lds, vector-map entries), then concatenated in
  // cluster order with the offsets rebased.
  struct ClusterBuild {
    PrepTask pt;
    SketchTask sk;
    GemmTask gY, gXT, gE, gE2;
    SchurTask sc;
    bool has_sk = false, has_Y = false, has_E = false, has_sc = false;
    std::vector<Seg> segs;
    std::vector<int64_t> sbase;
    std::vector<int> sld;
    std::vector<ScatterSeg> segN, segW;
    std::vector<std::pair<int, int>> nbs;  // neighbours (id, width), column order
    int64_t ws = 0, wsd = 0;
    int nw = 0, nwf = 0, maxw = 0;
    bool bad = false;
  };
  std::vector<ClusterBuild> cbs_keep;
  // The classes run as a pipeline between host and device: a class's ranks
  // are final once its pivoted QR has run (the cluster-QR kernel, or the
  // per-cluster kernel where the QR runs inside it), so they are copied back
  // right then, and the host builds the next class's tasks while the device
  // still runs this class's remaining kernels.  Device errors (a failed
  // Cholesky or LU pivot) are copied back behind each class and read one
  // class later.
  struct ClassTasks {
    std::vector<int> S;
    int nt = 0;
    std::vector<PrepTask> prep;
    std::vector<SketchTask> sk;
    int maxl = 0;
    std::vector<GemmTask> gY, gXT, gE, gE2;
    std::vector<SchurTask> sch;
    std::vector<ScatterSeg> segN, segW;
    std::vector<Seg> segs;
    std::vector<int64_t> sbase;
    std::vector<int> sld;
    int64_t ws_e = 0, wsd_e = 0;
    int maxm = 0, maxnw = 0, maxnwf = 0, maxw_seg = 0;
    Blob b;
    size_t o_sk = 0, o_prep = 0, o_gY = 0, o_gXT = 0, o_gE = 0, o_gE2 = 0, o_sch = 0,
           o_segN = 0, o_segW = 0, o_segs = 0, o_sbase = 0, o_sld = 0;
  };
  // Tasks of the first class at or after c with clusters left; false when
  // no class is left.
  auto build_class = [&](size_t& c, ClassTasks& T) -> bool {
    HostTimer hb(h, "host.build");
    for (; c < P.classes.size(); c++) {
      T.S.clear();
      for (int s : P.classes[c])
        if (cur[s] > 0) T.S.push_back(s);
      if (!T.S.empty()) break;
    }
    if (c >= P.classes.size()) return false;
    const std::vector<int>& S = T.S;
    FL.cls.push_back(S);
    const int nt = (int)S.size();
    T.nt = nt;
    std::vector<PrepTask>& prep = T.prep;
    prep.assign(nt, PrepTask{});
    std::vector<SketchTask>& sk = T.sk;
    int& maxl = T.maxl;
    std::vector<GemmTask>&gY = T.gY, &gXT = T.gXT, &gE = T.gE, &gE2 = T.gE2;
    std::vector<SchurTask>& sch = T.sch;
    std::vector<ScatterSeg>&segN = T.segN, &segW = T.segW;
    std::vector<Seg>& segs = T.segs;
    std::vector<int64_t>& sbase = T.sbase;
    std::vector<int>& sld = T.sld;
    int64_t &ws_e = T.ws_e, &wsd_e = T.wsd_e;
    int &maxm = T.maxm, &maxnw = T.maxnw, &maxnwf = T.maxnwf, &maxw_seg = T.maxw_seg;
    sk.clear();
    gY.clear();
    gXT.clear();
    gE.clear();
    gE2.clear();
    sch.clear();
    segN.clear();
    segW.clear();
    segs.clear();
    sbase.clear();
    sld.clear();
    maxl = 0;
    ws_e = wsd_e = 0;
    maxm = maxnw = maxnwf = maxw_seg = 0;
    // Every cluster's tasks are built in parallel with offsets relative to
    // the cluster (its gathered-column runs, workspace, norms workspace,
    // Schur block bases and neighbour lds, vector-map entries), then
    // concatenated in cluster order with the offsets rebased.
    if ((int)cbs_keep.size() < nt) cbs_keep.resize(nt);
    std::vector<ClusterBuild>& cbs = cbs_keep;  // kept across classes (capacities reused)
    std::unique_ptr<HostTimer> hpar(new HostTimer(h, "host.b_par"));
    parallel_for(nt, [&](int t) {
      ClusterBuild& cb = cbs[t];
      cb.has_sk = cb.has_Y = cb.has_E = cb.has_sc = cb.bad = false;
      cb.segs.clear();
      cb.sbase.clear();
      cb.sld.clear();
      cb.segN.clear();
      cb.segW.clear();
      cb.nbs.clear();
      cb.maxw = 0;
      const int s = S[t];
      const int m = cur[s];
      std::vector<Nb> N, W;
      int nn_all = 0;  // neighbours in the pattern (index base of pre_sb)
      for (auto& e0 : pre_nb[s]) {
        const int ia = e0.kind == 1 ? nn_all++ : -1;
        if (cur[e0.j] == 0) continue;
        Nb e{e0.j, cur[e0.j], e0.p_sj, e0.p_js, ia};
        if (e0.kind == 1) N.push_back(e);
        else W.push_back(e);
      }
      int nw = 0, nwf = 0;
      for (auto& e : N) nw += e.w;
      for (auto& e : W) nwf += e.w;
      cb.nw = nw;
      cb.nwf = nwf;
      // gathered-column runs, one per block: G = [A_sw columns, (general)
      // rows of A_ws]; its first nfs runs alone are A_sW (for C U^T A_sW);
      // A_ws^T alone (for the general far-to-coarse product); A_sN columns;
      // (general) rows of A_Ns
      std::vector<Seg>& segs = cb.segs;
      auto add_runs = [&](const std::vector<Nb>& L, bool trans, int c0) {
        for (auto& e : L) {
          Seg g{};
          g.off = trans ? e.p_js : e.p_sj;
          g.colstart = c0;
          g.ld = trans ? P.ld[e.j] : P.ld[s];
          g.trans = trans ? 1 : 0;
          segs.push_back(g);
          c0 += e.w;
        }
      };
      const int64_t gcol = (int64_t)segs.size();
      add_runs(W, false, 0);
      if (!sym) add_runs(W, true, nwf);
      const int ngcol = (int)(segs.size() - gcol);
      const int64_t gcolT = (int64_t)segs.size();
      if (!sym) add_runs(W, true, 0);
      const int ncolG = sym ? nwf : 2 * nwf;
      const int64_t ncol0 = (int64_t)segs.size();
      add_runs(N, false, 0);
      const int64_t ncol1 = (int64_t)segs.size();
      if (!sym) add_runs(N, true, 0);
      // workspace (offsets relative to the cluster's share)
      const int64_t mm = (int64_t)m * m;
      int64_t ws_e = 0;
      PrepTask& pt = cb.pt;
      pt = PrepTask{};
      pt.s = s;
      pt.m = m;
      pt.ld = P.ld[s];
      pt.ncolG = ncolG;
      pt.a_ss = P.off[P.find(s, s)];
      pt.gcol = gcol;
      pt.ngcol = ngcol;
      pt.pv = P.voff[s];
      pt.ws = ws_e;
      ws_e += 11 * mm + (int64_t)m * ncolG;
      pt.D = ws_e;
      ws_e += mm;
      pt.D2 = ws_e;
      ws_e += mm;
      const int64_t Eoff = ws_e;
      ws_e += (int64_t)m * std::max(nwf, 1);
      const int64_t E2off = ws_e;
      if (!sym) ws_e += (int64_t)m * std::max(nwf, 1);
      ws_e = (ws_e + 3) / 4 * 4;
      // randomized compression: sketch Y = G Omega when G is wider than m + 8
      pt.l = 0;
      pt.Y = 0;
      if (h->opts.compress == 1 && ncolG > m + kSketchOversample) {
        pt.l = m + kSketchOversample;
        pt.Y = ws_e;
        ws_e += (int64_t)m * pt.l;
        ws_e = (ws_e + 3) / 4 * 4;
        SketchTask& k = cb.sk;
        k = SketchTask{};
        k.m = m;
        k.l = pt.l;
        k.ncol = ncolG;
        k.gcol = gcol;
        k.nseg = ngcol;
        k.Y = pt.Y;
        cb.has_sk = true;
      }
      cb.ws = ws_e;
      pt.qr = 0;
      pt.wsd = 0;
      cb.wsd = 2 * (int64_t)std::max(ncolG, m + kSketchOversample) + 4 * m + 8;
      pt.T = oT[s];
      pt.TR = sym ? oT[s] : oTR[s];
      // Y = T' A_sN  (rows 0..k coarse rows, rows k.. = B_R)
      if (nw > 0) {
        GemmTask g{};
        g.s = s; g.M = m; g.N = nw; g.K = m; g.mode = 0; g.lda = m; g.ldc = m;
        g.A = oT[s]; g.C = oY[s]; g.bcol = ncol0; g.nseg = (int)N.size();
        cb.gY = g;
        g.A = sym ? 0 : oTR[s]; g.C = sym ? 0 : oXT[s]; g.bcol = ncol1;
        cb.gXT = g;
        cb.has_Y = true;
      }
      // E = D A_sW (coarse-to-far rows), E2 = D2 A_wsT (far-to-coarse cols)
      if (nwf > 0) {
        GemmTask g{};
        g.s = s; g.M = m; g.N = nwf; g.K = m; g.mode = 1; g.lda = m; g.ldc = m;
        g.A = pt.D; g.C = Eoff; g.bcol = gcol; g.nseg = (int)W.size();
        cb.gE = g;
        g.A = pt.D2; g.C = E2off; g.bcol = gcolT;
        cb.gE2 = g;
        cb.has_E = true;
      }
      // scatter segments (the fill ones read the workspace: rebased later)
      int c0 = 0;
      for (auto& e : N) {
        ScatterSeg sg{};
        sg.s = s; sg.width = e.w; sg.ld_s = P.ld[s]; sg.ld_o = P.ld[e.j];
        sg.src = oY[s] + (int64_t)c0 * m;
        sg.src2 = sym ? -1 : oXT[s] + (int64_t)c0 * m;
        sg.ld_src = m; sg.m = m;
        sg.dst_row = e.p_sj; sg.dst_col = e.p_js;
        cb.segN.push_back(sg);
        cb.maxw = std::max(cb.maxw, e.w);
        c0 += e.w;
      }
      c0 = 0;
      for (auto& e : W) {
        ScatterSeg sg{};
        sg.s = s; sg.width = e.w; sg.ld_s = P.ld[s]; sg.ld_o = P.ld[e.j];
        sg.src = Eoff + (int64_t)c0 * m;
        sg.src2 = sym ? -1 : E2off + (int64_t)c0 * m;
        sg.ld_src = m; sg.m = m;
        sg.dst_row = e.p_sj; sg.dst_col = e.p_js;
        cb.segW.push_back(sg);
        cb.maxw = std::max(cb.maxw, e.w);
        c0 += e.w;
      }
      // Schur task: maps and block bases
      if (nw > 0) {
        SchurTask sc{};
        sc.s = s; sc.m = m; sc.nw = nw; sc.nb = (int)N.size();
        sc.P = sym ? oY[s] : oXT[s];
        sc.Q = oY[s];
        sc.map = ncol0;  // the A_sN runs: one per neighbour, colstart = its offset
        sc.base = 0;
        const auto& sb = pre_sb[s];
        for (int a = 0; a < (int)N.size(); a++)
          for (int b = 0; b < (int)N.size(); b++) {
            const int64_t o = sb[(size_t)N[a].ia * nn_all + N[b].ia];
            if (o < 0) cb.bad = true;
            cb.sbase.push_back(o);
          }
        sc.ldn = 0;
        for (auto& e : N) cb.sld.push_back(P.ld[e.j]);
        cb.sc = sc;
        cb.has_sc = true;
      }
      for (auto& e : N) cb.nbs.push_back({e.j, e.w});
    });
    hpar.reset();
    std::unique_ptr<HostTimer> hmerge(new HostTimer(h, "host.b_merge"));
    for (int t = 0; t < nt; t++) {
      ClusterBuild& cb = cbs[t];
      if (cb.bad) throw Fail(HSOLVE_ERR_CUDA, "internal: missing Schur target block");
      const int s = S[t];
      const int m = cur[s];
      maxm = std::max(maxm, m);
      maxnw = std::max(maxnw, cb.nw);
      maxnwf = std::max(maxnwf, cb.nwf);
      maxw_seg = std::max(maxw_seg, cb.maxw);
      fillw[s] = cb.nwf;
      fillcols[s] = sym ? cb.nwf : 2 * cb.nwf;
      const int64_t sg0 = (int64_t)segs.size(), W0 = ws_e;
      PrepTask pt = cb.pt;
      pt.gcol += sg0;
      pt.ws += W0;
      pt.D += W0;
      pt.D2 += W0;
      if (pt.l > 0) pt.Y += W0;
      pt.wsd = wsd_e;
      prep[t] = pt;
      if (cb.has_sk) {
        SketchTask k = cb.sk;
        k.gcol += sg0;
        k.Y += W0;
        sk.push_back(k);
        maxl = std::max(maxl, k.l);
      }
      if (cb.has_Y) {
        GemmTask g = cb.gY;
        g.bcol += sg0;
        gY.push_back(g);
        if (!sym) {
          g = cb.gXT;
          g.bcol += sg0;
          gXT.push_back(g);
        }
      }
      if (cb.has_E) {
        GemmTask g = cb.gE;
        g.A += W0;
        g.C += W0;
        g.bcol += sg0;
        gE.push_back(g);
        if (!sym) {
          g = cb.gE2;
          g.A += W0;
          g.C += W0;
          g.bcol += sg0;
          gE2.push_back(g);
        }
      }
      segN.insert(segN.end(), cb.segN.begin(), cb.segN.end());
      for (ScatterSeg sg : cb.segW) {
        sg.src += W0;
        if (sg.src2 >= 0) sg.src2 += W0;
        segW.push_back(sg);
      }
      if (cb.has_sc) {
        SchurTask sc = cb.sc;
        sc.map += sg0;
        sc.base = (int64_t)sbase.size();
        sc.ldn = (int64_t)sld.size();
        sbase.insert(sbase.end(), cb.sbase.begin(), cb.sbase.end());
        sld.insert(sld.end(), cb.sld.begin(), cb.sld.end());
        sch.push_back(sc);
      }
      segs.insert(segs.end(), cb.segs.begin(), cb.segs.end());
      ws_e += cb.ws;
      wsd_e += cb.wsd;
      // apply record (k filled after the class completes)
      ApplyRec& r = recs[s];
      r.m = m; r.k = 0; r.nw = cb.nw; r.sym = sym ? 1 : 0;
      r.voff = P.voff[s];
      r.T = oT[s]; r.TR = sym ? oT[s] : oTR[s];
      r.Y = oY[s]; r.XT = sym ? oY[s] : oXT[s];
      r.map = vmap_n;
      for (auto& e : cb.nbs) {
        vruns.push_back({vmap_n, P.voff[e.first], e.second, 0});
        vmap_n += e.second;
        nbl[s].push_back(e);
      }
    }
    hmerge.reset();
    Blob& b = T.b;
    b.h.clear();
    T.o_sk = b.add(sk);
    T.o_prep = b.add(prep);
    T.o_gY = b.add(gY);
    T.o_gXT = b.add(gXT);
    T.o_gE = b.add(gE);
    T.o_gE2 = b.add(gE2);
    T.o_sch = b.add(sch);
    T.o_segN = b.add(segN);
    T.o_segW = b.add(segW);
    T.o_segs = b.add(segs);
    T.o_sbase = b.add(sbase);
    T.o_sld = b.add(sld);
    return true;
  };
  h->pin_rank.ensure(sizeof(int) * std::max(nc, 1) + 2 * sizeof(DevError));
  int* krank = reinterpret_cast<int*>(h->pin_rank.p);
  DevError* kerr = reinterpret_cast<DevError*>(krank + std::max(nc, 1));  // 2 slots
  cudaEvent_t ev_rank = nullptr;
  HS_CUDA(cudaEventCreateWithFlags(&ev_rank, cudaEventDisableTiming));
  struct EventGuard {
    cudaEvent_t e;
    ~EventGuard() { cudaEventDestroy(e); }
  } ev_guard{ev_rank};
  ClassTasks TA, TB;
  ClassTasks* Tc = &TA;
  ClassTasks* Tn = &TB;
  size_t cidx = 0;
  int nclass = 0;
  bool have = !dense_top && build_class(cidx, *Tc);
  while (have) {
    ClassTasks& T = *Tc;
    const std::vector<int>& S = T.S;
    const int nt = T.nt;
    std::vector<PrepTask>& prep = T.prep;
    const std::vector<SketchTask>& sk = T.sk;
    const int maxl = T.maxl;
    const std::vector<GemmTask>&gY = T.gY, &gXT = T.gXT, &gE = T.gE, &gE2 = T.gE2;
    const std::vector<SchurTask>& sch = T.sch;
    const std::vector<ScatterSeg>&segN = T.segN, &segW = T.segW;
    const int maxm = T.maxm, maxnw = T.maxnw, maxnwf = T.maxnwf, maxw_seg = T.maxw_seg;
    const size_t o_sk = T.o_sk, o_prep = T.o_prep, o_gY = T.o_gY, o_gXT = T.o_gXT,
                 o_gE = T.o_gE, o_gE2 = T.o_gE2, o_sch = T.o_sch, o_segN = T.o_segN,
                 o_segW = T.o_segW, o_segs = T.o_segs, o_sbase = T.o_sbase, o_sld = T.o_sld;
    h->ws.ensure(std::max<int64_t>(T.ws_e, 4) * sizeof(real));
    h->wsd.ensure(std::max<int64_t>(T.wsd_e, 4) * sizeof(double));
    char* d = upload_blob(h, T.b);
    // the ranks are final after the pivoted QR: in the cluster-QR kernel,
    // unless some cluster's QR runs inside the per-cluster kernel
    bool rank_in_prep = !sk.empty() || !h->opts.cluster_qr;
    bool rank_copied = false;
    auto copy_ranks = [&] {
      HS_CUDA(cudaMemcpyAsync(krank, rank, sizeof(int) * nc, cudaMemcpyDeviceToHost, h->st));
      HS_CUDA(cudaEventRecord(ev_rank, h->st));
      rank_copied = true;
    };
    real* ws = h->ws.as<real>();
    const PrepTask* d_prep = reinterpret_cast<const PrepTask*>(d + o_prep);
    const Seg* d_segs = reinterpret_cast<const Seg*>(d + o_segs);
    // pivoted QR of the fill blocks on thread-block clusters (distributed
    // shared memory) for every cluster that neither sketches nor has no fill
    std::vector<PrepTask> qrt;
    int qm = 0, qc = 0;
    if (h->opts.cluster_qr)
      for (auto& pt : prep)
        if (pt.l == 0 && pt.ncolG > 0) {
          qm = std::max(qm, pt.m);
          qc = std::max(qc, pt.ncolG);
          PrepTask q = pt;
          q.qr = 2;
          qrt.push_back(q);
        }
    if (!qrt.empty()) {
      // count the nonzero fill columns on the device; the cluster size and
      // shared memory follow the largest compacted block
      Blob b2;
      size_t o2_qr = b2.add(qrt);
      h->blob2.ensure(std::max<size_t>(b2.h.size(), 16));
      h->pin2.ensure(std::max<size_t>(b2.h.size(), 16));
      std::memcpy(h->pin2.p, b2.h.data(), b2.h.size());
      HS_CUDA(cudaMemcpyAsync(h->blob2.p, h->pin2.p, b2.h.size(), cudaMemcpyHostToDevice, h->st));
      const PrepTask* d_qrt = reinterpret_cast<const PrepTask*>(h->blob2.as<char>() + o2_qr);
      h->cnt.ensure(sizeof(int) * qrt.size());
      timed_lv(h, "count_nz", level, 1, [&] {
        Launch<real>::count_nz(d_qrt, (int)qrt.size(), qc, arena, h->wsd.as<double>(), d_segs,
                               h->cnt.as<int>(), h->st);
      });
      std::vector<int> cnt(qrt.size());
      {
        HostTimer ht(h, "host.count_copy");
        HS_CUDA(cudaMemcpyAsync(cnt.data(), h->cnt.p, sizeof(int) * cnt.size(),
                                cudaMemcpyDeviceToHost, h->st));
      }
      {
        HostTimer ht(h, "host.wait_count");
        HS_CUDA(cudaStreamSynchronize(h->st));
      }
      for (size_t i = 0; i < qrt.size(); i++) nzcols[qrt[i].s] = cnt[i];
      const int nzmax = std::max(1, *std::max_element(cnt.begin(), cnt.end()));
      int CL = Launch<real>::qr_cluster_size(qm, nzmax);
      // a class of few clusters spreads each block over more CTAs (up to the
      // portable cluster size 8, at least 64 columns each) to occupy the SMs
      if (CL > 0)
        while (CL < 8 && (int64_t)qrt.size() * CL * 2 <= 2 * kNumSMs && nzmax >= CL * 2 * 64)
          CL *= 2;
      if (CL > 0) {
        for (auto& pt : prep)
          if (pt.l == 0 && pt.ncolG > 0) pt.qr = 2;
        Blob b3;
        size_t o3_prep = b3.add(prep);
        h->blob3.ensure(std::max<size_t>(b3.h.size(), 16));
        h->pin3.ensure(std::max<size_t>(b3.h.size(), 16));
        std::memcpy(h->pin3.p, b3.h.data(), b3.h.size());
        HS_CUDA(cudaMemcpyAsync(h->blob3.p, h->pin3.p, b3.h.size(), cudaMemcpyHostToDevice,
                                h->st));
        d_prep = reinterpret_cast<const PrepTask*>(h->blob3.as<char>() + o3_prep);
        timed_lv(h, "qr_cluster", level, 1, [&] {
          Launch<real>::qr_cluster(d_qrt, (int)qrt.size(), qm, nzmax, CL, arena, ws,
                                   h->wsd.as<double>(), d_segs, rank, pivd, fpiv,
                                   h->cnt.as<int>(), eps, max_rank_arg, h->st);
        });
        if (!rank_in_prep) copy_ranks();
      }
    }
    if (!sk.empty())
      timed_lv(h, "sketch", level, 1, [&] {
        Launch<real>::sketch(reinterpret_cast<const SketchTask*>(d + o_sk), (int)sk.size(), maxm,
                             maxl, arena, ws, d_segs, h->st);
      });
    long long* dbg = nullptr;
    if (h->profiling && h->profile_levels) {
      h->dbg.ensure(sizeof(long long) * 8 * (size_t)nt);
      HS_CUDA(cudaMemsetAsync(h->dbg.p, 0, sizeof(long long) * 8 * (size_t)nt, h->st));
      dbg = h->dbg.as<long long>();
    }
    timed_lv(h, "prep", level, 1, [&] {
      Launch<real>::prep(d_prep, nt, arena, fac, ws,
                         h->wsd.as<double>(), d_segs, rank, pivd, fpiv, eps, sym ? 1 : 0,
                         max_rank_arg, maxm, h->d_err.as<DevError>(), level, dbg, h->st);
    });
    if (!rank_copied) copy_ranks();
    if (dbg) {
      // per checkpoint interval: the slowest cluster of the class, in ms at
      // the 2.07 GHz maximum SM clock
      std::vector<long long> hd(8 * (size_t)nt);
      HS_CUDA(cudaMemcpy(hd.data(), dbg, sizeof(long long) * hd.size(), cudaMemcpyDeviceToHost));
      static const char* nm[7] = {"chol", "gather", "cpqr", "inverse", "complement", "T_C",
                                  "F_tail"};
      for (int q = 0; q < 7; q++) {
        long long mx = 0;
        for (int t = 0; t < nt; t++) {
          long long a = hd[t * 8 + q], b2 = 0;
          for (int r = q + 1; r < 8 && !b2; r++) b2 = hd[t * 8 + r];
          if (a && b2 > a) mx = std::max(mx, b2 - a);
        }
        std::string key = std::string("prep.") + nm[q] + ".L" + std::to_string(level);
        phase_add(h, key.c_str(), mx / 2.07e6, 0);
      }
    }
    timed_lv(h, "gemm_coarse", level, sym ? 1 : 2, [&] {
      Launch<real>::gemm_gather(reinterpret_cast<const GemmTask*>(d + o_gY), (int)gY.size(), maxm,
                                maxnw, fac, fac, arena, d_segs, rank, h->st);
      if (!sym)
        Launch<real>::gemm_gather(reinterpret_cast<const GemmTask*>(d + o_gXT), (int)gXT.size(),
                                  maxm, maxnw, fac, fac, arena, d_segs, rank, h->st);
    });
    timed_lv(h, "gemm_fill", level, sym ? 1 : 2, [&] {
      Launch<real>::gemm_gather(reinterpret_cast<const GemmTask*>(d + o_gE), (int)gE.size(), maxm,
                                maxnwf, ws, ws, arena, d_segs, rank, h->st);
      if (!sym)
        Launch<real>::gemm_gather(reinterpret_cast<const GemmTask*>(d + o_gE2), (int)gE2.size(),
                                  maxm, maxnwf, ws, ws, arena, d_segs, rank, h->st);
    });
    timed_lv(h, "scatter", level, 2, [&] {
      Launch<real>::scatter(reinterpret_cast<const ScatterSeg*>(d + o_segN), (int)segN.size(),
                            maxw_seg, fac, arena, rank, h->st);
      Launch<real>::scatter(reinterpret_cast<const ScatterSeg*>(d + o_segW), (int)segW.size(),
                            maxw_seg, ws, arena, rank, h->st);
    });
    timed_lv(h, "schur", level, 1, [&] {
      const int tm = tc_schur_mode(h->prec);
      if (std::is_same<real, float>::value && tm >= 0)
        schur_tc(tm, reinterpret_cast<const SchurTask*>(d + o_sch), (int)sch.size(), maxnw,
                 reinterpret_cast<const float*>(fac), reinterpret_cast<float*>(arena), d_segs,
                 reinterpret_cast<const int64_t*>(d + o_sbase),
                 reinterpret_cast<const int*>(d + o_sld), rank, h->d_err.as<DevError>(), h->st);
      else
        Launch<real>::schur(reinterpret_cast<const SchurTask*>(d + o_sch), (int)sch.size(),
                            maxnw, fac, arena, d_segs,
                            reinterpret_cast<const int64_t*>(d + o_sbase),
                            reinterpret_cast<const int*>(d + o_sld), rank, h->st);
    });
    if (!rank_copied) copy_ranks();
    // the error word behind this class's kernels (read one class later)
    HS_CUDA(cudaMemcpyAsync(kerr + (nclass & 1), h->d_err.p, sizeof(DevError),
                            cudaMemcpyDeviceToHost, h->st));
    {
      HostTimer ht(h, "host.wait_rank");
      HS_CUDA(cudaEventSynchronize(ev_rank));
    }
    if (nclass > 0) check_err_copy(kerr[(nclass - 1) & 1]);
    std::vector<int> kk(krank, krank + nc);
    for (int s : S) {
      FL.k[s] = kk[s];
      cur[s] = kk[s];
      recs[s].k = kk[s];
      const int m = recs[s].m, k = kk[s], f = m - k;
      const int nw = recs[s].nw;
      // algorithmic flops: dense per-cluster work + the batched products
      double mf = m;
      if (k < m) {
        // per-cluster dense work: Cholesky m^3/3 (+ its inverse m^3/3 for
        // k = 0); with fill: inverse m^3, pivoted QR 4 m c k, complement
        // 4 m^2 k, T 2 m^3, F and C 2 m^2 m, L_F^{-1} T 2 f^2 m
        double pf = 2.0 / 3.0 * mf * mf * mf;
        if (k > 0)
          pf = mf * mf * mf / 3.0 + mf * mf * mf + 4.0 * mf * fillcols[s] * k +
               4.0 * mf * mf * k + 2.0 * mf * mf * mf + 2.0 * mf * mf * mf +
               2.0 * (double)f * f * mf;
        double gf = 2.0 * mf * mf * nw * (sym ? 1 : 2) +
                    (k > 0 ? 2.0 * k * mf * fillw[s] * (sym ? 1 : 2) : 0.0);
        double sf = 2.0 * f * (double)nw * nw;
        if (k > 0) h->qr_flops += 4.0 * mf * (nzcols[s] >= 0 ? nzcols[s] : fillcols[s]) * k;
        h->prep_flops += pf;
        h->gemm_flops += gf;
        h->schur_flops += sf;
        h->factor_flops += pf + gf + sf;
        // operators: T' and B_R each read by both sweeps (SPD), or T', T_R',
        // B_L, B_R each read once (general): 2 (m^2 + f nw) words either way
        h->apply_bytes += (int64_t)sizeof(real) * 2 * ((int64_t)m * m + (int64_t)f * nw);
        h->apply_bytes += (int64_t)sizeof(real) * 2 * (2 * (int64_t)m + 2 * (int64_t)nw);
      }
    }
    nclass++;
    cidx++;
    have = build_class(cidx, *Tn);  // overlaps this class's remaining kernels
    std::swap(Tc, Tn);
  }
  if (nclass > 0) {
    HostTimer ht(h, "host.wait_last");
    HS_CUDA(cudaStreamSynchronize(h->st));
    check_err_copy(kerr[(nclass - 1) & 1]);
  }
  // ---- apply records and maps for this level
  HostTimer ht_end(h, "host.level_end");
  Blob b;
  FL.recs.alloc(sizeof(ApplyRec) * std::max(nc, 1));
  FL.vmap.alloc(sizeof(int64_t) * std::max<int64_t>(vmap_n, 1));
  DevBuf d_vruns;  // kept until the level's final synchronisation below
  if (!vruns.empty()) {
    d_vruns.alloc(sizeof(VRun) * vruns.size());
    HS_CUDA(cudaMemcpyAsync(d_vruns.p, vruns.data(), sizeof(VRun) * vruns.size(),
                            cudaMemcpyHostToDevice, h->st));
    expand_runs(d_vruns.as<VRun>(), (int64_t)vruns.size(), FL.vmap.as<int64_t>(), h->st);
    HS_CUDA(cudaGetLastError());
  }
  std::vector<int> ids;
  FL.cls_off.clear();
  FL.cls_maxm.clear();
  FL.cls_maxnw.clear();
  FL.part_elems = 0;
  for (auto& S : FL.cls) {
    FL.cls_off.push_back((int)ids.size());
    int mx = 1, mw = 0;
    for (int s : S) {
      ids.push_back(s);
      mx = std::max(mx, recs[s].m);
      mw = std::max(mw, recs[s].nw);
      const int f = recs[s].m - recs[s].k;
      const int nchunk = (recs[s].nw + 63) / 64;
      recs[s].part = FL.part_elems;
      FL.part_elems += (int64_t)nchunk * std::max(f, 0);
    }
    FL.cls_maxm.push_back(mx);
    FL.cls_maxnw.push_back(mw);
  }
  HS_CUDA(cudaMemcpyAsync(FL.recs.p, recs.data(), sizeof(ApplyRec) * nc, cudaMemcpyHostToDevice,
                          h->st));
  FL.hrecs = recs;
  FL.nb_id.clear();
  FL.nb_w.clear();
  for (int s = 0; s < nc; s++) {
    for (auto& e : nbl[s]) {
      FL.nb_id.push_back(e.first);
      FL.nb_w.push_back(e.second);
    }
    FL.nb_ptr[s + 1] = (int)FL.nb_id.size();
  }
  FL.cls_off.push_back((int)ids.size());
  FL.ids.alloc(sizeof(int) * std::max<size_t>(ids.size(), 1));
  if (!ids.empty())
    HS_CUDA(cudaMemcpyAsync(FL.ids.p, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice,
                            h->st));
  HS_CUDA(cudaStreamSynchronize(h->st));
  h->colours_total += (int)FL.cls.size();
}

// Next level (Alg. 1 recursion): cluster I holds the coarse unknowns of
// clusters 2I and 2I+1 (left first); the block pattern is the set of child
// pairs that were within distance two and both kept coarse unknowns.  With
// `to_top`, every live cluster merges into one (dense top factor).
template <typename real>
void build_next(hsolve_handle* h, FLevel& FL, const real* arena, std::unique_ptr<FLevel>& out,
                DevBuf& out_arena, bool to_top, const std::vector<int>& kin) {
  const LevelPattern& P = FL.P;
  const int nc = P.nclu;
  out.reset(new FLevel());
  LevelPattern& Q = out->P;
  auto parent = [&](int a) { return to_top ? 0 : a / 2; };
  Q.nclu = to_top ? 1 : nc / 2;
  Q.m.assign(Q.nclu, 0);
  std::vector<int> ro(nc, 0);  // row offset of child a inside its parent
  for (int a = 0; a < nc; a++) {
    int I = parent(a);
    ro[a] = Q.m[I];
    Q.m[I] += kin[a];
  }
  // the next pattern (and its colouring) depends only on this pattern and on
  // which children keep unknowns and how many: reuse it when a previous
  // factorization met the same (a refactorization with the same eps)
  hsolve_handle::PatCache* hit = nullptr;
  for (auto& pc : h->pcache)
    if (pc.to_top == to_top && pc.kin == kin && pc.m == P.m && pc.col == P.col &&
        pc.ptr == P.ptr)
      hit = &pc;
  if (hit) {
    Q = hit->Q;
  } else {
    std::vector<std::vector<int>> adj(Q.nclu);
    for (int a = 0; a < nc; a++) {
      if (kin[a] == 0) continue;
      for (int p = P.ptr[a]; p < P.ptr[a + 1]; p++) {
        int b = P.col[p];
        if (kin[b] == 0) continue;
        int I = parent(a), J = parent(b);
        if (I != J) adj[I].push_back(J);
      }
    }
    for (auto& v : adj) {
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    build_level_pattern(Q, adj);
    if (h->pcache.size() >= 32) h->pcache.erase(h->pcache.begin());
    h->pcache.push_back({to_top, kin, P.m, P.ptr, P.col, Q});
  }
  {
    HostTimer ht(h, "host.next_alloc");
    out_arena.alloc(Q.arena_elems * sizeof(real));
  }
  HS_CUDA(cudaMemsetAsync(out_arena.p, 0, Q.arena_elems * sizeof(real), h->st));
  HostTimer ht_tasks(h, "host.next_tasks");
  // one copy per kept block, counted and then written per cluster row in
  // parallel
  std::vector<int64_t> tstart(nc + 1, 0);
  for (int a = 0; a < nc; a++) {
    int cnt = 0;
    if (kin[a] > 0)
      for (int p = P.ptr[a]; p < P.ptr[a + 1]; p++) cnt += kin[P.col[p]] > 0;
    tstart[a + 1] = tstart[a] + cnt;
  }
  std::vector<CopyTask> tasks((size_t)tstart[nc]);
  std::atomic<int> missing{0};
  parallel_for(nc, [&](int a) {
    if (kin[a] == 0) return;
    int64_t o = tstart[a];
    for (int p = P.ptr[a]; p < P.ptr[a + 1]; p++) {
      const int b = P.col[p];
      if (kin[b] == 0) continue;
      const int I = parent(a), J = parent(b);
      const int64_t q = Q.find(I, J);
      if (q < 0) {
        missing.store(1);
        return;
      }
      CopyTask& t = tasks[(size_t)o++];
      t.rows = kin[a];
      t.cols = kin[b];
      t.ld_src = P.ld[a];
      t.ld_dst = Q.ld[I];
      t.src = P.off[p];
      t.dst = Q.off[q] + ro[a] + (int64_t)ro[b] * Q.ld[I];
    }
  });
  if (missing.load()) throw Fail(HSOLVE_ERR_CUDA, "internal: missing next-level block");
  if (!tasks.empty()) {
    Blob bl;
    size_t o = bl.add(tasks);
    char* d = upload_blob(h, bl);
    timed(h, "assemble", 1, [&] {
      Launch<real>::copy_blocks(reinterpret_cast<const CopyTask*>(d + o), (int)tasks.size(), arena,
                                out_arena.as<real>(), h->st);
    });
  }
  // vector gather map: next-level position -> this level's position
  HostTimer ht_idx(h, "host.next_idx");
  // children of parent I are contiguous in a (2I, 2I+1; every a for the
  // top), so one pass in order lists them parent by parent
  int64_t nidx = 0;
  for (int a = 0; a < nc; a++) nidx += kin[a];
  std::vector<int64_t> idx((size_t)nidx);
  {
    int64_t o = 0;
    for (int a = 0; a < nc; a++)
      for (int i = 0; i < kin[a]; i++) idx[(size_t)o++] = P.voff[a] + i;
  }
  FL.next_n = (int64_t)idx.size();
  FL.next_idx.alloc(sizeof(int64_t) * std::max<size_t>(idx.size(), 1));
  if (!idx.empty())
    HS_CUDA(cudaMemcpyAsync(FL.next_idx.p, idx.data(), sizeof(int64_t) * idx.size(),
                            cudaMemcpyHostToDevice, h->st));
  HS_CUDA(cudaStreamSynchronize(h->st));
}

template <typename real>
void factor_impl(hsolve_handle* h, double eps) {
  // a merged dense top must fit the substitution sweeps' shared-memory slot
  // vectors and, for a general matrix, the LU panel's thread-block cluster
  int64_t top_max = Launch<real>::apply_max_m();
  if (!h->symmetric) top_max = std::min<int64_t>(top_max, Launch<real>::lu_top_max());
  if (h->opts.top_size > top_max)
    throw Fail(HSOLVE_ERR_ARG, "top_size " + std::to_string(h->opts.top_size) +
                                   " above the dense-top limit of " + std::to_string(top_max) +
                                   " unknowns for this precision and matrix type");
  {
    HostTimer ht(h, "host.clear");
    h->F.clear();
  }
  h->factor_flops = h->schur_flops = h->prep_flops = h->gemm_flops = h->qr_flops = 0;
  h->apply_bytes = h->factor_bytes = h->block_bytes = 0;
  h->launches = 0;
  h->colours_total = 0;
  h->coarse_total = 0;
  resolve_pending(h);
  h->phases.clear();
  HS_CUDA(cudaMemsetAsync(h->d_err.p, 0, sizeof(DevError), h->st));
  cudaEvent_t e0, e1;
  HS_CUDA(cudaEventCreate(&e0));
  HS_CUDA(cudaEventCreate(&e1));
  HS_CUDA(cudaEventRecord(e0, h->st));
  // level-0 blocks from the CSR values
  std::unique_ptr<FLevel> cur(new FLevel());
  cur->P = h->L0;
  DevBuf arena;
  arena.alloc(cur->P.arena_elems * sizeof(real));
  HS_CUDA(cudaMemsetAsync(arena.p, 0, cur->P.arena_elems * sizeof(real), h->st));
  timed(h, "upload", 1, [&] {
    Launch<real>::scatter_csr(h->d_csr_dst.as<int64_t>(),
                              h->opts.equilibrate ? h->d_fval.as<double>() : h->d_val.as<double>(),
                              h->nnz, arena.as<real>(), h->st);
  });
  int level = 0;
  while (true) {
    LevelPattern& P = cur->P;
    h->block_bytes = std::max<int64_t>(h->block_bytes, (int64_t)arena.bytes);
    int live = 0;
    for (int i = 0; i < P.nclu; i++) live += P.m[i] > 0;
    const int64_t vlen = P.voff[P.nclu];
    // a level of at most top_size unknowns merges into the dense top
    // (blocked Cholesky or LU; top_size was checked against their limits)
    const bool small = (P.nclu == 1 || live <= 1 || vlen <= h->opts.top_size);
    if (small && !(P.nclu == 1)) {
      // merge everything into one cluster for the dense top factor
      std::unique_ptr<FLevel> nxt;
      DevBuf narena;
      std::vector<int> kin(P.m.begin(), P.m.end());
      {
        HostTimer ht(h, "host.build_next");
        build_next<real>(h, *cur, arena.as<real>(), nxt, narena, true, kin);
      }
      // the merge level itself has no factors: mark it as a pass-through
      cur->cls.clear();
      cur->cls_off.assign(1, 0);
      cur->k = kin;
      cur->recs.alloc(16);
      cur->vmap.alloc(16);
      cur->ids.alloc(16);
      h->F.push_back(std::move(cur));
      cur = std::move(nxt);
      arena = std::move(narena);
      level++;
      continue;
    }
    factor_level<real>(h, *cur, arena.as<real>(), level, eps);
    for (int i = 0; i < P.nclu; i++) h->coarse_total += cur->k[i];
    if (P.nclu == 1) {
      cur->top = true;
      h->F.push_back(std::move(cur));
      break;
    }
    std::unique_ptr<FLevel> nxt;
    DevBuf narena;
    std::vector<int> kin = cur->k;
    {
      HostTimer ht(h, "host.build_next");
      build_next<real>(h, *cur, arena.as<real>(), nxt, narena, false, kin);
    }
    h->F.push_back(std::move(cur));
    cur = std::move(nxt);
    {
      HostTimer ht(h, "host.arena_free");
      arena = std::move(narena);
    }
    level++;
  }
  HS_CUDA(cudaEventRecord(e1, h->st));
  HS_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->factor_ms = ms;
}

// ---------------------------------------------------------------------------
// Substitution (Alg. 2)
// ---------------------------------------------------------------------------
// The vectors one application of the sweeps works in, per level: the level
// vector, a scratch vector and the backward partial sums.
struct LevelVecs {
  void* vec;
  void* zvec;
  void* part;
};

// The level sweeps of Alg. 2 between the level-0 vector and itself: a fixed
// sequence of launches once the factorization and nrhs are fixed (one group
// of launches per colour class and direction).
template <typename real>
void apply_levels(hsolve_handle* h, int nrhs, cudaStream_t st, const std::vector<LevelVecs>& B) {
  const int L = (int)h->F.size();
  auto vec = [&](int l) { return static_cast<real*>(B[l].vec); };
  for (int l = 0; l < L; l++) {
    FLevel& F = *h->F[l];
    const int64_t nl = std::max<int64_t>(F.P.voff[F.P.nclu], 1);
    for (size_t c = 0; c < F.cls.size(); c++)
      Launch<real>::apply_fwd(F.recs.as<ApplyRec>(), F.ids.as<int>() + F.cls_off[c],
                              (int)F.cls[c].size(), F.cls_maxm[c], F.cls_maxnw[c],
                              F.fac.as<real>(), F.vmap.as<int64_t>(), vec(l),
                              static_cast<real*>(B[l].zvec), nl, nrhs, st);
    if (l + 1 < L) {
      FLevel& G = *h->F[l + 1];
      const int64_t ng = std::max<int64_t>(G.P.voff[G.P.nclu], 1);
      Launch<real>::gather_vec(F.next_idx.as<int64_t>(), F.next_n, vec(l), nl, vec(l + 1), ng,
                               nrhs, st);
    }
  }
  for (int l = L - 1; l >= 0; l--) {
    FLevel& F = *h->F[l];
    const int64_t nl = std::max<int64_t>(F.P.voff[F.P.nclu], 1);
    if (l + 1 < L) {
      FLevel& G = *h->F[l + 1];
      const int64_t ng = std::max<int64_t>(G.P.voff[G.P.nclu], 1);
      Launch<real>::scatter_vec(F.next_idx.as<int64_t>(), F.next_n, vec(l + 1), ng, vec(l), nl,
                                nrhs, st);
    }
    for (int c = (int)F.cls.size() - 1; c >= 0; c--)
      Launch<real>::apply_bwd(F.recs.as<ApplyRec>(), F.ids.as<int>() + F.cls_off[c],
                              (int)F.cls[c].size(), F.cls_maxm[c], F.cls_maxnw[c],
                              F.fac.as<real>(), F.vmap.as<int64_t>(), vec(l),
                              static_cast<real*>(B[l].zvec), static_cast<real*>(B[l].part), nl,
                              nrhs, st);
  }
}

template <typename real>
void apply_impl(hsolve_handle* h, const double* rhs, double* out, int nrhs, int64_t ld) {
  bool realloc = false;
  for (auto& F : h->F) {
    if (F->vec_nrhs < nrhs) {
      const size_t nv = sizeof(real) * (size_t)std::max<int64_t>(F->P.voff[F->P.nclu], 1) * nrhs;
      F->vec.alloc(nv);
      F->zvec.alloc(nv);
      F->part.alloc(sizeof(real) * (size_t)std::max<int64_t>(F->part_elems, 1) * nrhs);
      F->vec_nrhs = nrhs;
      realloc = true;
    }
  }
  if (realloc) h->drop_graphs();
  std::vector<LevelVecs> B;
  for (auto& F : h->F) B.push_back({F->vec.p, F->zvec.p, F->part.p});
  FLevel& F0 = *h->F[0];
  const int64_t n0 = F0.P.voff[F0.P.nclu];
  Launch<real>::perm_in(h->d_perm.as<int64_t>(), hscale(h), h->n, rhs, ld, F0.vec.as<real>(), n0, nrhs, h->st);
  if (!h->use_graphs) {
    apply_levels<real>(h, nrhs, h->st, B);
  } else {
    // the sweeps are captured once per nrhs into a CUDA graph (on a private
    // stream: capture does not execute) and replayed on the caller's stream
    ApplyGraph* g = nullptr;
    for (auto& x : h->graphs)
      if (x.nrhs == nrhs) g = &x;
    if (!g) {
      std::lock_guard<std::mutex> lk(device_mutex());
      if (!h->cap_stream) HS_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      if (h->graphs.size() >= 8) {  // keep the graphs of the 8 latest widths
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
      }
      const int64_t l0 = launches_total();
      HS_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
      apply_levels<real>(h, nrhs, h->cap_stream, B);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
      if (e != cudaSuccess) throw Fail(HSOLVE_ERR_CUDA, std::string("apply capture: ") + cudaGetErrorString(e));
      ApplyGraph ng;
      ng.nrhs = nrhs;
      ng.nodes = (int)(launches_total() - l0);
      e = cudaGraphInstantiate(&ng.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) throw Fail(HSOLVE_ERR_CUDA, std::string("apply graph: ") + cudaGetErrorString(e));
      // capture counted the launches once; replays add them below
      count_launch(-ng.nodes);
      h->graphs.push_back(ng);
      g = &h->graphs.back();
    }
    HS_CUDA(cudaGraphLaunch(g->exec, h->st));
    count_launch(g->nodes);
  }
  Launch<real>::perm_out(h->d_perm.as<int64_t>(), hscale(h), h->n, F0.vec.as<real>(), n0, out, ld, nrhs, h->st);
}

void apply_any(hsolve_handle* h, const double* rhs, double* out, int nrhs, int64_t ld) {
  if (h->prec == HSOLVE_FP64)
    apply_impl<double>(h, rhs, out, nrhs, ld);
  else
    apply_impl<float>(h, rhs, out, nrhs, ld);
}

// ---------------------------------------------------------------------------
// Substitution with a fixed, library-owned scratch (hsolve_apply_noalloc)
// ---------------------------------------------------------------------------
// Some callers cannot let this library call cudaMalloc: their device memory
// is owned by another allocator (a framework's caching allocator or a
// pre-reserved pool that leaves nothing outside it), or they must not pay
// the implicit device synchronisation that cudaMalloc/cudaFree can bring.
// For them the substitution sweeps take every temporary vector from this
// fixed array instead of the handle's lazily allocated buffers.  It is a
// file-scope device array, so every GPU that loads the library holds it
// until the process exits.  All calls share it: calls whose device work
// overlaps (on different streams, or from different handles) race on it.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code cannot use g_noalloc_scratch's name as a device address (it is a
// host-side stand-in); its device address is looked up once per device,
// with that device current, and cached here.
constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

hsolve_status noalloc_scratch_address(void** out, std::string* why) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return HSOLVE_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    *why = "device index beyond the scratch table";
    return HSOLVE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return HSOLVE_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HSOLVE_OK;
}

// Scratch layout per level: level vector, scratch vector, partial sums,
// each nrhs wide and 256-byte aligned.  Returns the bytes needed.
template <typename real>
size_t noalloc_layout(const hsolve_handle* h, int nrhs, std::vector<size_t>* offs) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) / 256 * 256;
    return at;
  };
  for (auto& F : h->F) {
    const size_t nv = sizeof(real) * (size_t)std::max<int64_t>(F->P.voff[F->P.nclu], 1) * nrhs;
    const size_t np = sizeof(real) * (size_t)std::max<int64_t>(F->part_elems, 1) * nrhs;
    size_t a = take(nv), b = take(nv), c = take(np);
    if (offs) {
      offs->push_back(a);
      offs->push_back(b);
      offs->push_back(c);
    }
  }
  return o;
}

// Same sweeps as apply_impl, with every temporary taken from `base`.  No
// element of the scratch needs to start at zero: each one the sweeps read is
// written earlier in the same call (perm_in fills level 0, the gathers fill
// every coarser level, the partial sums are written before they are summed).
template <typename real>
void apply_scratch_impl(hsolve_handle* h, const double* rhs, double* out, int nrhs, int64_t ld,
                        unsigned char* base) {
  std::vector<size_t> offs;
  noalloc_layout<real>(h, nrhs, &offs);
  std::vector<LevelVecs> B;
  for (size_t l = 0; l < h->F.size(); l++)
    B.push_back({base + offs[3 * l], base + offs[3 * l + 1], base + offs[3 * l + 2]});
  FLevel& F0 = *h->F[0];
  const int64_t n0 = F0.P.voff[F0.P.nclu];
  real* v0 = static_cast<real*>(B[0].vec);
  Launch<real>::perm_in(h->d_perm.as<int64_t>(), hscale(h), h->n, rhs, ld, v0, n0, nrhs, h->st);
  apply_levels<real>(h, nrhs, h->st, B);
  Launch<real>::perm_out(h->d_perm.as<int64_t>(), hscale(h), h->n, v0, n0, out, ld, nrhs, h->st);
}

// ---------------------------------------------------------------------------
// Krylov solvers (float64)
// ---------------------------------------------------------------------------
struct Scalars {  // device scratch for dot products
  double* part;
  double* res;
};

// out[c] = a[:,c].b[:,c] for c < nrhs, copied to host vector
void dots_host(hsolve_handle* h, const double* a, const double* b, int64_t ld, int nrhs,
               std::vector<double>& out) {
  const int kDotBlocks = 256;
  h->dots.ensure(sizeof(double) * (size_t)(nrhs + 64) * (kDotBlocks + 1));
  double* d = h->dots.as<double>();
  hs::dots(h->n, a, ld, b, ld, nrhs, d, h->st);
  out.resize(nrhs);
  h->pin_small.ensure(sizeof(double) * (nrhs + 64) * 2);
  HS_CUDA(cudaMemcpyAsync(h->pin_small.p, d + (int64_t)nrhs * kDotBlocks, sizeof(double) * nrhs,
                          cudaMemcpyDeviceToHost, h->st));
  HS_CUDA(cudaStreamSynchronize(h->st));
  std::memcpy(out.data(), h->pin_small.p, sizeof(double) * nrhs);
}

void upload_coefs(hsolve_handle* h, const std::vector<double>& v, double* dst) {
  h->pin_small.ensure(sizeof(double) * (v.size() + 64) * 2);
  double* p = reinterpret_cast<double*>(h->pin_small.p) + 64 + v.size();
  // the pinned area is reused: wait for the previous copy out of it
  HS_CUDA(cudaStreamSynchronize(h->st));
  std::memcpy(p, v.data(), sizeof(double) * v.size());
  HS_CUDA(cudaMemcpyAsync(dst, p, sizeof(double) * v.size(), cudaMemcpyHostToDevice, h->st));
}

hsolve_status pcg_impl(hsolve_handle* h, double tol, int maxit, const double* b, double* x,
                       int nrhs, int64_t ldx, hsolve_solve_info* info) {
  const int64_t n = h->n;
  // vectors: r, z, p, q (n x nrhs each, ld n) + coefficient arrays
  h->kry.ensure(sizeof(double) * ((size_t)4 * n * nrhs + 8 * (size_t)nrhs + 64));
  double* r = h->kry.as<double>();
  double* z = r + n * nrhs;
  double* p = z + n * nrhs;
  double* q = p + n * nrhs;
  double* coef = q + n * nrhs;  // [alpha | -alpha | one | beta | zero] per rhs
  std::vector<double> bb, rr, rz, pq;
  dots_host(h, b, b, ldx, nrhs, bb);  // b uses ldx
  // x = 0, r = b
  for (int c = 0; c < nrhs; c++) {
    HS_CUDA(cudaMemsetAsync(x + c * ldx, 0, sizeof(double) * n, h->st));
    HS_CUDA(cudaMemcpyAsync(r + c * n, b + c * ldx, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                            h->st));
  }
  std::vector<double> nb(nrhs);
  for (int c = 0; c < nrhs; c++) nb[c] = std::sqrt(bb[c]);
  apply_any(h, r, z, nrhs, n);
  HS_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, h->st));
  dots_host(h, r, z, n, nrhs, rz);
  std::vector<char> done(nrhs, 0);
  for (int c = 0; c < nrhs; c++) done[c] = (nb[c] == 0.0);
  int it = 0;
  std::vector<double> res(nrhs, 0.0);
  bool all = std::all_of(done.begin(), done.end(), [](char d) { return d != 0; });
  std::vector<double> ones(nrhs, 1.0), cf(nrhs), cm(nrhs);
  while (!all && it < maxit) {
    it++;
    spmv_csr(n, h->d_rowptr.as<int64_t>(), h->d_col.as<int>(), h->d_val.as<double>(), p, n, q, n,
             nrhs, h->st);
    dots_host(h, p, q, n, nrhs, pq);
    for (int c = 0; c < nrhs; c++) {
      double a = (done[c] || pq[c] == 0.0) ? 0.0 : rz[c] / pq[c];
      cf[c] = a;
      cm[c] = -a;
    }
    // x += a p ; r -= a q
    upload_coefs(h, cf, coef);
    upload_coefs(h, ones, coef + 2 * nrhs);
    axpby_cols(n, nrhs, coef, p, n, coef + 2 * nrhs, x, ldx, h->st);
    upload_coefs(h, cm, coef + nrhs);
    axpby_cols(n, nrhs, coef + nrhs, q, n, coef + 2 * nrhs, r, n, h->st);
    dots_host(h, r, r, n, nrhs, rr);
    for (int c = 0; c < nrhs; c++) {
      res[c] = std::sqrt(rr[c]) / (nb[c] > 0 ? nb[c] : 1.0);
      if (!done[c] && res[c] <= tol) done[c] = 1;
    }
    all = std::all_of(done.begin(), done.end(), [](char d) { return d != 0; });
    if (all) break;
    apply_any(h, r, z, nrhs, n);
    std::vector<double> rzn;
    dots_host(h, r, z, n, nrhs, rzn);
    for (int c = 0; c < nrhs; c++) {
      cf[c] = (done[c] || rz[c] == 0.0) ? 0.0 : rzn[c] / rz[c];
      rz[c] = rzn[c];
    }
    // p = z + beta p
    upload_coefs(h, cf, coef + 3 * nrhs);
    axpby_cols(n, nrhs, coef + 2 * nrhs, z, n, coef + 3 * nrhs, p, n, h->st);
  }
  // true residual b - A x
  spmv_csr(n, h->d_rowptr.as<int64_t>(), h->d_col.as<int>(), h->d_val.as<double>(), x, ldx, q, n,
           nrhs, h->st);
  for (int c = 0; c < nrhs; c++) cm[c] = -1.0;
  upload_coefs(h, cm, coef + nrhs);
  for (int c = 0; c < nrhs; c++)
    HS_CUDA(cudaMemcpyAsync(r + c * n, b + c * ldx, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                            h->st));
  axpby_cols(n, nrhs, coef + 2 * nrhs, r, n, coef + nrhs, q, n, h->st);  // q = r - q
  dots_host(h, q, q, n, nrhs, rr);
  double worst = 0;
  for (int c = 0; c < nrhs; c++)
    worst = std::max(worst, nb[c] > 0 ? std::sqrt(rr[c]) / nb[c] : 0.0);
  if (info) {
    info->iterations = it;
    info->rel_residual = worst;
  }
  if (worst > tol) return HSOLVE_ERR_NO_CONVERGENCE;
  return HSOLVE_OK;
}

// Right-preconditioned flexible GMRES(restart) with CGS2 for a block of
// right-hand sides at once: each column has its own Krylov space, Hessenberg
// matrix and Givens rotations (host), but every preconditioner application,
// SpMV and orthogonalisation runs on the whole n x nrhs block.  A column that
// meets the tolerance stops contributing at that step of the cycle (its
// solution update uses the steps up to it); the others continue.
hsolve_status fgmres_batch(hsolve_handle* h, double tol, int maxit, const double* b, double* x,
                           int nrhs, int64_t ldx, int restart, int* iters, double* relres) {
  const int64_t n = h->n;
  const int R = restart;
  const int64_t bs = n * (int64_t)nrhs;
  h->kry.ensure(sizeof(double) * ((size_t)(2 * R + 2) * bs + 8 * (size_t)(R + 2) * nrhs + 256));
  double* V = h->kry.as<double>();          // R+1 blocks
  double* Z = V + (int64_t)(R + 1) * bs;    // R blocks
  double* w = Z + (int64_t)R * bs;          // one block
  double* coef = w + bs;                    // (R+2) * nrhs coefficients
  const int kDotBlocks = 256;
  auto block_dots = [&](int nv, const double* Vb, const double* wb, std::vector<double>& out) {
    const int ncol = nv * nrhs;
    h->dots.ensure(sizeof(double) * (size_t)(ncol + 64) * (kDotBlocks + 1));
    double* d = h->dots.as<double>();
    block_multi_dot(n, nv, nrhs, Vb, wb, d, h->st);
    out.resize(ncol);
    h->pin_small.ensure(sizeof(double) * (size_t)(ncol + 64) * 4);
    HS_CUDA(cudaMemcpyAsync(h->pin_small.p, d + (int64_t)ncol * kDotBlocks, sizeof(double) * ncol,
                            cudaMemcpyDeviceToHost, h->st));
    HS_CUDA(cudaStreamSynchronize(h->st));
    std::memcpy(out.data(), h->pin_small.p, sizeof(double) * ncol);
  };
  std::vector<double> nb2;
  dots_host(h, b, b, ldx, nrhs, nb2);
  std::vector<double> nb(nrhs), res(nrhs, 0.0);
  for (int c = 0; c < nrhs; c++) nb[c] = std::sqrt(nb2[c]);
  for (int c = 0; c < nrhs; c++) HS_CUDA(cudaMemsetAsync(x + c * ldx, 0, sizeof(double) * n, h->st));
  std::vector<int> its(nrhs, 0);
  std::vector<char> active(nrhs, 0);
  std::vector<double> ones(nrhs, 1.0), mones(nrhs, -1.0), zeros(nrhs, 0.0);
  int total = 0;
  auto residual = [&]() {  // V_0 = b - A x, res = ||V_0|| / ||b||
    spmv_csr(n, h->d_rowptr.as<int64_t>(), h->d_col.as<int>(), h->d_val.as<double>(), x, ldx, w,
             n, nrhs, h->st);
    for (int c = 0; c < nrhs; c++)
      HS_CUDA(cudaMemcpyAsync(V + c * n, b + c * ldx, sizeof(double) * n,
                              cudaMemcpyDeviceToDevice, h->st));
    upload_coefs(h, ones, coef);
    upload_coefs(h, mones, coef + nrhs);
    axpby_cols(n, nrhs, coef + nrhs, w, n, coef, V, n, h->st);  // V0 = -w + V0
    std::vector<double> r2;
    dots_host(h, V, V, n, nrhs, r2);
    std::vector<double> beta(nrhs);
    for (int c = 0; c < nrhs; c++) {
      beta[c] = std::sqrt(r2[c]);
      res[c] = nb[c] > 0 ? beta[c] / nb[c] : 0.0;
    }
    return beta;
  };
  while (true) {
    std::vector<double> beta = residual();
    bool any = false;
    for (int c = 0; c < nrhs; c++) {
      active[c] = res[c] > tol;
      any |= active[c] != 0;
    }
    if (!any || total >= maxit) break;
    // V_0[:, c] /= beta_c (inactive columns become zero)
    std::vector<double> sc(nrhs);
    for (int c = 0; c < nrhs; c++) sc[c] = active[c] ? 1.0 / beta[c] : 0.0;
    upload_coefs(h, sc, coef);
    upload_coefs(h, zeros, coef + nrhs);
    axpby_cols(n, nrhs, coef, V, n, coef + nrhs, V, n, h->st);
    // per column: Hessenberg (column-major by step), rotations, g
    std::vector<std::vector<double>> H(nrhs, std::vector<double>((size_t)(R + 1) * R, 0.0));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(R)),
        sn(nrhs, std::vector<double>(R)), g(nrhs, std::vector<double>(R + 1, 0.0));
    std::vector<int> jdone(nrhs, 0);
    std::vector<char> open(active);  // still iterating in this cycle
    for (int c = 0; c < nrhs; c++) g[c][0] = beta[c];
    for (int j = 0; j < R; j++) {
      apply_any(h, V + j * bs, Z + j * bs, nrhs, n);
      spmv_csr(n, h->d_rowptr.as<int64_t>(), h->d_col.as<int>(), h->d_val.as<double>(),
               Z + j * bs, n, w, n, nrhs, h->st);
      std::vector<double> hcol((size_t)(j + 1) * nrhs, 0.0);
      for (int pass = 0; pass < 2; pass++) {
        std::vector<double> hh;
        block_dots(j + 1, V, w, hh);
        upload_coefs(h, hh, coef);
        block_multi_axpy(n, j + 1, nrhs, V, coef, -1.0, w, n, h->st);
        for (size_t q = 0; q < hh.size(); q++) hcol[q] += hh[q];
      }
      std::vector<double> w2;
      dots_host(h, w, w, n, nrhs, w2);
      std::vector<double> inv(nrhs);
      for (int c = 0; c < nrhs; c++) {
        const double hn = std::sqrt(w2[c]);
        inv[c] = (open[c] && hn > 0) ? 1.0 / hn : 0.0;
        if (!open[c]) continue;
        std::vector<double>& Hc = H[c];
        double* col = Hc.data() + (size_t)j * (R + 1);
        for (int i = 0; i <= j; i++) col[i] = hcol[(size_t)i * nrhs + c];
        col[j + 1] = hn;
        for (int i = 0; i < j; i++) {
          const double t = cs[c][i] * col[i] + sn[c][i] * col[i + 1];
          col[i + 1] = -sn[c][i] * col[i] + cs[c][i] * col[i + 1];
          col[i] = t;
        }
        const double den = std::hypot(col[j], col[j + 1]);
        cs[c][j] = den > 0 ? col[j] / den : 1.0;
        sn[c][j] = den > 0 ? col[j + 1] / den : 0.0;
        col[j] = den;
        col[j + 1] = 0;
        g[c][j + 1] = -sn[c][j] * g[c][j];
        g[c][j] = cs[c][j] * g[c][j];
        jdone[c] = j + 1;
        its[c]++;
        if (std::fabs(g[c][j + 1]) <= tol * nb[c] || den == 0.0) open[c] = 0;
      }
      // V_{j+1} = w / ||w|| (zero for columns no longer iterating)
      upload_coefs(h, inv, coef);
      upload_coefs(h, zeros, coef + nrhs);
      axpby_cols(n, nrhs, coef, w, n, coef + nrhs, V + (j + 1) * bs, n, h->st);
      total++;
      bool still = false;
      for (int c = 0; c < nrhs; c++) still |= open[c] != 0;
      if (!still || total >= maxit) break;
    }
    // y_c = H_c^{-1} g_c over its jdone_c steps; x += Z y
    int jmax = 0;
    for (int c = 0; c < nrhs; c++) jmax = std::max(jmax, jdone[c]);
    if (jmax == 0) break;
    std::vector<double> Y((size_t)jmax * nrhs, 0.0);
    for (int c = 0; c < nrhs; c++) {
      const int jd = jdone[c];
      const std::vector<double>& Hc = H[c];
      std::vector<double> y(jd);
      for (int i = jd - 1; i >= 0; i--) {
        double t = g[c][i];
        for (int l = i + 1; l < jd; l++) t -= Hc[(size_t)l * (R + 1) + i] * y[l];
        const double d = Hc[(size_t)i * (R + 1) + i];
        y[i] = d != 0.0 ? t / d : 0.0;
      }
      for (int i = 0; i < jd; i++) Y[(size_t)i * nrhs + c] = y[i];
    }
    upload_coefs(h, Y, coef);
    block_multi_axpy(n, jmax, nrhs, Z, coef, 1.0, x, ldx, h->st);
  }
  int itmax = 0;
  double worst = 0;
  for (int c = 0; c < nrhs; c++) {
    itmax = std::max(itmax, its[c]);
    worst = std::max(worst, res[c]);
  }
  *iters = itmax;
  *relres = worst;
  return worst <= tol ? HSOLVE_OK : HSOLVE_ERR_NO_CONVERGENCE;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

void hsolve_default_opts(hsolve_opts* o) {
  if (!o) return;
  o->leaf_size = 128;
  o->symmetric = -1;
  o->top_size = 0;
  o->max_rank = 0;
  o->gmres_restart = 50;
  o->compress = 0;
  o->cluster_qr = 1;
  o->equilibrate = 0;
}

hsolve_status hsolve_analyze(const hsolve_csr* A, const double* coords, int dim,
                             const hsolve_opts* opts, void* cuda_stream, hsolve_handle** out) {
  if (!out) return HSOLVE_ERR_ARG;
  *out = nullptr;
  if (!A || A->n <= 0 || A->nnz < 0 || !A->rowptr || !A->col || !A->val) return HSOLVE_ERR_ARG;
  if (coords && (dim < 1 || dim > 3)) return HSOLVE_ERR_ARG;
  const int64_t n = A->n;
  if (A->rowptr[0] != 0 || A->rowptr[n] != A->nnz) return HSOLVE_ERR_ARG;
  for (int64_t i = 0; i < n; i++)
    if (A->rowptr[i + 1] < A->rowptr[i]) return HSOLVE_ERR_ARG;
  for (int64_t p = 0; p < A->nnz; p++)
    if (A->col[p] < 0 || A->col[p] >= n) return HSOLVE_ERR_ARG;
  std::unique_ptr<hsolve_handle> h(new hsolve_handle());
  hsolve_default_opts(&h->opts);
  if (opts) h->opts = *opts;
  if (h->opts.leaf_size < 1) return HSOLVE_ERR_ARG;
  if (h->opts.gmres_restart < 1) h->opts.gmres_restart = 50;
  h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->n = n;
  h->nnz = A->nnz;
  h->rowptr.assign(A->rowptr, A->rowptr + n + 1);
  h->col.assign(A->col, A->col + A->nnz);
  h->val.assign(A->val, A->val + A->nnz);
  try {
    // exact value symmetry check (symmetric = -1)
    if (h->opts.symmetric < 0) {
      bool symm = true;
      for (int64_t i = 0; i < n && symm; i++)
        for (int64_t p = h->rowptr[i]; p < h->rowptr[i + 1] && symm; p++) {
          int64_t j = h->col[p];
          double v = h->val[p];
          // find (j, i)
          auto b = h->col.begin() + h->rowptr[j], e = h->col.begin() + h->rowptr[j + 1];
          bool found = false;
          for (auto it = b; it != e; ++it)
            if (*it == i) {
              found = (h->val[it - h->col.begin()] == v);
              break;
            }
          if (!found) symm = false;
        }
      h->symmetric = symm ? 1 : 0;
    } else {
      h->symmetric = h->opts.symmetric ? 1 : 0;
    }
    // clusters
    std::vector<std::vector<int64_t>> leaves;
    rcb_leaves(n, coords, dim, h->opts.leaf_size, leaves);
    const int nc = (int)leaves.size();
    std::vector<int> clu(n);
    std::vector<int> loc(n);
    h->perm.clear();
    for (int i = 0; i < nc; i++) {
      for (size_t q = 0; q < leaves[i].size(); q++) {
        clu[leaves[i][q]] = i;
        loc[leaves[i][q]] = (int)q;
        h->perm.push_back(leaves[i][q]);
      }
    }
    LevelPattern& L = h->L0;
    L.nclu = nc;
    L.m.resize(nc);
    for (int i = 0; i < nc; i++) L.m[i] = (int)leaves[i].size();
    h->adj0.assign(nc, {});
    for (int64_t i = 0; i < n; i++)
      for (int64_t p = h->rowptr[i]; p < h->rowptr[i + 1]; p++) {
        int a = clu[i], b = clu[h->col[p]];
        if (a != b) h->adj0[a].push_back(b);
      }
    for (int i = 0; i < nc; i++) {
      // A_B is made symmetric in structure: a nonzero (i,j) or (j,i) couples
      for (int j : std::vector<int>(h->adj0[i])) h->adj0[j].push_back(i);
    }
    for (auto& v : h->adj0) {
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    build_level_pattern(L, h->adj0);
    h->csr_dst.resize(h->nnz);
    for (int64_t i = 0; i < n; i++)
      for (int64_t p = h->rowptr[i]; p < h->rowptr[i + 1]; p++) {
        int a = clu[i], b = clu[h->col[p]];
        int64_t q = L.find(a, b);
        h->csr_dst[p] = L.off[q] + loc[i] + (int64_t)loc[h->col[p]] * L.ld[a];
      }
    // device copies
    h->d_rowptr.alloc(sizeof(int64_t) * (n + 1));
    h->d_col.alloc(sizeof(int) * std::max<int64_t>(h->nnz, 1));
    h->d_val.alloc(sizeof(double) * std::max<int64_t>(h->nnz, 1));
    h->d_csr_dst.alloc(sizeof(int64_t) * std::max<int64_t>(h->nnz, 1));
    h->d_perm.alloc(sizeof(int64_t) * n);
    h->d_err.alloc(sizeof(DevError));
    HS_CUDA(cudaMemcpyAsync(h->d_rowptr.p, h->rowptr.data(), sizeof(int64_t) * (n + 1),
                            cudaMemcpyHostToDevice, h->st));
    HS_CUDA(cudaMemcpyAsync(h->d_col.p, h->col.data(), sizeof(int) * h->nnz,
                            cudaMemcpyHostToDevice, h->st));
    HS_CUDA(cudaMemcpyAsync(h->d_val.p, h->val.data(), sizeof(double) * h->nnz,
                            cudaMemcpyHostToDevice, h->st));
    HS_CUDA(cudaMemcpyAsync(h->d_csr_dst.p, h->csr_dst.data(), sizeof(int64_t) * h->nnz,
                            cudaMemcpyHostToDevice, h->st));
    HS_CUDA(cudaMemcpyAsync(h->d_perm.p, h->perm.data(), sizeof(int64_t) * n,
                            cudaMemcpyHostToDevice, h->st));
    if (h->opts.equilibrate) {
      // S = diag(|a_ii|)^{-1/2} (duplicates summed; 1 for a zero diagonal)
      std::vector<double> dg(n, 0.0);
      for (int64_t i = 0; i < n; i++)
        for (int64_t p = h->rowptr[i]; p < h->rowptr[i + 1]; p++)
          if (h->col[p] == i) dg[i] += h->val[p];
      h->scale.resize(n);
      for (int64_t i = 0; i < n; i++)
        h->scale[i] = dg[i] != 0.0 ? 1.0 / std::sqrt(std::fabs(dg[i])) : 1.0;
      std::vector<double> fv(h->nnz);
      for (int64_t i = 0; i < n; i++)
        for (int64_t p = h->rowptr[i]; p < h->rowptr[i + 1]; p++)
          fv[p] = h->val[p] * h->scale[i] * h->scale[h->col[p]];
      h->d_fval.alloc(sizeof(double) * std::max<int64_t>(h->nnz, 1));
      h->d_scale.alloc(sizeof(double) * n);
      HS_CUDA(cudaMemcpyAsync(h->d_fval.p, fv.data(), sizeof(double) * h->nnz,
                              cudaMemcpyHostToDevice, h->st));
      HS_CUDA(cudaMemcpyAsync(h->d_scale.p, h->scale.data(), sizeof(double) * n,
                              cudaMemcpyHostToDevice, h->st));
      HS_CUDA(cudaStreamSynchronize(h->st));
    }
    HS_CUDA(cudaMemsetAsync(h->d_err.p, 0, sizeof(DevError), h->st));
    HS_CUDA(cudaStreamSynchronize(h->st));
  } catch (const Fail& f) {
    return f.code;
  } catch (const std::bad_alloc&) {
    return HSOLVE_ERR_OOM;
  }
  *out = h.release();
  return HSOLVE_OK;
}

hsolve_status hsolve_factor(hsolve_handle* h, double eps, hsolve_precision prec) {
  if (!h) return HSOLVE_ERR_ARG;
  cudaGetLastError();  // a stale error of another runtime user is not ours
  if (!(eps >= 0.0) || prec < HSOLVE_FP64 || prec > HSOLVE_MIXED_3XTF32)
    return set_err(h, HSOLVE_ERR_ARG, "bad eps or precision");
  h->factored = false;
  h->drop_graphs();
  h->F.clear();
  try {
    h->prec = prec;
    if (prec == HSOLVE_FP64)
      factor_impl<double>(h, eps);
    else
      factor_impl<float>(h, eps);
    h->factored = true;
  } catch (const Fail& f) {
    h->F.clear();
    cudaStreamSynchronize(h->st);
    cudaMemsetAsync(h->d_err.p, 0, sizeof(DevError), h->st);
    cudaStreamSynchronize(h->st);
    return set_err(h, f.code, f.msg);
  } catch (const std::bad_alloc&) {
    h->F.clear();
    return set_err(h, HSOLVE_ERR_OOM, "host allocation failed");
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_factor_forced(hsolve_handle* h, hsolve_precision prec, const int32_t* ranks,
                                   const int32_t* counts, int32_t nlevels,
                                   const int32_t* pivots) {
  if (!h || !ranks || !counts || nlevels < 1) return HSOLVE_ERR_ARG;
  h->forced.assign(nlevels, {});
  h->forced_piv.clear();
  int64_t o = 0, po = 0;
  for (int l = 0; l < nlevels; l++) {
    if (counts[l] < 0) return HSOLVE_ERR_ARG;
    h->forced[l].assign(ranks + o, ranks + o + counts[l]);
    o += counts[l];
    if (pivots) {
      int64_t np = 0;
      for (int32_t k : h->forced[l]) {
        if (k < 0) return HSOLVE_ERR_ARG;
        np += k;
      }
      h->forced_piv.emplace_back(pivots + po, pivots + po + np);
      po += np;
    }
  }
  h->force_ranks = true;
  const hsolve_status st = hsolve_factor(h, 0.0, prec);
  h->force_ranks = false;
  h->forced.clear();
  h->forced_piv.clear();
  return st;
}

hsolve_status hsolve_apply(hsolve_handle* h, const double* rhs, double* out, int nrhs, int64_t ld) {
  if (!h) return HSOLVE_ERR_ARG;
  cudaGetLastError();  // a stale error of another runtime user is not ours
  if (!h->factored) return set_err(h, HSOLVE_ERR_STATE, "apply before factor");
  if (!rhs || !out || nrhs < 1 || ld < h->n) return set_err(h, HSOLVE_ERR_ARG, "bad apply args");
  try {
    apply_any(h, rhs, out, nrhs, ld);
    HS_CUDA(cudaGetLastError());
    HS_CUDA(cudaStreamSynchronize(h->st));
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_apply_noalloc(hsolve_handle* h, const double* rhs, double* out, int nrhs,
                                   int64_t ld) {
  if (!h) return HSOLVE_ERR_ARG;
  cudaGetLastError();  // a stale error of another runtime user is not ours
  if (!h->factored) return set_err(h, HSOLVE_ERR_STATE, "apply before factor");
  if (!rhs || !out || nrhs < 1 || ld < h->n) return set_err(h, HSOLVE_ERR_ARG, "bad apply args");
  const size_t need = h->prec == HSOLVE_FP64 ? noalloc_layout<double>(h, nrhs, nullptr)
                                             : noalloc_layout<float>(h, nrhs, nullptr);
  if (need > kNoAllocScratchBytes)
    return set_err(h, HSOLVE_ERR_BUDGET,
                   "hsolve_apply_noalloc needs " + std::to_string(need) +
                       " bytes of scratch for this factorization and nrhs; the fixed scratch "
                       "holds " + std::to_string(kNoAllocScratchBytes) +
                       " bytes (use fewer right-hand sides per call, or hsolve_apply)");
  void* base = nullptr;
  std::string why;
  hsolve_status st = noalloc_scratch_address(&base, &why);
  if (st != HSOLVE_OK) return set_err(h, st, why);
  try {
    if (h->prec == HSOLVE_FP64)
      apply_scratch_impl<double>(h, rhs, out, nrhs, ld, static_cast<unsigned char*>(base));
    else
      apply_scratch_impl<float>(h, rhs, out, nrhs, ld, static_cast<unsigned char*>(base));
    HS_CUDA(cudaGetLastError());
    HS_CUDA(cudaStreamSynchronize(h->st));
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_spmv(hsolve_handle* h, const double* x, double* y, int nrhs, int64_t ld) {
  if (!h || !x || !y || nrhs < 1 || ld < h->n) return HSOLVE_ERR_ARG;
  try {
    spmv_csr(h->n, h->d_rowptr.as<int64_t>(), h->d_col.as<int>(), h->d_val.as<double>(), x, ld, y,
             ld, nrhs, h->st);
    HS_CUDA(cudaGetLastError());
    HS_CUDA(cudaStreamSynchronize(h->st));
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_tc_gemm(int mode, int M, int N, int K, const float* A, int64_t rsa,
                             int64_t csa, const float* B, int64_t rsb, int64_t csb, float* C,
                             int64_t ldc, float alpha, float beta, int lower, void* stream) {
  if (mode < 0 || mode > 2 || M < 0 || N < 0 || K < 0 || ((!A || !B) && K > 0) || !C ||
      ldc < std::max(M, 1))
    return HSOLVE_ERR_ARG;
  cudaGetLastError();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevError* err = nullptr;
  {
    std::lock_guard<std::mutex> lk(device_mutex());
    if (cudaMalloc(&err, sizeof(DevError)) != cudaSuccess) return HSOLVE_ERR_OOM;
  }
  DevError e{};
  hsolve_status rc = HSOLVE_OK;
  if (cudaMemsetAsync(err, 0, sizeof(DevError), st) != cudaSuccess) rc = HSOLVE_ERR_CUDA;
  if (rc == HSOLVE_OK) {
    tc_gemm(mode, M, N, K, A, rsa, csa, B, rsb, csb, C, ldc, alpha, beta, lower != 0, err, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&e, err, sizeof(DevError), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = HSOLVE_ERR_CUDA;
    else if (e.code != 0)
      rc = (hsolve_status)e.code;
  }
  {
    std::lock_guard<std::mutex> lk(device_mutex());
    cudaFree(err);
  }
  return rc;
}

hsolve_status hsolve_wait_selftest(int kind, int64_t limit_cycles, void* stream) {
  if (kind != 0 || limit_cycles < 0) return HSOLVE_ERR_ARG;
  cudaGetLastError();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* buf = nullptr;  // [0] error word
  {
    std::lock_guard<std::mutex> lk(device_mutex());
    if (cudaMalloc(&buf, 8 * sizeof(int)) != cudaSuccess) return HSOLVE_ERR_OOM;
  }
  int e = 0;
  hsolve_status rc = HSOLVE_OK;
  if (cudaMemsetAsync(buf, 0, 8 * sizeof(int), st) != cudaSuccess) rc = HSOLVE_ERR_CUDA;
  if (rc == HSOLVE_OK) {
    mbar_wait_probe(limit_cycles, buf, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&e, buf, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = HSOLVE_ERR_CUDA;
    else
      rc = (hsolve_status)e;
  }
  {
    std::lock_guard<std::mutex> lk(device_mutex());
    cudaFree(buf);
  }
  return rc;
}

hsolve_status hsolve_solve(hsolve_handle* h, hsolve_krylov krylov, double tol, int maxit,
                           const double* b, double* x, int nrhs, int64_t ld,
                           hsolve_solve_info* info) {
  if (!h) return HSOLVE_ERR_ARG;
  cudaGetLastError();  // a stale error of another runtime user is not ours
  if (!h->factored) return set_err(h, HSOLVE_ERR_STATE, "solve before factor");
  if (!b || !x || nrhs < 1 || ld < h->n || maxit < 1 || !(tol > 0))
    return set_err(h, HSOLVE_ERR_ARG, "bad solve args");
  hsolve_status st = HSOLVE_OK;
  try {
    cudaEvent_t e0, e1;
    HS_CUDA(cudaEventCreate(&e0));
    HS_CUDA(cudaEventCreate(&e1));
    HS_CUDA(cudaEventRecord(e0, h->st));
    int it = 0;
    double rr = 0;
    if (krylov == HSOLVE_PCG) {
      hsolve_solve_info tmp{};
      st = pcg_impl(h, tol, maxit, b, x, nrhs, ld, &tmp);
      it = tmp.iterations;
      rr = tmp.rel_residual;
    } else {
      st = fgmres_batch(h, tol, maxit, b, x, nrhs, ld, h->opts.gmres_restart, &it, &rr);
    }
    HS_CUDA(cudaEventRecord(e1, h->st));
    HS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
      info->iterations = it;
      info->rel_residual = rr;
      info->factor_ms = h->factor_ms;
      info->solve_ms = ms;
    }
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  if (st == HSOLVE_ERR_NO_CONVERGENCE) set_err(h, st, "Krylov solve did not converge");
  return st;
}

hsolve_status hsolve_solve_host(hsolve_handle* h, hsolve_krylov krylov, double tol, int maxit,
                                const double* b, double* x, int nrhs, int64_t ld,
                                hsolve_solve_info* info) {
  if (!h) return HSOLVE_ERR_ARG;
  if (!b || !x || nrhs < 1 || ld < h->n) return set_err(h, HSOLVE_ERR_ARG, "bad solve args");
  DevBuf db, dx;
  try {
    db.alloc(sizeof(double) * h->n * nrhs);
    dx.alloc(sizeof(double) * h->n * nrhs);
    for (int c = 0; c < nrhs; c++)
      HS_CUDA(cudaMemcpyAsync(db.as<double>() + c * h->n, b + c * ld, sizeof(double) * h->n,
                              cudaMemcpyHostToDevice, h->st));
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  hsolve_status st = hsolve_solve(h, krylov, tol, maxit, db.as<double>(), dx.as<double>(), nrhs,
                                  h->n, info);
  if (st != HSOLVE_OK && st != HSOLVE_ERR_NO_CONVERGENCE) return st;
  try {
    for (int c = 0; c < nrhs; c++)
      HS_CUDA(cudaMemcpyAsync(x + c * ld, dx.as<double>() + c * h->n, sizeof(double) * h->n,
                              cudaMemcpyDeviceToHost, h->st));
    HS_CUDA(cudaStreamSynchronize(h->st));
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return st;
}

hsolve_status hsolve_get_stats(const hsolve_handle* h, hsolve_stats* o) {
  if (!h || !o) return HSOLVE_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->levels = (int)h->F.size();
  o->clusters0 = h->L0.nclu;
  o->colours_total = h->colours_total;
  o->top_size = 0;
  if (!h->F.empty() && h->F.back()->top) o->top_size = h->F.back()->P.m[0];
  o->coarse_total = h->coarse_total;
  o->factor_bytes = h->factor_bytes;
  o->block_bytes = h->block_bytes;
  o->apply_bytes = h->apply_bytes;
  o->factor_flops = h->factor_flops;
  o->schur_flops = h->schur_flops;
  o->prep_flops = h->prep_flops;
  o->gemm_flops = h->gemm_flops;
  o->kernel_launches = h->launches;
  o->precision = h->prec;
  o->launches_total = launches_total();
  o->qr_flops = h->qr_flops;
  return HSOLVE_OK;
}

hsolve_status hsolve_get_level(const hsolve_handle* h, int level, int32_t* nclu, int32_t* sizes,
                               int32_t* ranks, int32_t* colour, int32_t cap) {
  if (!h || !nclu || level < 0) return HSOLVE_ERR_ARG;
  if (level >= (int)h->F.size()) return HSOLVE_ERR_ARG;
  const FLevel& F = *h->F[level];
  *nclu = F.P.nclu;
  for (int i = 0; i < F.P.nclu && i < cap; i++) {
    if (sizes) sizes[i] = F.P.m[i];
    if (ranks) ranks[i] = i < (int)F.k.size() ? F.k[i] : 0;
    if (colour) colour[i] = F.P.colour[i];
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_export_level(const hsolve_handle* hc, int level, hsolve_level_export* info,
                                  hsolve_cluster_export* clusters, double* fac, int32_t* pivots,
                                  int32_t* nbr_id, int32_t* nbr_w) {
  hsolve_handle* h = const_cast<hsolve_handle*>(hc);
  if (!h || !info) return HSOLVE_ERR_ARG;
  if (!h->factored) return set_err(h, HSOLVE_ERR_STATE, "export before factor");
  if (level < 0 || level >= (int)h->F.size()) return set_err(h, HSOLVE_ERR_ARG, "no such level");
  const FLevel& F = *h->F[level];
  const int nc = F.P.nclu;
  const bool have = !F.hrecs.empty();  // false: a level that only merged into the top
  const size_t esz = h->prec == HSOLVE_FP64 ? sizeof(double) : sizeof(float);
  std::memset(info, 0, sizeof(*info));
  info->nclu = nc;
  info->dense_top = F.top ? 1 : 0;
  info->symmetric = h->symmetric;
  info->precision = h->prec;
  info->fac_elems = have ? (int64_t)(F.fac.bytes / esz) : 0;
  info->nbr_total = (int64_t)F.nb_id.size();
  int64_t np = 0;
  if (have)
    for (int s = 0; s < nc; s++) np += F.hrecs[s].m > 0 ? F.hrecs[s].k : 0;
  info->piv_total = np;
  try {
    if (clusters) {
      int64_t po = 0;
      for (int s = 0; s < nc; s++) {
        hsolve_cluster_export& c = clusters[s];
        std::memset(&c, 0, sizeof(c));
        c.colour = s < (int)F.P.colour.size() ? F.P.colour[s] : 0;
        c.T = c.TR = c.Y = c.XT = -1;
        c.piv = po;
        c.nb = have ? F.nb_ptr[s] : 0;
        if (!have) continue;
        const ApplyRec& r = F.hrecs[s];
        c.m = r.m;
        c.k = r.m > 0 ? r.k : 0;
        c.nw = r.nw;
        c.nnb = F.nb_ptr[s + 1] - F.nb_ptr[s];
        c.npiv = c.k;
        po += c.npiv;
        if (r.m > 0 && r.k < r.m) {
          c.T = r.T;
          c.Y = r.nw > 0 ? r.Y : -1;
          if (!r.sym) {
            c.TR = r.TR;
            c.XT = r.nw > 0 ? r.XT : -1;
          }
        }
      }
    }
    if (fac && have && info->fac_elems > 0) {
      std::vector<char> buf(F.fac.bytes);
      HS_CUDA(cudaMemcpyAsync(buf.data(), F.fac.p, F.fac.bytes, cudaMemcpyDeviceToHost, h->st));
      HS_CUDA(cudaStreamSynchronize(h->st));
      if (esz == sizeof(double)) {
        std::memcpy(fac, buf.data(), sizeof(double) * info->fac_elems);
      } else {
        const float* f = reinterpret_cast<const float*>(buf.data());
        for (int64_t i = 0; i < info->fac_elems; i++) fac[i] = f[i];
      }
    }
    if (pivots && have && np > 0) {
      std::vector<int> all((size_t)std::max<int64_t>(F.P.voff[nc], 1));
      HS_CUDA(cudaMemcpyAsync(all.data(), F.piv.p, sizeof(int) * F.P.voff[nc],
                              cudaMemcpyDeviceToHost, h->st));
      HS_CUDA(cudaStreamSynchronize(h->st));
      int64_t po = 0;
      for (int s = 0; s < nc; s++) {
        const ApplyRec& r = F.hrecs[s];
        if (r.m == 0) continue;
        for (int j = 0; j < r.k; j++) pivots[po + j] = all[F.P.voff[s] + j];
        po += r.k;
      }
    }
    if (nbr_id)
      for (size_t i = 0; i < F.nb_id.size(); i++) nbr_id[i] = F.nb_id[i];
    if (nbr_w)
      for (size_t i = 0; i < F.nb_w.size(); i++) nbr_w[i] = F.nb_w[i];
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_export_cluster(const hsolve_handle* hc, int level, int cluster,
                                    hsolve_cluster_export* rec, double* T, double* TRt,
                                    double* Y, double* XT, int32_t* pivots, int32_t* nbr_id,
                                    int32_t* nbr_w) {
  hsolve_handle* h = const_cast<hsolve_handle*>(hc);
  if (!h || !rec) return HSOLVE_ERR_ARG;
  if (!h->factored) return set_err(h, HSOLVE_ERR_STATE, "export before factor");
  if (level < 0 || level >= (int)h->F.size()) return set_err(h, HSOLVE_ERR_ARG, "no such level");
  const FLevel& F = *h->F[level];
  if (cluster < 0 || cluster >= F.P.nclu) return set_err(h, HSOLVE_ERR_ARG, "no such cluster");
  std::memset(rec, 0, sizeof(*rec));
  rec->T = rec->TR = rec->Y = rec->XT = -1;
  rec->colour = cluster < (int)F.P.colour.size() ? F.P.colour[cluster] : 0;
  if (F.hrecs.empty()) return HSOLVE_OK;  // a level that only merged into the top
  const ApplyRec& r = F.hrecs[cluster];
  rec->m = r.m;
  rec->k = r.m > 0 ? r.k : 0;
  rec->nw = r.nw;
  rec->nnb = F.nb_ptr[cluster + 1] - F.nb_ptr[cluster];
  rec->npiv = rec->k;
  const bool have = r.m > 0 && r.k < r.m;
  if (have) {
    rec->T = 0;
    if (!r.sym) rec->TR = 0;
    if (r.nw > 0) {
      rec->Y = 0;
      if (!r.sym) rec->XT = 0;
    }
  }
  const size_t esz = h->prec == HSOLVE_FP64 ? sizeof(double) : sizeof(float);
  try {
    auto fetch = [&](int64_t off, int64_t elems, double* dst) {
      if (!dst || off < 0 || elems <= 0) return;
      std::vector<char> buf((size_t)elems * esz);
      HS_CUDA(cudaMemcpyAsync(buf.data(), F.fac.as<char>() + off * (int64_t)esz, buf.size(),
                              cudaMemcpyDeviceToHost, h->st));
      HS_CUDA(cudaStreamSynchronize(h->st));
      if (esz == sizeof(double)) {
        std::memcpy(dst, buf.data(), buf.size());
      } else {
        const float* f = reinterpret_cast<const float*>(buf.data());
        for (int64_t i = 0; i < elems; i++) dst[i] = f[i];
      }
    };
    if (have) {
      const int64_t mm = (int64_t)r.m * r.m, mw = (int64_t)r.m * r.nw;
      fetch(r.T, mm, T);
      if (!r.sym) fetch(r.TR, mm, TRt);
      fetch(r.Y, mw, Y);
      if (!r.sym) fetch(r.XT, mw, XT);
    }
    if (pivots && rec->k > 0) {
      std::vector<int> pv(rec->k);
      HS_CUDA(cudaMemcpyAsync(pv.data(), F.piv.as<int>() + F.P.voff[cluster], sizeof(int) * pv.size(),
                              cudaMemcpyDeviceToHost, h->st));
      HS_CUDA(cudaStreamSynchronize(h->st));
      for (int j = 0; j < rec->k; j++) pivots[j] = pv[j];
    }
    for (int q = 0; q < rec->nnb; q++) {
      if (nbr_id) nbr_id[q] = F.nb_id[F.nb_ptr[cluster] + q];
      if (nbr_w) nbr_w[q] = F.nb_w[F.nb_ptr[cluster] + q];
    }
  } catch (const Fail& f) {
    return set_err(h, f.code, f.msg);
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_get_perm(const hsolve_handle* h, int64_t* perm) {
  if (!h || !perm) return HSOLVE_ERR_ARG;
  std::memcpy(perm, h->perm.data(), sizeof(int64_t) * h->n);
  return HSOLVE_OK;
}

hsolve_status hsolve_get_phase_times(const hsolve_handle* h, hsolve_phase_time* out, int32_t cap,
                                     int32_t* count) {
  if (!h || !count) return HSOLVE_ERR_ARG;
  resolve_pending(const_cast<hsolve_handle*>(h));
  *count = (int)h->phases.size();
  for (int i = 0; i < (int)h->phases.size() && i < cap && out; i++) {
    std::memset(&out[i], 0, sizeof(out[i]));
    std::snprintf(out[i].name, sizeof(out[i].name), "%s", h->phases[i].name.c_str());
    out[i].ms = h->phases[i].ms;
    out[i].launches = h->phases[i].launches;
  }
  return HSOLVE_OK;
}

hsolve_status hsolve_set_profiling(hsolve_handle* h, int on) {
  if (!h) return HSOLVE_ERR_ARG;
  h->profiling = on != 0;
  h->profile_levels = on == 2;
  h->profile_deferred = on == 3;
  return HSOLVE_OK;
}

const char* hsolve_last_error(const hsolve_handle* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

void hsolve_destroy(hsolve_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

}  // extern "C"
