// Serving runtime: a request loop over the solver library for a stream of
// solves of different matrices (the service view of Sec. 1: factor once,
// solve many right-hand sides).
//
// Requests (matrix id, host right-hand sides) are queued by
// hsolve_server_submit and served by a fixed set of worker threads.  A worker
// takes the oldest request whose matrix no other worker is serving, batches
// every queued request of that matrix behind it (up to max_batch_rhs columns:
// continuous batching -- requests that arrive while a batch runs join the
// next one), makes the matrix's factorization resident if it is not (analysis
// and factorization on the matrix's own CUDA stream, evicting the least
// recently used idle factorizations while the resident bytes would exceed the
// memory budget), copies the batch's right-hand sides to the device once,
// solves them with one hsolve_solve call and hands each request its columns.  Different matrices are served by
// different workers at the same time, so their kernels overlap on the
// device.  Each column of a batched solve follows the same arithmetic as a
// solve of that column alone (the Krylov methods and the substitution sweeps
// treat right-hand sides independently), so a result does not depend on the
// company it was batched with.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <string>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "hsolve.h"

namespace hs {
std::mutex& device_mutex();  // the library's lock around allocation and capture
}

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Matrix {
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> coords;
  int dim = 0;
  hsolve_opts opts{};
  double eps = 0;
  hsolve_precision prec = HSOLVE_FP64;
  hsolve_krylov krylov = HSOLVE_PCG;
  double tol = 1e-10;
  int maxit = 500;
  hsolve_handle* h = nullptr;  // resident factorization, or null
  cudaStream_t st = nullptr;
  // batch staging: pinned host and device right-hand sides / solutions
  double* hb = nullptr;
  double* db = nullptr;
  double* dx = nullptr;
  int64_t cap = 0;  // columns the staging holds
  int64_t bytes = 0;            // device bytes charged while resident
  int64_t last_bytes = 0;       // measured size of the previous residency
  bool busy = false;
  int64_t last_use = 0;
};

struct Request {
  int32_t matrix = 0;
  int32_t nrhs = 0;
  std::vector<double> b, x;
  Clock::time_point t_submit, t_start, t_done;
  hsolve_server_result res{};
  bool done = false;
};

}  // namespace

struct hsolve_server {
  hsolve_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::unique_ptr<Matrix>> mats;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 1;
  int64_t tick = 0;
  int64_t resident_bytes = 0;
  hsolve_server_stats stats{};

  // a queued request that can start now: its matrix is idle and either
  // resident or admissible under the budget once idle residents are evicted
  bool admissible(const Matrix& M) const {
    if (M.h || opts.memory_budget <= 0) return true;
    // bytes held by matrices being served (a factorization in progress is
    // charged its estimate before its handle exists)
    int64_t busy_bytes = 0;
    for (auto& m : mats)
      if (m->busy) busy_bytes += m->bytes;
    return busy_bytes + estimate(M) <= opts.memory_budget || busy_bytes == 0;
  }
  int64_t estimate(const Matrix& M) const {
    if (M.last_bytes > 0) return M.last_bytes;
    // blocks, factors and workspace of a first factorization: a few
    // kilobytes per unknown for the usual 3D cluster sizes
    const int64_t per = M.prec == HSOLVE_FP64 ? 24 * 1024 : 12 * 1024;
    return M.n * per;
  }
  int pick() const {
    for (size_t i = 0; i < queue.size(); i++) {
      const Request& r = *reqs.at(queue[i]);
      const Matrix& M = *mats[r.matrix];
      if (!M.busy && admissible(M)) return (int)i;
    }
    return -1;
  }
  void evict_for(int64_t need) {
    while (opts.memory_budget > 0 && resident_bytes + need > opts.memory_budget) {
      Matrix* victim = nullptr;
      for (auto& m : mats)
        if (m->h && !m->busy && (!victim || m->last_use < victim->last_use)) victim = m.get();
      if (!victim) break;
      hsolve_destroy(victim->h);
      victim->h = nullptr;
      {
        std::lock_guard<std::mutex> dl(hs::device_mutex());
        if (victim->db) cudaFree(victim->db);
        if (victim->dx) cudaFree(victim->dx);
        if (victim->hb) cudaFreeHost(victim->hb);
      }
      victim->db = victim->dx = nullptr;
      victim->hb = nullptr;
      victim->cap = 0;
      resident_bytes -= victim->bytes;
      victim->bytes = 0;
      stats.evictions++;
    }
  }
  void worker();
};

void hsolve_server::worker() {
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    int qi = -1;
    cv_work.wait(lk, [&] { return stop || (qi = pick()) >= 0; });
    if (qi < 0) return;  // stopping with nothing startable
    const int64_t first = queue[qi];
    const int mid = reqs[first]->matrix;
    Matrix& M = *mats[mid];
    M.busy = true;
    // batch: every queued request of this matrix, oldest first
    std::vector<Request*> batch;
    int tot = 0;
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = reqs[*it].get();
      if (r->matrix == mid && (batch.empty() || tot + r->nrhs <= opts.max_batch_rhs)) {
        batch.push_back(r);
        tot += r->nrhs;
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
    const auto t_start = Clock::now();
    for (Request* r : batch) r->t_start = t_start;
    bool factored = false;
    if (!M.h) {
      const int64_t need = estimate(M);
      evict_for(need);
      resident_bytes += need;
      M.bytes = need;
      factored = true;
    }
    lk.unlock();

    hsolve_status st = HSOLVE_OK;
    if (factored) {
      if (!M.st) cudaStreamCreateWithFlags(&M.st, cudaStreamNonBlocking);
      hsolve_csr A{M.n, (int64_t)M.col.size(), M.rowptr.data(), M.col.data(), M.val.data()};
      st = hsolve_analyze(&A, M.coords.empty() ? nullptr : M.coords.data(), M.dim, &M.opts,
                          M.st, &M.h);
      if (st == HSOLVE_OK) st = hsolve_factor(M.h, M.eps, M.prec);
    }
    // staging: the batch's right-hand sides into pinned memory, one copy to
    // the device, the solve, one copy back (the buffers persist per matrix)
    if (st == HSOLVE_OK && M.cap < tot) {
      std::lock_guard<std::mutex> dl(hs::device_mutex());
      if (M.hb) cudaFreeHost(M.hb);
      if (M.db) cudaFree(M.db);
      if (M.dx) cudaFree(M.dx);
      M.hb = M.db = M.dx = nullptr;
      M.cap = 0;
      const size_t bytes = sizeof(double) * (size_t)M.n * tot;
      if (cudaMallocHost(&M.hb, bytes) != cudaSuccess || cudaMalloc(&M.db, bytes) != cudaSuccess ||
          cudaMalloc(&M.dx, bytes) != cudaSuccess) {
        cudaGetLastError();
        st = HSOLVE_ERR_OOM;
      } else {
        M.cap = tot;
      }
    }
    hsolve_solve_info info{};
    if (st == HSOLVE_OK) {
      int64_t c0 = 0;
      for (Request* r : batch) {
        std::memcpy(M.hb + c0 * M.n, r->b.data(), sizeof(double) * M.n * r->nrhs);
        c0 += r->nrhs;
      }
      const size_t bytes = sizeof(double) * (size_t)M.n * tot;
      if (cudaMemcpyAsync(M.db, M.hb, bytes, cudaMemcpyHostToDevice, M.st) != cudaSuccess)
        st = HSOLVE_ERR_CUDA;
      if (st == HSOLVE_OK)
        st = hsolve_solve(M.h, M.krylov, M.tol, M.maxit, M.db, M.dx, tot, M.n, &info);
      if (st == HSOLVE_OK || st == HSOLVE_ERR_NO_CONVERGENCE) {
        if (cudaMemcpyAsync(M.hb, M.dx, bytes, cudaMemcpyDeviceToHost, M.st) != cudaSuccess ||
            cudaStreamSynchronize(M.st) != cudaSuccess)
          st = HSOLVE_ERR_CUDA;
      }
    }
    hsolve_stats hs{};
    if (M.h) hsolve_get_stats(M.h, &hs);
    std::string msg;
    if (st != HSOLVE_OK && M.h) msg = hsolve_last_error(M.h);

    lk.lock();
    const auto t_done = Clock::now();
    // a failed batch (other than a plain non-convergence) leaves no handle
    // behind: the matrix's next batch analyses and factors it again
    const bool keep = M.h && (st == HSOLVE_OK || st == HSOLVE_ERR_NO_CONVERGENCE);
    if (!factored && !keep && M.h) {
      hsolve_destroy(M.h);
      M.h = nullptr;
      resident_bytes -= M.bytes;
      M.bytes = 0;
    }
    if (factored) {
      if (keep) {
        // charge the measured size: factors plus the largest level's blocks
        const int64_t real_bytes = hs.factor_bytes + hs.block_bytes;
        resident_bytes += real_bytes - M.bytes;
        M.bytes = real_bytes;
        M.last_bytes = real_bytes;
        stats.factorizations++;
      } else {
        if (M.h) hsolve_destroy(M.h);
        M.h = nullptr;
        resident_bytes -= M.bytes;
        M.bytes = 0;
      }
    }
    int64_t c0 = 0;
    for (Request* r : batch) {
      if (M.hb && M.cap >= tot)
        r->x.assign(M.hb + c0 * M.n, M.hb + (c0 + r->nrhs) * M.n);
      r->b.clear();
      r->b.shrink_to_fit();
      c0 += r->nrhs;
      r->t_done = t_done;
      r->res.status = (int32_t)st;
      std::snprintf(r->res.message, sizeof(r->res.message), "%s", msg.c_str());
      r->res.iterations = info.iterations;
      r->res.rel_residual = info.rel_residual;
      r->res.queue_ms = ms_between(r->t_submit, r->t_start);
      r->res.service_ms = ms_between(r->t_start, t_done);
      r->res.latency_ms = ms_between(r->t_submit, t_done);
      r->res.batch_rhs = tot;
      r->res.factored = factored ? 1 : 0;
      r->done = true;
    }
    stats.batches++;
    stats.requests_done += (int64_t)batch.size();
    stats.rhs_done += tot;
    M.busy = false;
    M.last_use = ++tick;
    int resident = 0;
    for (auto& m : mats) resident += m->h != nullptr;
    stats.resident = resident;
    stats.resident_bytes = resident_bytes;
    stats.peak_resident_bytes = std::max(stats.peak_resident_bytes, resident_bytes);
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

void hsolve_server_default_opts(hsolve_server_opts* o) {
  if (!o) return;
  o->memory_budget = 60ll << 30;
  o->max_batch_rhs = 256;
  o->workers = 4;
}

hsolve_status hsolve_server_create(const hsolve_server_opts* opts, hsolve_server** out) {
  if (!out) return HSOLVE_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hsolve_server> s(new hsolve_server());
  hsolve_server_default_opts(&s->opts);
  if (opts) s->opts = *opts;
  if (s->opts.workers < 1 || s->opts.workers > 64 || s->opts.max_batch_rhs < 1 ||
      s->opts.memory_budget < 0)
    return HSOLVE_ERR_ARG;
  for (int w = 0; w < s->opts.workers; w++)
    s->workers.emplace_back([p = s.get()] { p->worker(); });
  *out = s.release();
  return HSOLVE_OK;
}

hsolve_status hsolve_server_add_matrix(hsolve_server* s, const hsolve_csr* A,
                                       const double* coords, int dim, const hsolve_opts* opts,
                                       double eps, hsolve_precision prec, hsolve_krylov krylov,
                                       double tol, int maxit, int32_t* matrix_id) {
  if (!s || !A || !matrix_id || A->n <= 0 || !A->rowptr || !A->col || !A->val || !(tol > 0) ||
      maxit < 1 || !(eps >= 0) || (coords && (dim < 1 || dim > 3)))
    return HSOLVE_ERR_ARG;
  std::unique_ptr<Matrix> M(new Matrix());
  M->n = A->n;
  M->rowptr.assign(A->rowptr, A->rowptr + A->n + 1);
  M->col.assign(A->col, A->col + A->nnz);
  M->val.assign(A->val, A->val + A->nnz);
  if (coords) M->coords.assign(coords, coords + A->n * dim);
  M->dim = coords ? dim : 0;
  hsolve_default_opts(&M->opts);
  if (opts) M->opts = *opts;
  M->eps = eps;
  M->prec = prec;
  M->krylov = krylov;
  M->tol = tol;
  M->maxit = maxit;
  std::lock_guard<std::mutex> lk(s->mu);
  *matrix_id = (int32_t)s->mats.size();
  s->mats.push_back(std::move(M));
  return HSOLVE_OK;
}

hsolve_status hsolve_server_submit(hsolve_server* s, int32_t matrix_id, const double* b,
                                   int32_t nrhs, int64_t ld, int64_t* request_id) {
  if (!s || !b || !request_id || nrhs < 1) return HSOLVE_ERR_ARG;
  std::unique_ptr<Request> r(new Request());
  int64_t n = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (matrix_id < 0 || matrix_id >= (int32_t)s->mats.size()) return HSOLVE_ERR_ARG;
    n = s->mats[matrix_id]->n;
  }
  if (ld < n) return HSOLVE_ERR_ARG;
  r->matrix = matrix_id;
  r->nrhs = nrhs;
  r->b.resize((size_t)n * nrhs);
  for (int c = 0; c < nrhs; c++) std::memcpy(r->b.data() + c * n, b + c * ld, sizeof(double) * n);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t id = s->next_id++;
  s->reqs[id] = std::move(r);
  s->queue.push_back(id);
  s->stats.requests_submitted++;
  s->cv_work.notify_one();
  *request_id = id;
  return HSOLVE_OK;
}

hsolve_status hsolve_server_wait(hsolve_server* s, int64_t request_id, double* x, int64_t ld,
                                 hsolve_server_result* res, double timeout_s) {
  if (!s) return HSOLVE_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return HSOLVE_ERR_ARG;
  Request* r = it->second.get();
  const int64_t n = s->mats[r->matrix]->n;
  if (x && ld < n) return HSOLVE_ERR_ARG;
  const auto deadline =
      Clock::now() + std::chrono::microseconds((int64_t)(std::max(0.0, timeout_s) * 1e6));
  if (!s->cv_done.wait_until(lk, deadline, [&] { return r->done; })) return HSOLVE_ERR_TIMEOUT;
  if (x)
    for (int c = 0; c < r->nrhs; c++)
      std::memcpy(x + c * ld, r->x.data() + (size_t)c * n, sizeof(double) * n);
  if (res) *res = r->res;
  const hsolve_status st = (hsolve_status)r->res.status;
  s->reqs.erase(it);
  return st;
}

hsolve_status hsolve_server_get_stats(hsolve_server* s, hsolve_server_stats* out) {
  if (!s || !out) return HSOLVE_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  return HSOLVE_OK;
}

void hsolve_server_destroy(hsolve_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& m : s->mats) {
    if (m->h) hsolve_destroy(m->h);
    std::lock_guard<std::mutex> dl(hs::device_mutex());
    if (m->hb) cudaFreeHost(m->hb);
    if (m->db) cudaFree(m->db);
    if (m->dx) cudaFree(m->dx);
    if (m->st) cudaStreamDestroy(m->st);
  }
  delete s;
}

}  // extern "C"
