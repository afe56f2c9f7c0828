// Serving loop: scattering requests of different geometries, wavenumbers and right-hand-side counts
// are admitted by device memory and solved concurrently, each on its own CUDA stream, so the work of
// admitted requests overlaps on the device; a request that arrives while others run starts as soon
// as a slot and enough memory are free (continuous admission, not a queue drained one at a time).
//
// Every request is the whole path: host plan (cluster tree, lists), device set-up, right-hand sides,
// GMRES, far field at the requested directions.  The host plan gives the exact device bytes the
// request will hold, which the admission test compares with the budget.
//
// Batching and residency.  Requests for the same problem (same geometry handle and options, i.e. the
// same operator) that wait in the queue when a worker picks one of them are merged into one
// multi-right-hand-side solve: their incident directions become columns of one GMRES run, so every
// matrix-vector product, Gram-Schmidt pass and far-field launch serves all of them at once; each
// request then gets its own columns' far field.  A finished problem stays resident on the device (its
// tree, near-field blocks and tables) in a least-recently-used cache, so a later request for the same
// problem skips the set-up; cached problems count against the memory budget and are evicted, oldest
// first, when an admission needs their memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

struct igabem_request {
  igabem_server *srv = nullptr;
  igabem_geom *geom = nullptr;
  igabem_options opt{};
  int R = 0, n_dir = 0;
  std::vector<double> dirs, xhat;
  std::vector<double> uinf;          // [n_dir][R] complex, filled at completion
  igabem_solve_info info{};
  int status = IGABEM_OK;
  std::string error;
  double t_submit = 0, t_start = 0, t_done = 0;
  size_t bytes = 0;
  bool done = false;
  std::mutex mu;
  std::condition_variable cv;
};

// a resident problem: set up once, reused by later requests with the same key
struct CachedProblem {
  igabem_geom *geom = nullptr;
  igabem_options opt{};
  igabem_problem *P = nullptr;
  size_t bytes = 0;       // device memory it holds (set-up arena and work buffers)
  bool busy = false;      // taken by a worker
};

struct igabem_server {
  igabem_ctx *ctx = nullptr;
  size_t budget = 0;
  int slots = 1;
  std::deque<igabem_request *> queue;
  std::mutex mu;
  std::condition_variable cv_queue, cv_mem;
  size_t in_use = 0, peak_bytes = 0;   // in_use includes the resident cache
  int active = 0, peak_active = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::deque<CachedProblem> cache;     // least recently used first
  int max_merge_cols = 256;
  // statistics
  long submitted = 0, completed = 0, failed = 0, merged = 0, cache_hits = 0;
  std::vector<double> latency_ms;
  double t_first = 0, t_last = 0;
};

namespace igabem {

namespace {

void finish(igabem_request *r, int status, const std::string &err) {
  std::lock_guard<std::mutex> lk(r->mu);
  r->status = status;
  r->error = err;
  r->t_done = now_ms();
  r->done = true;
  r->cv.notify_all();
}

bool same_problem(const igabem_geom *g1, const igabem_options &o1, const igabem_geom *g2, const igabem_options &o2) {
  return g1 == g2 && std::memcmp(&o1, &o2, sizeof(igabem_options)) == 0;
}

size_t problem_bytes(igabem_problem *P) {
  igabem_info I{};
  igabem_problem_info(P, &I);
  return I.device_bytes;
}

// frees the least recently used idle cached problems until `need` more bytes fit (lock held)
void evict_for(igabem_server *S, size_t need) {
  for (auto it = S->cache.begin(); it != S->cache.end() && S->in_use + need > S->budget;) {
    if (it->busy) {
      ++it;
      continue;
    }
    S->in_use -= it->bytes;
    problem_release(it->P);
    it = S->cache.erase(it);
  }
}

// One worker: takes the oldest waiting request and every queued request for the same problem (merged
// into one multi-column solve), finds the problem in the resident cache or plans it on the host and
// waits until its device memory fits the budget, then runs it on the worker's own stream.
void worker_loop(igabem_server *S) {
  cudaSetDevice(S->ctx->device);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  for (;;) {
    std::vector<igabem_request *> batch;
    igabem_problem *P = nullptr;
    size_t held = 0;          // bytes of a cached problem taken by this worker
    bool from_cache = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_queue.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) break;
      batch.push_back(S->queue.front());
      S->queue.pop_front();
      int cols = batch[0]->R;
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        if (same_problem((*it)->geom, (*it)->opt, batch[0]->geom, batch[0]->opt) &&
            cols + (*it)->R <= S->max_merge_cols) {
          cols += (*it)->R;
          batch.push_back(*it);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
      S->merged += (long)batch.size() - 1;
      for (auto &c : S->cache)
        if (!c.busy && same_problem(c.geom, c.opt, batch[0]->geom, batch[0]->opt)) {
          c.busy = true;
          P = c.P;
          held = c.bytes;
          from_cache = true;
          S->cache_hits += 1;
          break;
        }
    }
    igabem_request *r = batch[0];
    int R = 0;
    for (auto *q : batch) R += q->R;
    int status = IGABEM_OK;
    std::string err;
    size_t need = 0;
    bool admitted = false;
    try {
      if (!P) P = problem_plan(r->geom, &r->opt);
      const size_t work = problem_work_bytes(P->S, R, std::max(1, r->opt.gmres_restart), r->opt.precision);
      need = from_cache ? (work > held - P->arena.cap ? work - (held - P->arena.cap) : 0) + (size_t(64) << 20)
                        : P->arena_bytes + P->temp_bytes + work + (size_t(64) << 20);
      for (auto *q : batch) q->bytes = need;
      if (need > S->budget) {
        status = IGABEM_ENOMEM;
        err = "request needs " + std::to_string(need >> 20) + " MiB, more than the server's budget of " +
              std::to_string(S->budget >> 20) + " MiB";
      } else {
        std::unique_lock<std::mutex> lk(S->mu);
        evict_for(S, need);
        S->cv_mem.wait(lk, [&] {
          evict_for(S, need);
          return S->in_use + need <= S->budget;
        });
        S->in_use += need;
        S->active += 1;
        S->peak_bytes = std::max(S->peak_bytes, S->in_use);
        S->peak_active = std::max(S->peak_active, S->active);
        admitted = true;
      }
      if (admitted) {
        const double t0 = now_ms();
        for (auto *q : batch) q->t_start = t0;
        if (from_cache) P->stream = st;
        else problem_materialize(P, st);
        std::vector<double> dirs;
        for (auto *q : batch) dirs.insert(dirs.end(), q->dirs.begin(), q->dirs.end());
        std::vector<double> dens(2 * (size_t)P->S.N * R);
        igabem_solve_info info{};
        int rc = igabem_solve(P, R, dirs.data(), dens.data(), &info);
        if (rc != IGABEM_OK && rc != IGABEM_ENOT_CONVERGED) {
          status = rc;
          err = igabem_last_error();
        } else {
          if (rc == IGABEM_ENOT_CONVERGED) {
            status = rc;
            err = igabem_last_error();
          }
          // each request's far field from its own columns of the density
          int c0 = 0;
          for (auto *q : batch) {
            q->info = info;
            std::vector<double> dq(2 * (size_t)P->S.N * q->R);
            for (long i = 0; i < P->S.N; ++i)
              std::memcpy(&dq[2 * (size_t)i * q->R], &dens[2 * ((size_t)i * R + c0)], 2 * sizeof(double) * q->R);
            q->uinf.assign(2 * (size_t)q->n_dir * q->R, 0.0);
            int rf = igabem_farfield(P, q->R, dq.data(), q->n_dir, q->xhat.data(), q->uinf.data());
            if (rf != IGABEM_OK && status == IGABEM_OK) {
              status = rf;
              err = igabem_last_error();
            }
            c0 += q->R;
          }
        }
      }
    } catch (...) {
      if (status == IGABEM_OK) {
        status = IGABEM_ECUDA;
        err = igabem_last_error();
        if (err.empty()) err = "request set-up failed";
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (admitted) {
        S->in_use -= need;
        S->active -= 1;
      }
      // keep a healthy problem resident (its bytes stay in in_use), drop a failed one
      const bool keep = P && admitted && (status == IGABEM_OK || status == IGABEM_ENOT_CONVERGED);
      if (from_cache) {
        for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
          if (it->P == P) {
            S->in_use -= it->bytes;
            S->cache.erase(it);
            break;
          }
      }
      if (keep) {
        CachedProblem c;
        c.geom = r->geom;
        c.opt = r->opt;
        c.P = P;
        c.bytes = problem_bytes(P);
        S->in_use += c.bytes;
        S->cache.push_back(c);
        P = nullptr;
      }
      for (auto *q : batch) {
        S->completed += status == IGABEM_OK ? 1 : 0;
        S->failed += status == IGABEM_OK ? 0 : 1;
      }
      double t = now_ms();
      if (status == IGABEM_OK)
        for (auto *q : batch) S->latency_ms.push_back(t - q->t_submit);
      S->t_last = t;
      if (S->in_use > S->budget) evict_for(S, 0);
    }
    if (P) problem_release(P);
    S->cv_mem.notify_all();
    for (auto *q : batch) finish(q, status, err);
  }
  cudaStreamDestroy(st);
}

int refuse(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

}  // namespace

}  // namespace igabem

using namespace igabem;

extern "C" {

int igabem_server_create(igabem_ctx *ctx, size_t memory_budget, int max_active, igabem_server **out) {
  if (!ctx || !out || max_active <= 0 || max_active > 64) return refuse(IGABEM_EINVAL, "invalid server arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return refuse(IGABEM_ECUDA, "cudaSetDevice failed");
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return refuse(IGABEM_ECUDA, "cudaMemGetInfo failed");
  auto *S = new igabem_server();
  S->ctx = ctx;
  S->budget = memory_budget ? std::min(memory_budget, free_b) : (size_t)(0.9 * free_b);
  S->slots = max_active;
  for (int i = 0; i < max_active; ++i) S->workers.emplace_back(worker_loop, S);
  *out = S;
  set_error("");
  return IGABEM_OK;
}

int igabem_server_destroy(igabem_server *S) {
  if (!S) return IGABEM_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_queue.notify_all();
  for (auto &t : S->workers) t.join();
  for (auto &c : S->cache) problem_release(c.P);
  S->cache.clear();
  delete S;
  return IGABEM_OK;
}

int igabem_submit(igabem_server *S, igabem_geom *geom, const igabem_options *opt, int n_rhs, const double *dirs,
                  int n_dir, const double *xhat, igabem_request **out) {
  if (!S || !geom || !opt || !dirs || !xhat || !out || n_rhs <= 0 || n_dir <= 0)
    return refuse(IGABEM_EINVAL, "invalid submit arguments");
  auto *r = new igabem_request();
  r->srv = S;
  r->geom = geom;
  r->opt = *opt;
  r->R = n_rhs;
  r->n_dir = n_dir;
  r->dirs.assign(dirs, dirs + 3 * n_rhs);
  r->xhat.assign(xhat, xhat + 3 * n_dir);
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      return refuse(IGABEM_EINVAL, "server is shutting down");
    }
    if (S->submitted == 0) S->t_first = r->t_submit;
    S->submitted += 1;
    S->queue.push_back(r);
  }
  S->cv_queue.notify_one();
  *out = r;
  set_error("");
  return IGABEM_OK;
}

int igabem_poll(igabem_request *r, int *done) {
  if (!r || !done) return refuse(IGABEM_EINVAL, "invalid poll arguments");
  std::lock_guard<std::mutex> lk(r->mu);
  *done = r->done ? 1 : 0;
  return IGABEM_OK;
}

int igabem_wait(igabem_request *r, double timeout_s) {
  if (!r) return refuse(IGABEM_EINVAL, "invalid wait arguments");
  std::unique_lock<std::mutex> lk(r->mu);
  if (timeout_s < 0) {
    r->cv.wait(lk, [&] { return r->done; });
  } else if (!r->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; })) {
    return refuse(IGABEM_ETIMEOUT, "request still running after the timeout");
  }
  return IGABEM_OK;
}

int igabem_result(igabem_request *r, void *uinf, igabem_solve_info *info) {
  if (!r) return refuse(IGABEM_EINVAL, "invalid result arguments");
  std::lock_guard<std::mutex> lk(r->mu);
  if (!r->done) return refuse(IGABEM_ETIMEOUT, "request not finished");
  if (info) {
    *info = r->info;
    info->solve_ms = r->t_done - r->t_submit;
  }
  if (uinf && !r->uinf.empty()) std::memcpy(uinf, r->uinf.data(), r->uinf.size() * sizeof(double));
  if (r->status != IGABEM_OK) set_error(r->error);
  return r->status;
}

void igabem_request_destroy(igabem_request *r) {
  if (!r) return;
  igabem_wait(r, -1.0);
  delete r;
}

int igabem_server_get_stats(igabem_server *S, igabem_server_stats *out) {
  if (!S || !out) return refuse(IGABEM_EINVAL, "invalid stats arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->peak_bytes = S->peak_bytes;
  out->peak_active = S->peak_active;
  out->merged = S->merged;
  out->cache_hits = S->cache_hits;
  out->resident = (long)S->cache.size();
  out->budget_bytes = S->budget;
  std::vector<double> l = S->latency_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    double pos = q * (l.size() - 1);
    size_t i = (size_t)pos;
    double f = pos - i;
    return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
  };
  out->p50_ms = pct(0.5);
  out->p99_ms = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  out->mean_ms = l.empty() ? 0.0 : sum / l.size();
  double span = (S->t_last - S->t_first) / 1e3;
  out->solves_per_s = span > 0 ? S->completed / span : 0.0;
  return IGABEM_OK;
}

}  // extern "C"
