// Serving loop: scattering requests of different geometries, wavenumbers and right-hand-side counts
// are admitted by device memory and solved concurrently, each on its own CUDA stream, so the work of
// admitted requests overlaps on the device; a request that arrives while others run starts as soon
// as a slot and enough memory are free (continuous admission, not a queue drained one at a time).
//
// Every request is the whole path: host plan (cluster tree, lists), device set-up, right-hand sides,
// GMRES, far field at the requested directions.  The host plan gives the exact device bytes the
// request will hold, which the admission test compares with the budget.
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

struct igabem_server {
  igabem_ctx *ctx = nullptr;
  size_t budget = 0;
  int slots = 1;
  std::deque<igabem_request *> queue;
  std::mutex mu;
  std::condition_variable cv_queue, cv_mem;
  size_t in_use = 0, peak_bytes = 0;
  int active = 0, peak_active = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  // statistics
  long submitted = 0, completed = 0, failed = 0;
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

// One worker: takes the oldest waiting request, plans it on the host, waits until its device memory
// fits the budget, then runs it on the worker's own stream.
void worker_loop(igabem_server *S) {
  cudaSetDevice(S->ctx->device);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  for (;;) {
    igabem_request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_queue.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) break;
      r = S->queue.front();
      S->queue.pop_front();
    }
    igabem_problem *P = nullptr;
    int status = IGABEM_OK;
    std::string err;
    size_t need = 0;
    bool admitted = false;
    try {
      P = problem_plan(r->geom, &r->opt);
      need = P->arena_bytes + P->temp_bytes +
             problem_work_bytes(P->S, r->R, std::max(1, r->opt.gmres_restart), r->opt.precision) + (size_t(64) << 20);
      r->bytes = need;
      if (need > S->budget) {
        status = IGABEM_ENOMEM;
        err = "request needs " + std::to_string(need >> 20) + " MiB, more than the server's budget of " +
              std::to_string(S->budget >> 20) + " MiB";
      } else {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_mem.wait(lk, [&] { return S->in_use + need <= S->budget; });
        S->in_use += need;
        S->active += 1;
        S->peak_bytes = std::max(S->peak_bytes, S->in_use);
        S->peak_active = std::max(S->peak_active, S->active);
        admitted = true;
      }
      if (admitted) {
        r->t_start = now_ms();
        problem_materialize(P, st);
        std::vector<double> dens(2 * (size_t)P->S.N * r->R);
        int rc = igabem_solve(P, r->R, r->dirs.data(), dens.data(), &r->info);
        if (rc != IGABEM_OK && rc != IGABEM_ENOT_CONVERGED) {
          status = rc;
          err = igabem_last_error();
        } else {
          if (rc == IGABEM_ENOT_CONVERGED) {
            status = rc;
            err = igabem_last_error();
          }
          r->uinf.assign(2 * (size_t)r->n_dir * r->R, 0.0);
          int rf = igabem_farfield(P, r->R, dens.data(), r->n_dir, r->xhat.data(), r->uinf.data());
          if (rf != IGABEM_OK) {
            status = rf;
            err = igabem_last_error();
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
    if (P) problem_release(P);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (admitted) {
        S->in_use -= need;
        S->active -= 1;
      }
      S->completed += status == IGABEM_OK ? 1 : 0;
      S->failed += status == IGABEM_OK ? 0 : 1;
      double t = now_ms();
      if (status == IGABEM_OK) S->latency_ms.push_back(t - r->t_submit);
      S->t_last = t;
    }
    S->cv_mem.notify_all();
    finish(r, status, err);
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
