// Autotuner of the problem layout (igabem_autotune): the leaf size of the cluster tree (leaf_offset b:
// leaves of 2^b x 2^b elements) and whether the M2L coupling blocks are stored or generated on the
// fly are chosen by timing the candidates on the device for the caller's geometry, options and column
// count, scoring set-up time + (expected products per set-up) x product time; the choice is cached in
// memory and, optionally, in a text file keyed by the discretisation, wavenumber, precision, column
// count and a fingerprint of the geometry.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace igabem {

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // key -> (leaf_offset, m2l_stored)

std::string tune_key(const igabem_geom *g, const igabem_options &o, int R) {
  double fp = 0;  // fingerprint of the control nets
  long i = 0;
  for (const auto &P : g->patches)
    for (double v : P.hw) fp += v * (1.0 + 1e-3 * (double)(i++ % 97));
  std::ostringstream k;
  k.precision(10);
  k << g->patches.size() << ':' << fp << ":m" << o.level_m << ":p" << o.degree_p << ":bc" << o.bc << ":pr"
    << o.precision << ":q" << o.cheb_q << '-' << o.q_max << ":cap" << o.kappa_cap << ":adm" << o.eta_adm << ":k"
    << std::round(o.kappa * 100) / 100 << ":R" << R << ":pc" << o.precond;
  return k.str();
}

void load_file(const char *path) {
  if (!path) return;
  std::ifstream f(path);
  std::string key;
  int b, st;
  while (f >> key >> b >> st) g_tune_cache[key] = {b, st};
}

void append_file(const char *path, const std::string &key, int b, int st) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << ' ' << b << ' ' << st << '\n';
}

}  // namespace

}  // namespace igabem

using namespace igabem;

extern "C" int igabem_autotune(igabem_geom *geom, const igabem_options *opt, int n_rhs, int matvecs_per_setup,
                               const char *cache_path, igabem_options *out, igabem_tune_info *info) {
  return run_guarded([&] {
    if (!geom || !opt || !out || n_rhs <= 0) fail(IGABEM_EINVAL, "invalid autotune arguments");
    const int nmv = std::max(1, matvecs_per_setup);
    const std::string key = tune_key(geom, *opt, n_rhs);
    igabem_tune_info ti{};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      load_file(cache_path);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        *out = *opt;
        out->leaf_offset = it->second.first;
        out->m2l_stored = it->second.second;
        ti.leaf_offset = out->leaf_offset;
        ti.m2l_stored = out->m2l_stored;
        ti.from_cache = 1;
        if (info) *info = ti;
        return;
      }
    }
    IGA_CUDA(cudaSetDevice(geom->ctx->device));
    cudaStream_t st = geom->ctx->stream;
    size_t free_b = 0, total_b = 0;
    IGA_CUDA(cudaMemGetInfo(&free_b, &total_b));
    // the caller's vectors for the timed products (device memory, freed at the end)
    double *x = nullptr, *y = nullptr;
    cudaEvent_t a, b;
    IGA_CUDA(cudaEventCreate(&a));
    IGA_CUDA(cudaEventCreate(&b));
    double best = INFINITY;
    igabem_options best_o = *opt;
    const int bmax = std::min(opt->level_m, 3);
    try {
      for (int lb = std::min(1, bmax); lb <= bmax; ++lb)
        for (int stored = 0; stored <= 1; ++stored) {
          igabem_options o = *opt;
          o.leaf_offset = lb;
          o.m2l_stored = stored;
          o.profile = 0;
          igabem_problem *P = problem_plan(geom, &o);
          const size_t need = P->arena_bytes + P->temp_bytes + problem_work_bytes(P->S, n_rhs, 0, o.precision);
          if (need > 0.6 * free_b || (stored && P->S.n_far == 0)) {
            problem_release(P);
            continue;
          }
          try {
            problem_materialize(P, st);
          } catch (...) {
            problem_release(P);
            throw;
          }
          const double setup_ms = P->info.setup_ms;
          const size_t vb = (size_t)P->S.N * n_rhs * 2 * sizeof(double);
          if (!x) {
            IGA_CUDA(cudaMalloc(&x, vb));
            IGA_CUDA(cudaMalloc(&y, vb));
            IGA_CUDA(cudaMemsetAsync(x, 0, vb, st));
          }
          int rc = igabem_matvec(P, n_rhs, x, y);  // warm-up (work buffers, kernel attributes)
          float ms = 0.f;
          if (rc == IGABEM_OK) {
            IGA_CUDA(cudaEventRecord(a, st));
            for (int k = 0; k < 3 && rc == IGABEM_OK; ++k) rc = igabem_matvec(P, n_rhs, x, y);
            IGA_CUDA(cudaEventRecord(b, st));
            IGA_CUDA(cudaEventSynchronize(b));
            IGA_CUDA(cudaEventElapsedTime(&ms, a, b));
            ms /= 3;
          }
          problem_release(P);
          if (rc != IGABEM_OK) continue;
          const double score = setup_ms + nmv * (double)ms;
          ++ti.candidates;
          if (score < best) {
            best = score;
            best_o = o;
            ti.setup_ms = setup_ms;
            ti.matvec_ms = ms;
            ti.score_ms = score;
          }
        }
    } catch (...) {
      if (x) cudaFree(x);
      if (y) cudaFree(y);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      throw;
    }
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (ti.candidates == 0) fail(IGABEM_ENOMEM, "autotune: no candidate layout fits the device memory");
    *out = *opt;
    out->leaf_offset = best_o.leaf_offset;
    out->m2l_stored = best_o.m2l_stored;
    ti.leaf_offset = out->leaf_offset;
    ti.m2l_stored = out->m2l_stored;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = {out->leaf_offset, out->m2l_stored};
      append_file(cache_path, key, out->leaf_offset, out->m2l_stored);
    }
    if (info) *info = ti;
  });
}
