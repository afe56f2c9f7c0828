// Per-problem profiling: kernel launch counters and per-phase device time from CUDA events.
#include "internal.h"

namespace igabem {

namespace {
thread_local Profiler *t_prof = nullptr;
thread_local int t_phase = -1;
}  // namespace

cudaEvent_t Profiler::event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  IGA_CUDA(cudaEventCreate(&e));
  return e;
}

void Profiler::flush() {
  for (auto &pe : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) {
      ms[pe.first] += t;
      calls[pe.first] += 1;
    } else {
      cudaGetLastError();
    }
    pool.push_back(pe.second.first);
    pool.push_back(pe.second.second);
  }
  pending.clear();
}

void Profiler::reset() {
  launches = 0;
  for (int i = 0; i < IGABEM_NPHASE; ++i) {
    phase_launches[i] = 0;
    ms[i] = 0;
    calls[i] = 0;
  }
}

Profiler::~Profiler() {
  for (auto &pe : pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

Phase::Phase(Profiler *p, int phase, cudaStream_t st) : p_(p), ph_(phase), st_(st) {
  prev_p_ = t_prof;
  prev_ph_ = t_phase;
  t_prof = p;
  t_phase = phase;
  if (p_ && p_->on) {
    a_ = p_->event();
    IGA_CUDA(cudaEventRecord(a_, st_));
  }
}

Phase::~Phase() {
  if (p_ && p_->on && a_) {
    cudaEvent_t b = nullptr;
    try {
      b = p_->event();
    } catch (...) {
      b = nullptr;
    }
    if (b && cudaEventRecord(b, st_) == cudaSuccess) {
      p_->pending.push_back({ph_, {a_, b}});
    } else {
      cudaGetLastError();
      p_->pool.push_back(a_);
      if (b) p_->pool.push_back(b);
    }
  }
  t_prof = prev_p_;
  t_phase = prev_ph_;
}

int max_optin_smem() {
  static int v = -1;
  if (v < 0) {
    int dev = 0, x = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
      v = x;
    else
      v = 48 * 1024;
  }
  return v;
}

void note_launch() {
  if (t_prof) {
    t_prof->launches++;
    if (t_phase >= 0) t_prof->phase_launches[t_phase]++;
  }
}

}  // namespace igabem
