// C ABI of the library (include/igabem.h): handles, memory placement, problem set-up and the GMRES
// driver.  The kernels live in k_*.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace igabem {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {
thread_local std::string g_error;

struct Failure {
  int code;
};

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class F> int guarded(F &&f) {
  try {
    g_error.clear();
    f();
    return IGABEM_OK;
  } catch (const Failure &e) {
    return e.code;
  } catch (const std::bad_alloc &) {
    g_error = "host memory exhausted";
    return IGABEM_ENOMEM;
  } catch (const std::exception &e) {
    g_error = e.what();
    return IGABEM_EINVAL;
  }
}
}  // namespace

void set_error(const std::string &msg) { g_error = msg; }

int run_guarded(const std::function<void()> &f) { return guarded(f); }

void fail(int code, const std::string &msg) {
  g_error = msg;
  throw Failure{code};
}

void Arena::reserve(size_t bytes) {
  release();
  cap = bytes;
  off = 0;
  if (bytes == 0) return;
  cudaError_t e = cudaMalloc(&base, bytes);
  if (e != cudaSuccess) {
    base = nullptr;
    cap = 0;
    cudaGetLastError();
    fail(IGABEM_ENOMEM, "device allocation of " + std::to_string(bytes >> 20) + " MiB failed: " +
                            cudaGetErrorString(e));
  }
}

void *Arena::take(size_t bytes) {
  size_t a = (bytes + 255) & ~size_t(255);
  if (off + a > cap) fail(IGABEM_ENOMEM, "arena exhausted (internal sizing error)");
  void *p = base + off;
  off += a;
  return p;
}

void Arena::release() {
  if (base) cudaFree(base);
  base = nullptr;
  cap = off = 0;
}

// device bytes of the per-call work buffers for R columns (and a GMRES basis of gmres_m + 1 vectors)
size_t problem_work_bytes(const HostSetup &S, int R, int gmres_m, int precision) {
  const int C = S.hard ? 7 : 1, nq = S.ng * S.ng;
  const size_t cz = 2 * sizeof(double);
  const long nleaf = S.lev[S.L].n;
  size_t total = 0;
  auto add = [&](size_t n) { total += (n + 255) & ~size_t(255); };
  add(S.NX * R * cz);
  add(nleaf * S.nL * R * cz);
  add((size_t)S.E * nq * C * R * cz);
  add(S.N * R * cz);
  add(S.N * R * cz);
  add((size_t)std::max(34, gmres_m + 2) * 304 * R * cz + 4096);
  for (int l = S.lmin; l <= S.L; ++l) {
    const size_t Q = (size_t)S.lev[l].q * S.lev[l].q;
    add((size_t)S.lev[l].n * Q * C * R * cz);
    add((size_t)S.lev[l].n * Q * C * R * cz);
  }
  if (precision != IGABEM_FP64) {  // FP32 copies of the input vector and of the expansions
    add(S.NX * R * sizeof(float2));
    for (int l = S.lmin; l <= S.L; ++l) add((size_t)S.lev[l].n * S.lev[l].q * S.lev[l].q * C * R * sizeof(float2));
    add((size_t)S.lev[S.L].n * S.q * S.q * C * R * sizeof(float2));
  }
  if (precision == IGABEM_MIXED_TC && S.n_far > 0 && m2l_tc_supported(S, R))
    for (int l = S.lmin; l <= S.L; ++l) {
      add(m2l_tc_image_bytes(S, l, R));
      add((size_t)S.lev[l].n * sizeof(float));
    }
  if (gmres_m) {
    const size_t m = gmres_m;
    add((m + 1) * S.N * R * cz);
    for (int k = 0; k < 7; ++k) add(S.N * R * cz);
    add((m + 1) * m * R * cz);                            // H
    for (int k = 0; k < 2; ++k) add(m * R * cz);          // cs, sn
    for (int k = 0; k < 4; ++k) add((m + 1) * R * cz);    // g, y, hA, hB
    for (int k = 0; k < 4; ++k) add(R * sizeof(double));  // nrm, s, bn, beta
    for (int k = 0; k < 4; ++k) add(R * sizeof(int));     // k, its, done, active
    add(16);                                              // j, flags
  }
  return total;
}

}  // namespace igabem

using namespace igabem;

// one GMRES iteration (Sec. 5.1) captured as a CUDA graph for a problem's work buffers
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  int R = 0, precond = -1;
  const void *base = nullptr;        // the work arena the graph's pointers belong to
  long launches = 0;                 // kernels per replay (for the launch counters)
  long phase_launches[IGABEM_NPHASE] = {};
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    base = nullptr;
  }
};

struct ProblemWork {
  int R = 0;
  int gmres_m = 0;
  Arena arena;
  double *xX, *yleaf, *gq, *xin, *yout, *red;
  std::vector<void *> xhat, yhat;
  std::vector<uint8_t *> tc_bimg;
  std::vector<float *> tc_bscale;
  std::vector<float2 *> xhat32;      // mixed precisions: FP32 copies of the expansions, the input vector
  float2 *xX32 = nullptr, *y32 = nullptr;  // and the leaf-level local expansions
  // GMRES
  double *V, *w, *x, *b, *r, *t, *u, *vj;
  GmDev G{};
  double *beta = nullptr;
  int *active = nullptr;
  int *hflags = nullptr;             // page-locked copy of G.flags, written by every iteration
  IterGraph graph;
  ~ProblemWork() {
    graph.release();
    if (hflags) cudaFreeHost(hflags);
  }
};

namespace {

struct ProblemExt {
  ProblemWork work;
};

ProblemExt *ext(igabem_problem *p);

}  // namespace

// The problem object carries its work buffers in a side table keyed by the handle.
#include <map>
#include <mutex>
static std::map<const igabem_problem *, ProblemExt *> g_ext;
static std::mutex g_ext_mu;

namespace {
ProblemExt *ext(igabem_problem *p) {
  std::lock_guard<std::mutex> lk(g_ext_mu);
  auto it = g_ext.find(p);
  if (it == g_ext.end()) it = g_ext.emplace(p, new ProblemExt()).first;
  return it->second;
}

void ensure_work(igabem_problem *P, int R, bool with_gmres) {
  ProblemWork &W = ext(P)->work;
  const HostSetup &S = P->S;
  int m = std::max(1, P->opt.gmres_restart);
  if (W.R >= R && (!with_gmres || W.gmres_m >= m)) return;
  R = std::max(R, W.R);
  if (with_gmres) W.gmres_m = std::max(W.gmres_m, m);
  const int C = S.hard ? 7 : 1, nq = S.ng * S.ng;
  const long nleaf = S.lev[S.L].n;
  size_t total = problem_work_bytes(S, R, W.gmres_m, P->opt.precision);
  W.arena.reserve(total);
  W.R = R;
  W.xX = W.arena.get<double>(S.NX * R * 2);
  W.yleaf = W.arena.get<double>(nleaf * S.nL * R * 2);
  W.gq = W.arena.get<double>((size_t)S.E * nq * C * R * 2);
  W.xin = W.arena.get<double>(S.N * R * 2);
  W.yout = W.arena.get<double>(S.N * R * 2);
  W.red = W.arena.get<double>((size_t)34 * 304 * R * 2 + 512);
  W.xhat.assign(S.L + 1, nullptr);
  W.yhat.assign(S.L + 1, nullptr);
  for (int l = S.lmin; l <= S.L; ++l) {
    const size_t Q = (size_t)S.lev[l].q * S.lev[l].q;
    W.xhat[l] = W.arena.get<double>((size_t)S.lev[l].n * Q * C * R * 2);
    W.yhat[l] = W.arena.get<double>((size_t)S.lev[l].n * Q * C * R * 2);
  }
  W.xhat32.assign(S.L + 1, nullptr);
  W.xX32 = W.y32 = nullptr;
  if (P->opt.precision != IGABEM_FP64) {
    W.xX32 = W.arena.get<float2>(S.NX * R);
    for (int l = S.lmin; l <= S.L; ++l)
      W.xhat32[l] = W.arena.get<float2>((size_t)S.lev[l].n * S.lev[l].q * S.lev[l].q * C * R);
    W.y32 = W.arena.get<float2>((size_t)S.lev[S.L].n * S.q * S.q * C * R);
  }
  W.tc_bimg.assign(S.L + 1, nullptr);
  W.tc_bscale.assign(S.L + 1, nullptr);
  if (P->opt.precision == IGABEM_MIXED_TC && S.n_far > 0 && m2l_tc_supported(S, R))
    for (int l = S.lmin; l <= S.L; ++l) {
      W.tc_bimg[l] = W.arena.get<uint8_t>(m2l_tc_image_bytes(S, l, R));
      W.tc_bscale[l] = W.arena.get<float>(S.lev[l].n);
    }
  W.graph.release();  // its pointers belong to the previous arena
  if (W.gmres_m) {
    const size_t m = W.gmres_m;
    W.V = W.arena.get<double>((m + 1) * S.N * R * 2);
    W.w = W.arena.get<double>(S.N * R * 2);
    W.x = W.arena.get<double>(S.N * R * 2);
    W.b = W.arena.get<double>(S.N * R * 2);
    W.r = W.arena.get<double>(S.N * R * 2);
    W.t = W.arena.get<double>(S.N * R * 2);
    W.u = W.arena.get<double>(S.N * R * 2);
    W.vj = W.arena.get<double>(S.N * R * 2);
    GmDev &G = W.G;
    G.m = (int)m;
    G.R = R;
    G.H = W.arena.get<double2>((m + 1) * m * R);
    G.cs = W.arena.get<double2>(m * R);
    G.sn = W.arena.get<double2>(m * R);
    G.g = W.arena.get<double2>((m + 1) * R);
    G.y = W.arena.get<double2>((m + 1) * R);
    G.hA = W.arena.get<double2>((m + 1) * R);
    G.hB = W.arena.get<double2>((m + 1) * R);
    G.nrm = W.arena.get<double>(R);
    G.s = W.arena.get<double>(R);
    G.bn = W.arena.get<double>(R);
    W.beta = W.arena.get<double>(R);
    G.k = W.arena.get<int>(R);
    G.its = W.arena.get<int>(R);
    G.done = W.arena.get<int>(R);
    W.active = W.arena.get<int>(R);
    G.j = W.arena.get<int>(4);
    G.flags = G.j + 2;
    G.V = W.V;
    G.w = W.w;
    if (!W.hflags) IGA_CUDA(cudaMallocHost(&W.hflags, 2 * sizeof(int)));
  }
  DeviceProblem &d = P->d;
  d.max_rhs = R;
  d.xX = W.xX;
  d.yleaf = W.yleaf;
  d.gq = W.gq;
  d.xin = W.xin;
  d.yout = W.yout;
  d.red = W.red;
  d.xhat = W.xhat;
  d.yhat = W.yhat;
  d.tc_bimg = W.tc_bimg;
  d.tc_bscale = W.tc_bscale;
  d.xhat32 = W.xhat32;
  d.xX32 = W.xX32;
  d.y32 = W.y32;
}

// the device status word: a kernel whose bounded wait ran out has set it (the stream is synchronised)
void check_status(igabem_problem *P) {
  int v = 0;
  IGA_CUDA(cudaMemcpy(&v, P->d.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    IGA_CUDA(cudaMemset(P->d.status, 0, sizeof(int)));
    fail(IGABEM_ETIMEOUT, "a tensor-core M2L wait timed out; the result is incomplete");
  }
}

template <class T> T *upload(Arena &A, const std::vector<T> &v, cudaStream_t st) {
  T *p = A.get<T>(std::max<size_t>(v.size(), 1));
  if (!v.empty()) IGA_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

template <class T> size_t bytes_of(const std::vector<T> &v) {
  return ((std::max<size_t>(v.size(), 1) * sizeof(T)) + 255) & ~size_t(255);
}

void matvec_dev(igabem_problem *P, int R, const double *x, double *y) {
  launch_matvec(P->d, P->S, P->opt, R, x, y, P->stream);
}

// Complex Givens rotation [[c, s], [-conj(s), conj(c)]], c = conj(a)/den, s = conj(b)/den.
struct Col {
  std::vector<std::complex<double>> H, cs, sn, g;
  int k = 0;
  bool done = false;
};

}  // namespace

namespace igabem {

// host-side plan of a problem: validation, set-up tables and the device memory it will hold
igabem_problem *problem_plan(igabem_geom *geom, const igabem_options *opt) {
  if (!geom || !opt) fail(IGABEM_EINVAL, "invalid problem arguments");
  if (opt->precision != IGABEM_FP64 && opt->precision != IGABEM_MIXED_FP32 && opt->precision != IGABEM_MIXED_TC)
    fail(IGABEM_EINVAL, "unknown precision");
  if (!(opt->eta_adm > 0)) fail(IGABEM_EINVAL, "eta_adm must be positive");
  if (!(opt->kappa >= 0)) fail(IGABEM_EINVAL, "kappa must be >= 0");
  auto *P = new igabem_problem();
  P->geom = geom;
  P->opt = *opt;
  P->stream = geom->ctx->stream;
  P->prof.on = opt->profile != 0;
  P->t_plan = now_ms();
  try {
    HostSetup &S = P->S;
    std::shared_ptr<const GeoCache> hit;
    {
      std::lock_guard<std::mutex> lk(geom->cache_mu);
      if (geom->cache && geom->cache->m == opt->level_m) hit = geom->cache;
    }
    auto fill = std::make_shared<GeoCache>();
    build_setup(geom->patches, *opt, S, hit.get(), fill.get());
    if (fill->m >= 0) {
      std::lock_guard<std::mutex> lk(geom->cache_mu);
      geom->cache = fill;
    }
    P->info.host_setup_ms = now_ms() - P->t_plan;
    const int nq = S.ng * S.ng;
    size_t total = 0;
    std::vector<int> dummy_tgt(S.near_src.size());
    size_t nrule = S.r_id.w.size() + S.r_edge.w.size() + S.r_vert.w.size();
    total += bytes_of(S.edeg) + bytes_of(S.eoff) + bytes_of(S.ebez) + bytes_of(S.corners);
    size_t gst = (size_t)S.E * nq;
    total += 13 * ((gst * sizeof(double) + 255) & ~size_t(255));
    total += bytes_of(S.phi1) + bytes_of(S.dphi1) + bytes_of(S.ext1) + bytes_of(S.gx) + bytes_of(S.gw);
    total += bytes_of(std::vector<float>(S.phi1.size())) + bytes_of(std::vector<float>((size_t)nq));
    total += 3 * 256 + 5 * nrule * sizeof(double);
    for (const Rule4 *r : {&S.r_id, &S.r_edge, &S.r_vert}) total += (r->share.size() + 255) & ~size_t(255);
    total += bytes_of(S.touch) + bytes_of(S.touch_blk) + bytes_of(S.sing) + bytes_of(S.x2g) + bytes_of(S.g2x_ptr) +
             bytes_of(S.g2x_idx);
    total += bytes_of(S.near_ptr) + bytes_of(S.near_src) + bytes_of(dummy_tgt);
    total += bytes_of(S.T1) + bytes_of(S.LG1);
    for (int l = 0; l <= S.L; ++l) {
      const size_t Q = (size_t)S.lev[l].q * S.lev[l].q;
      total += bytes_of(S.lev[l].cheb) + bytes_of(S.lev[l].T1) + bytes_of(S.lev[l].LG);
      total += bytes_of(S.lev[l].far_ptr) + bytes_of(S.lev[l].far_src);
      total += ((size_t)7 * S.lev[l].n * Q * sizeof(double) + 255) & ~size_t(255);
      total += ((size_t)7 * S.lev[l].n * Q * sizeof(float) + 255) & ~size_t(255);
      total += bytes_of(S.lev[l].center);
      total += ((std::max<size_t>(S.lev[l].far_src.size(), 1) * 8 * sizeof(float)) + 255) & ~size_t(255);
      total += ((size_t)S.lev[l].n * 2 * sizeof(double) + 255) & ~size_t(255);
    }
    const bool mixed = opt->precision != IGABEM_FP64;
    size_t blk_entries = S.near_src.size() * (size_t)S.nL * S.nL * 2;
    size_t blk_bytes = blk_entries * sizeof(double);
    // mixed precision keeps the near-field blocks in FP32; the FP64 assembly buffer is temporary
    total += mixed ? ((blk_entries * sizeof(float) + 255) & ~size_t(255)) : ((blk_bytes + 255) & ~size_t(255));
    if (opt->precond) {
      if (opt->precond != 1) fail(IGABEM_EINVAL, "unknown preconditioner");
      if (S.nL > 64) fail(IGABEM_EINVAL, "the block preconditioner needs leaves with at most 64 local functions");
      const size_t nleaf = S.lev[S.L].n;
      total += ((nleaf * S.nL * S.nL * 2 * sizeof(double)) + 255) & ~size_t(255);
      total += 3 * (((nleaf + 1) * sizeof(int) + 255) & ~size_t(255));
    }
    total += 256;  // status word
    total += bytes_of(S.nbr);
    if (opt->m2l_stored && S.n_far > 0)
      for (int l = S.lmin; l <= S.L; ++l)
        total += (m2l_stored_entries(S, l) * (mixed ? sizeof(float2) : sizeof(double2)) + 255) & ~size_t(255);
    if (S.n_far > 0 && leaf_moments_supported(S))
      total += ((leaf_moment_entries(S) * (mixed ? sizeof(float) : sizeof(double))) + 255) & ~size_t(255);
    P->arena_bytes = total + 4096;
    P->temp_bytes = (mixed ? blk_bytes : 0) + near_table_bytes(S, *opt);
  } catch (...) {
    delete P;
    throw;
  }
  return P;
}

// device set-up of a planned problem on stream st: tables, near-field quadrature
void problem_materialize(igabem_problem *P, cudaStream_t st) {
  const igabem_options *opt = &P->opt;
  P->stream = st;
  HostSetup &S = P->S;
  IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
  const int nq = S.ng * S.ng;
  const long nleaf = S.lev[S.L].n;
  std::vector<int> near_tgt(S.near_src.size());
  for (long t = 0; t < nleaf; ++t)
    for (int k = S.near_ptr[t]; k < S.near_ptr[t + 1]; ++k) near_tgt[k] = (int)t;
  std::vector<double> rules[3];
  const Rule4 *R4[3] = {&S.r_id, &S.r_edge, &S.r_vert};
  for (int k = 0; k < 3; ++k) {
    const Rule4 &r = *R4[k];
    for (const auto *v : {&r.x1, &r.x2, &r.y1, &r.y2, &r.w}) rules[k].insert(rules[k].end(), v->begin(), v->end());
  }
  const size_t gst = (size_t)S.E * nq;
  const bool mixed = opt->precision != IGABEM_FP64;
  const size_t blk_entries = S.near_src.size() * (size_t)S.nL * S.nL * 2;
  const size_t blk_bytes = blk_entries * sizeof(double);
  P->arena.reserve(P->arena_bytes);
  Arena &A = P->arena;
  DeviceProblem &d = P->d;
  d.prof = &P->prof;
  d.status = A.get<int>(1);
  IGA_CUDA(cudaMemsetAsync(d.status, 0, sizeof(int), st));
  d.edeg = upload(A, S.edeg, st);
  d.eoff = upload(A, S.eoff, st);
  d.ebez = upload(A, S.ebez, st);
  d.corners = upload(A, S.corners, st);
  d.gpx = A.get<double>(3 * gst);
  d.gpn = A.get<double>(3 * gst);
  d.gpa = A.get<double>(gst);
  d.gfs = A.get<double>(3 * gst);
  d.gft = A.get<double>(3 * gst);
  d.phi1 = upload(A, S.phi1, st);
  d.dphi1 = upload(A, S.dphi1, st);
  d.ext1 = upload(A, S.ext1, st);
  d.gx = upload(A, S.gx, st);
  d.gw = upload(A, S.gw, st);
  {
    const std::vector<float> phi1f(S.phi1.begin(), S.phi1.end());
    std::vector<float> gwq((size_t)nq);
    for (int q = 0; q < nq; ++q) gwq[q] = (float)(S.gw[q / S.ng] * S.gw[q % S.ng] * S.h * S.h);
    d.phi1f = upload(A, phi1f, st);
    d.gwqf = upload(A, gwq, st);
    IGA_CUDA(cudaStreamSynchronize(st));  // the host vectors above go out of scope
  }
  for (int k = 0; k < 3; ++k) {
    d.rule[k] = upload(A, rules[k], st);
    d.rule_n[k] = (int)R4[k]->w.size();
    d.share[k] = upload(A, R4[k]->share, st);
  }
  d.touch = upload(A, S.touch, st);
  d.touch_blk = upload(A, S.touch_blk, st);
  d.sing = upload(A, S.sing, st);
  d.nbr = upload(A, S.nbr, st);
  d.x2g = upload(A, S.x2g, st);
  d.g2x_ptr = upload(A, S.g2x_ptr, st);
  d.g2x_idx = upload(A, S.g2x_idx, st);
  d.near_ptr = upload(A, S.near_ptr, st);
  d.near_src = upload(A, S.near_src, st);
  d.near_tgt = upload(A, near_tgt, st);
  d.T1 = upload(A, S.T1, st);
  d.LG1 = upload(A, S.LG1, st);
  d.far_ptr.assign(S.L + 1, nullptr);
  d.far_src.assign(S.L + 1, nullptr);
  d.nodes.assign(S.L + 1, nullptr);
  d.nodes32.assign(S.L + 1, nullptr);
  d.centers.assign(S.L + 1, nullptr);
  d.pairc.assign(S.L + 1, nullptr);
  d.cext.assign(S.L + 1, nullptr);
  d.chebl.assign(S.L + 1, nullptr);
  d.T1l.assign(S.L + 1, nullptr);
  d.LGl.assign(S.L + 1, nullptr);
  for (int l = 0; l <= S.L; ++l) {
    const size_t Q = (size_t)S.lev[l].q * S.lev[l].q;
    d.chebl[l] = upload(A, S.lev[l].cheb, st);
    d.T1l[l] = upload(A, S.lev[l].T1, st);
    d.LGl[l] = upload(A, S.lev[l].LG, st);
    d.far_ptr[l] = upload(A, S.lev[l].far_ptr, st);
    d.far_src[l] = upload(A, S.lev[l].far_src, st);
    d.nodes[l] = A.get<double>((size_t)7 * S.lev[l].n * Q);
    d.nodes32[l] = A.get<float>((size_t)7 * S.lev[l].n * Q);
    d.centers[l] = upload(A, S.lev[l].center, st);
    d.pairc[l] = A.get<float>(std::max<size_t>(S.lev[l].far_src.size(), 1) * 8);
    d.cext[l] = A.get<double>((size_t)S.lev[l].n * 2);
  }
  double *blk_tmp = nullptr;
  if (mixed) {
    d.blk32 = A.get<float>(blk_entries);
    IGA_CUDA(cudaMalloc(&blk_tmp, std::max<size_t>(blk_bytes, 256)));
    d.blk = blk_tmp;
  } else {
    d.blk = A.get<double>(blk_entries);
  }
  IGA_CUDA(cudaMemsetAsync(d.blk, 0, blk_bytes, st));
  IGA_CUDA(cudaMalloc(&d.near_tab, std::max<size_t>(near_table_bytes(S, *opt), 256)));
  launch_gauss_geometry(d, S, st);
  launch_node_geometry(d, S, st);
  if (S.n_far > 0 && leaf_moments_supported(S)) {
    if (mixed)
      d.lm32 = A.get<float>(leaf_moment_entries(S));
    else
      d.lm64 = A.get<double>(leaf_moment_entries(S));
    Phase ph(&P->prof, IGABEM_PH_SETUP_TABLES, st);
    launch_leaf_moments(d, S, *opt, st);
  }
  if (S.n_far > 0) {
    Phase ph(&P->prof, IGABEM_PH_SETUP_TABLES, st);
    launch_pair_consts(d, S, opt->kappa, opt->eta_cfie, st);
  }
  d.m2ls.assign(S.L + 1, nullptr);
  if (opt->m2l_stored && S.n_far > 0) {
    for (int l = S.lmin; l <= S.L; ++l)
      d.m2ls[l] = A.get<double>(m2l_stored_entries(S, l) * (mixed ? 1 : 2));
    Phase ph(&P->prof, IGABEM_PH_SETUP_TABLES, st);
    launch_m2l_fill(d, S, *opt, st);
  }
  launch_near_field(d, S, *opt, st);
  if (opt->precond) {
    std::vector<int> ip(nleaf + 1), is(nleaf);
    for (long t = 0; t <= nleaf; ++t) ip[t] = (int)t;
    for (long t = 0; t < nleaf; ++t) is[t] = (int)t;
    d.diag_blk = upload(A, S.diag_blk, st);
    d.ident_ptr = upload(A, ip, st);
    d.ident_src = upload(A, is, st);
    d.binv = A.get<double>((size_t)nleaf * S.nL * S.nL * 2);
    Phase ph(&P->prof, IGABEM_PH_SETUP_NEAR, st);
    launch_block_inverse(d, S, st);
  }
  if (mixed) {
    {
      Phase ph(&P->prof, IGABEM_PH_SETUP_NEAR, st);
      launch_blocks_to_fp32(d.blk, d.blk32, blk_entries, st);
    }
    IGA_CUDA(cudaStreamSynchronize(st));
    IGA_CUDA(cudaFree(blk_tmp));
    d.blk = nullptr;
  }
  IGA_CUDA(cudaStreamSynchronize(st));
  IGA_CUDA(cudaFree(d.near_tab));
  d.near_tab = nullptr;
  IGA_CUDA(cudaGetLastError());
  P->prof.flush();
  igabem_info &I = P->info;
  I.n_dofs = S.N;
  I.n_patch_dofs = S.NX;
  I.n_elements = S.E;
  long ncl = 0;
  for (auto &lv : S.lev) ncl += lv.n;
  I.n_clusters = ncl;
  I.n_near_pairs = (long)S.near_src.size();
  I.n_near_element_pairs = I.n_near_pairs << (4 * S.b);
  I.n_touching_pairs = (long)S.touch.size() / 5;
  I.n_far_pairs = S.n_far;
  I.n_singular_points = 0;
  I.n_singular_geo_points = 0;
  I.n_singular_geo_columns = 0;
  I.n_singular_groups = 0;
  I.n_singular_factored_points = 0;
  // per rule, summed over the chunks a pair integrates: distinct x1, x2, x-points, y1, y2, y-points,
  // and the groups of the side with fewer distinct points
  long chunk_sum[3][7] = {};
  for (int k = 0; k < 3; ++k) {
    const int n = (int)R4[k]->w.size(), nuse = k == 0 ? n / 2 : n, ch = S.sing_ch;
    for (int c0 = 0; c0 < nuse; c0 += ch) {
      const unsigned char *H = R4[k]->share.data() + (size_t)(c0 / ch) * sing_share_header(ch);
      for (int j = 0; j < 6; ++j) chunk_sum[k][j] += H[j];
      chunk_sum[k][6] += std::min(H[2], H[5]);
    }
  }
  for (size_t i = 0; i + 6 < S.sing.size(); i += 7) {
    const int kind = S.sing[i + 2], te = S.sing[i + 3], tf = S.sing[i + 4];
    const int r = kind == 0 ? 0 : (kind == 2 ? 1 : 2);
    I.n_singular_points += r == 0 ? (long)S.r_id.w.size() / 2 : (long)R4[r]->w.size();
    // the rule coordinate that becomes the second local coordinate (as in k_near_singular)
    const int vse = ((te & 1) != (te >= 4)) ? 0 : 1, vsf = ((tf & 1) != (tf >= 4)) ? 0 : 1;
    I.n_singular_geo_points += chunk_sum[r][2] + chunk_sum[r][5];
    I.n_singular_geo_columns += chunk_sum[r][vse] + chunk_sum[r][3 + vsf];
    if (r == 0 && S.sing_fact) I.n_singular_factored_points += (long)S.r_id.w.size() / 2;
    else I.n_singular_groups += chunk_sum[r][6];
  }
  I.n_levels = S.L + 1;
  for (int l = 0; l <= S.L && l < 24; ++l) {
    I.level_q[l] = S.lev[l].q;
    I.level_far[l] = (long)S.lev[l].far_src.size();
  }
  I.device_bytes = A.cap;
  I.setup_ms = now_ms() - P->t_plan;
}

void problem_release(igabem_problem *P) {
  {
    std::lock_guard<std::mutex> lk(g_ext_mu);
    auto it = g_ext.find(P);
    if (it != g_ext.end()) {
      it->second->work.arena.release();
      delete it->second;
      g_ext.erase(it);
    }
  }
  P->arena.release();
  delete P;
}

}  // namespace igabem

extern "C" {

const char *igabem_last_error(void) { return g_error.c_str(); }

void igabem_default_options(igabem_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->degree_p = 2;
  o->level_m = 3;
  o->kappa = 1.0;
  o->eta_cfie = 1.0;
  o->bc = IGABEM_SOUND_SOFT;
  o->cheb_q = 7;
  o->leaf_offset = 0;
  o->eta_adm = 0.5;
  o->kappa_cap = 0.0;
  o->gauss_regular = 4;
  o->gauss_singular = 5;
  o->precision = IGABEM_FP64;
  o->gmres_restart = 30;
  o->max_iter = 1000;
  o->tol = 1e-6;
  o->no_fmm = 0;
  o->profile = 0;
  o->precond = 0;
}

int igabem_create(igabem_ctx **out, int device, void *stream) {
  return guarded([&] {
    if (!out) fail(IGABEM_EINVAL, "out is NULL");
    int n = 0;
    IGA_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) fail(IGABEM_EINVAL, "no such CUDA device");
    IGA_CUDA(cudaSetDevice(device));
    auto *c = new igabem_ctx();
    c->device = device;
    if (stream) {
      c->stream = static_cast<cudaStream_t>(stream);
    } else {
      IGA_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    *out = c;
  });
}

void igabem_destroy(igabem_ctx *ctx) {
  if (!ctx) return;
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int igabem_geometry_create(igabem_ctx *ctx, int n_patches, const int *degrees, const int *counts,
                           const double *knots, const double *ctrl, const double *weights,
                           igabem_geom **out) {
  return guarded([&] {
    if (!ctx || !out || !degrees || !counts || !knots || !ctrl || !weights || n_patches <= 0)
      fail(IGABEM_EINVAL, "invalid geometry arguments");
    auto *g = new igabem_geom();
    g->ctx = ctx;
    long ko = 0, co = 0;
    for (int j = 0; j < n_patches; ++j) {
      Patch P;
      P.p1 = degrees[2 * j]; P.p2 = degrees[2 * j + 1];
      P.k1 = counts[2 * j]; P.k2 = counts[2 * j + 1];
      if (P.p1 < 1 || P.p1 > 6 || P.p2 < 1 || P.p2 > 6 || P.k1 <= P.p1 || P.k2 <= P.p2) {
        delete g;
        fail(IGABEM_EINVAL, "patch " + std::to_string(j) + ": degrees must lie in 1..6, counts > degrees");
      }
      P.kn1.assign(knots + ko, knots + ko + P.k1 + P.p1 + 1);
      ko += P.k1 + P.p1 + 1;
      P.kn2.assign(knots + ko, knots + ko + P.k2 + P.p2 + 1);
      ko += P.k2 + P.p2 + 1;
      for (const auto *kn : {&P.kn1, &P.kn2}) {
        int p = kn == &P.kn1 ? P.p1 : P.p2;
        bool ok = true;
        for (size_t i = 1; i < kn->size(); ++i) ok = ok && (*kn)[i] >= (*kn)[i - 1];
        for (int i = 0; i <= p; ++i) ok = ok && (*kn)[i] == 0.0 && (*kn)[kn->size() - 1 - i] == 1.0;
        if (!ok) {
          delete g;
          fail(IGABEM_EINVAL, "patch " + std::to_string(j) + ": knots must be p-open on [0,1] and sorted");
        }
      }
      P.hw.resize(4L * P.k1 * P.k2);
      for (long i = 0; i < (long)P.k1 * P.k2; ++i) {
        double w = weights[co + i];
        if (!(w > 0)) {
          delete g;
          fail(IGABEM_EINVAL, "weights must be positive");
        }
        for (int c = 0; c < 3; ++c) P.hw[4 * i + c] = w * ctrl[3 * (co + i) + c];
        P.hw[4 * i + 3] = w;
      }
      co += (long)P.k1 * P.k2;
      g->patches.push_back(std::move(P));
    }
    *out = g;
  });
}

void igabem_geometry_destroy(igabem_geom *geom) { delete geom; }

int igabem_problem_create(igabem_geom *geom, const igabem_options *opt, igabem_problem **out) {
  return guarded([&] {
    if (!geom || !opt || !out) fail(IGABEM_EINVAL, "invalid problem arguments");
    IGA_CUDA(cudaSetDevice(geom->ctx->device));
    igabem_problem *P = problem_plan(geom, opt);
    try {
      problem_materialize(P, geom->ctx->stream);
    } catch (...) {
      problem_release(P);
      throw;
    }
    *out = P;
  });
}

int igabem_problem_info(const igabem_problem *prob, igabem_info *out) {
  return guarded([&] {
    if (!prob || !out) fail(IGABEM_EINVAL, "NULL argument");
    *out = prob->info;
    std::lock_guard<std::mutex> lk(g_ext_mu);
    auto it = g_ext.find(prob);
    if (it != g_ext.end()) out->device_bytes += it->second->work.arena.cap;
  });
}

void igabem_problem_destroy(igabem_problem *prob) {
  if (prob) problem_release(prob);
}

int igabem_profile_enable(igabem_problem *P, int on) {
  return guarded([&] {
    if (!P) fail(IGABEM_EINVAL, "NULL problem");
    P->prof.on = on != 0;
  });
}

int igabem_profile_get(igabem_problem *P, igabem_profile *out, int reset) {
  return guarded([&] {
    if (!P || !out) fail(IGABEM_EINVAL, "NULL argument");
    P->prof.flush();
    out->launches = P->prof.launches;
    for (int i = 0; i < IGABEM_NPHASE; ++i) {
      out->ms[i] = P->prof.ms[i];
      out->calls[i] = P->prof.calls[i];
      out->phase_launches[i] = P->prof.phase_launches[i];
    }
    if (reset) P->prof.reset();
  });
}

int igabem_rhs(igabem_problem *P, int n_rhs, const double *dirs, void *b) {
  return guarded([&] {
    if (!P || !dirs || !b || n_rhs <= 0) fail(IGABEM_EINVAL, "invalid rhs arguments");
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    ensure_work(P, n_rhs, false);
    cudaStream_t st = P->stream;
    ProblemWork &W = ext(P)->work;
    double *ddir = W.red;  // 3 n_rhs doubles fit in the reduction scratch
    IGA_CUDA(cudaMemcpyAsync(ddir, dirs, 3 * sizeof(double) * n_rhs, cudaMemcpyHostToDevice, st));
    bool dev = is_device_ptr(b);
    double *out = dev ? static_cast<double *>(b) : W.yout;
    launch_rhs(P->d, P->S, P->opt, n_rhs, ddir, out, st);
    if (!dev)
      IGA_CUDA(cudaMemcpyAsync(b, out, P->S.N * n_rhs * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    P->prof.flush();
  });
}

int igabem_wait_selftest(igabem_ctx *ctx, double limit_s) {
  return guarded([&] {
    if (!ctx || !(limit_s > 0.0) || limit_s > 10.0) fail(IGABEM_EINVAL, "invalid self-test arguments");
    IGA_CUDA(cudaSetDevice(ctx->device));
    int *status = nullptr, v = 0;
    IGA_CUDA(cudaMalloc(&status, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) {
      launch_wait_selftest(status, limit_s, ctx->stream);
      e = cudaStreamSynchronize(ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpy(&v, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(status);
    IGA_CUDA(e);
    if (v) fail(IGABEM_ETIMEOUT, "bounded device wait gave up after its time limit (self-test)");
  });
}

int igabem_matvec(igabem_problem *P, int n_rhs, const void *x, void *y) {
  return guarded([&] {
    if (!P || !x || !y || n_rhs <= 0) fail(IGABEM_EINVAL, "invalid matvec arguments");
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    ensure_work(P, n_rhs, false);
    cudaStream_t st = P->stream;
    ProblemWork &W = ext(P)->work;
    size_t bytes = P->S.N * n_rhs * 2 * sizeof(double);
    bool dx = is_device_ptr(x), dy = is_device_ptr(y);
    const double *xi = dx ? static_cast<const double *>(x) : W.xin;
    double *yo = dy ? static_cast<double *>(y) : W.yout;
    if (!dx) IGA_CUDA(cudaMemcpyAsync(W.xin, x, bytes, cudaMemcpyHostToDevice, st));
    matvec_dev(P, n_rhs, xi, yo);
    if (!dy) IGA_CUDA(cudaMemcpyAsync(y, yo, bytes, cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    check_status(P);
    P->prof.flush();
  });
}

namespace {
int solve_impl(igabem_problem *P, int n_rhs, const double *dirs, int kind, void *density, igabem_solve_info *info);
}

int igabem_solve(igabem_problem *P, int n_rhs, const double *dirs, void *density, igabem_solve_info *info) {
  return solve_impl(P, n_rhs, dirs, 0, density, info);
}

int igabem_solve_sources(igabem_problem *P, int n_rhs, const double *z, void *density, igabem_solve_info *info) {
  return solve_impl(P, n_rhs, z, 1, density, info);
}

int igabem_rhs_sources(igabem_problem *P, int n_rhs, const double *z, void *b) {
  return guarded([&] {
    if (!P || !z || !b || n_rhs <= 0) fail(IGABEM_EINVAL, "invalid rhs arguments");
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    ensure_work(P, n_rhs, false);
    cudaStream_t st = P->stream;
    ProblemWork &W = ext(P)->work;
    IGA_CUDA(cudaMemcpyAsync(W.red, z, 3 * sizeof(double) * n_rhs, cudaMemcpyHostToDevice, st));
    bool dev = is_device_ptr(b);
    double *out = dev ? static_cast<double *>(b) : W.yout;
    launch_rhs(P->d, P->S, P->opt, n_rhs, W.red, out, st, 1);
    if (!dev)
      IGA_CUDA(cudaMemcpyAsync(b, out, P->S.N * n_rhs * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    P->prof.flush();
  });
}

}  // extern "C"

namespace {
int solve_impl(igabem_problem *P, int n_rhs, const double *dirs, int kind, void *density, igabem_solve_info *info) {
  int status = IGABEM_OK;
  int rc = guarded([&] {
    if (!P || !dirs || !density || n_rhs <= 0) fail(IGABEM_EINVAL, "invalid solve arguments");
    double t0 = now_ms();
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    ensure_work(P, n_rhs, true);
    cudaStream_t st = P->stream;
    ProblemWork &W = ext(P)->work;
    const HostSetup &S = P->S;
    const long N = S.N;
    const int R = n_rhs, m = W.gmres_m;
    const double tol = P->opt.tol;
    const size_t vb = N * R * 2 * sizeof(double);
    const int maxit = std::max(1, P->opt.max_iter);
    GmDev G = W.G;
    G.R = R;  // the buffers may be sized for more columns; every kernel works on the first R
    G.maxit = maxit;
    G.tol = tol;
    IGA_CUDA(cudaMemcpyAsync(W.red, dirs, 3 * sizeof(double) * R, cudaMemcpyHostToDevice, st));
    launch_rhs(P->d, S, P->opt, R, W.red, W.b, st, kind);
    std::vector<double> bn(R), beta(R);
    std::vector<int> its(R, 0), act(R);
    auto norms = [&](const double *v, std::vector<double> &out, double *dev_copy) {
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_norms(v, N, R, W.red, G.nrm, st);
      }
      if (dev_copy) IGA_CUDA(cudaMemcpyAsync(dev_copy, G.nrm, R * sizeof(double), cudaMemcpyDeviceToDevice, st));
      IGA_CUDA(cudaMemcpyAsync(out.data(), G.nrm, R * sizeof(double), cudaMemcpyDeviceToHost, st));
      IGA_CUDA(cudaStreamSynchronize(st));
    };
    norms(W.b, bn, G.bn);
    IGA_CUDA(cudaMemsetAsync(W.x, 0, vb, st));
    IGA_CUDA(cudaMemsetAsync(W.u, 0, vb, st));
    IGA_CUDA(cudaMemsetAsync(G.its, 0, R * sizeof(int), st));
    IGA_CUDA(cudaMemcpyAsync(W.r, W.b, vb, cudaMemcpyDeviceToDevice, st));
    beta = bn;
    int n_mv = 0;
    const bool pc = P->opt.precond != 0;
    // one Arnoldi step on the device: w = A V_j (A M^-1 V_j with the preconditioner), two CGS passes,
    // the Givens update and V_{j+1}; the finished flags are copied to page-locked host memory
    auto iteration = [&] {
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_copy_vj(G, W.vj, N, st);
        if (pc) launch_precond(P->d, S, P->opt, R, W.vj, W.t, st);
      }
      matvec_dev(P, R, pc ? W.t : W.vj, W.w);
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_gm_iteration_tail(G, W.red, N, st);
      }
      IGA_CUDA(cudaMemcpyAsync(W.hflags, G.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    };
    const bool use_graph = !P->opt.no_graph;
    IterGraph &IG = W.graph;
    if (use_graph && (!IG.exec || IG.R != R || IG.precond != (int)pc || IG.base != W.arena.base)) {
      IG.release();
      Profiler &pf = P->prof;
      const bool on = pf.on;
      const long l0 = pf.launches;
      long p0[IGABEM_NPHASE];
      std::copy(pf.phase_launches, pf.phase_launches + IGABEM_NPHASE, p0);
      pf.on = false;  // no event records inside the graph
      cudaGraph_t graph = nullptr;
      IGA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      try {
        iteration();
      } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        pf.on = on;
        throw;
      }
      pf.on = on;
      IGA_CUDA(cudaStreamEndCapture(st, &graph));
      cudaError_t e = cudaGraphInstantiate(&IG.exec, graph, 0);
      cudaGraphDestroy(graph);
      IGA_CUDA(e);
      IG.R = R;
      IG.precond = (int)pc;
      IG.base = W.arena.base;
      IG.launches = pf.launches - l0;
      for (int i = 0; i < IGABEM_NPHASE; ++i) {
        IG.phase_launches[i] = pf.phase_launches[i] - p0[i];
        pf.phase_launches[i] = p0[i];  // counted again at every replay
      }
      pf.launches = l0;
    }
    auto run_iteration = [&] {
      if (use_graph) {
        IGA_CUDA(cudaGraphLaunch(IG.exec, st));
        P->prof.launches += IG.launches;
        for (int i = 0; i < IGABEM_NPHASE; ++i) P->prof.phase_launches[i] += IG.phase_launches[i];
      } else {
        iteration();
      }
    };
    cudaEvent_t ev[2];
    IGA_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    IGA_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    struct EvGuard {
      cudaEvent_t *e;
      ~EvGuard() {
        cudaEventDestroy(e[0]);
        cudaEventDestroy(e[1]);
      }
    } ev_guard{ev};
    auto max_its = [&] { return *std::max_element(its.begin(), its.end()); };
    for (int r = 0; r < R; ++r) act[r] = beta[r] > tol * bn[r];
    auto any_active = [&] { return std::any_of(act.begin(), act.end(), [](int c) { return c != 0; }); };
    while (any_active() && max_its() < maxit) {
      IGA_CUDA(cudaMemcpyAsync(W.beta, beta.data(), R * sizeof(double), cudaMemcpyHostToDevice, st));
      IGA_CUDA(cudaMemcpyAsync(W.active, act.data(), R * sizeof(int), cudaMemcpyHostToDevice, st));
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_gm_init(G, W.beta, W.active, st);
        launch_scale(W.r, G.s, W.V, N, R, st);  // V_0 = r / beta
      }
      W.hflags[0] = W.hflags[1] = 0;
      for (int j = 0; j < m; ++j) {
        run_iteration();
        ++n_mv;
        IGA_CUDA(cudaEventRecord(ev[j & 1], st));
        // look one iteration behind: the flags only ever turn on within a cycle
        if (j >= 1) {
          IGA_CUDA(cudaEventSynchronize(ev[(j - 1) & 1]));
          if (W.hflags[0] || W.hflags[1]) break;
        }
      }
      IGA_CUDA(cudaStreamSynchronize(st));
      if (W.hflags[1]) fail(IGABEM_ENUMERIC, "GMRES met a non-finite value");
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_gm_solve(G, st);
        if (pc) {  // u += V y;  x = M^-1 u
          launch_update(W.V, m, reinterpret_cast<const double *>(G.y), W.u, N, R, st);
          launch_precond(P->d, S, P->opt, R, W.u, W.x, st);
        } else {
          launch_update(W.V, m, reinterpret_cast<const double *>(G.y), W.x, N, R, st);
        }
      }
      matvec_dev(P, R, W.x, W.w);
      ++n_mv;
      {
        Phase ph(&P->prof, IGABEM_PH_KRYLOV, st);
        launch_sub(W.b, W.w, W.r, N * R * 2, st);
      }
      norms(W.r, beta, nullptr);
      check_status(P);
      IGA_CUDA(cudaMemcpy(its.data(), G.its, R * sizeof(int), cudaMemcpyDeviceToHost));
      for (int r = 0; r < R; ++r) {
        if (!std::isfinite(beta[r])) fail(IGABEM_ENUMERIC, "GMRES met a non-finite residual");
        act[r] = beta[r] > tol * bn[r] && its[r] < maxit;
      }
    }
    bool dev = is_device_ptr(density);
    if (dev)
      IGA_CUDA(cudaMemcpyAsync(density, W.x, vb, cudaMemcpyDeviceToDevice, st));
    else
      IGA_CUDA(cudaMemcpyAsync(density, W.x, vb, cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    P->prof.flush();
    double worst = 0;
    for (int r = 0; r < R; ++r) worst = std::max(worst, bn[r] > 0 ? beta[r] / bn[r] : 0.0);
    if (info) {
      info->iterations = max_its();
      info->rel_residual = worst;
      info->n_matvecs = n_mv;
      info->solve_ms = now_ms() - t0;
    }
    if (worst > tol) {
      status = IGABEM_ENOT_CONVERGED;
      set_error("GMRES did not reach the tolerance within max_iter");
    }
  });
  return rc != IGABEM_OK ? rc : status;
}
}  // namespace

extern "C" {

int igabem_farfield(igabem_problem *P, int n_rhs, const void *density, int n_dir, const double *xhat,
                    void *uinf) {
  return guarded([&] {
    if (!P || !density || !xhat || !uinf || n_rhs <= 0 || n_dir <= 0) fail(IGABEM_EINVAL, "invalid far-field arguments");
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    ensure_work(P, n_rhs, false);
    cudaStream_t st = P->stream;
    ProblemWork &W = ext(P)->work;
    size_t db = P->S.N * n_rhs * 2 * sizeof(double);
    bool dd = is_device_ptr(density), du = is_device_ptr(uinf);
    const double *dens = dd ? static_cast<const double *>(density) : W.xin;
    if (!dd) IGA_CUDA(cudaMemcpyAsync(W.xin, density, db, cudaMemcpyHostToDevice, st));
    // directions and the result need their own device space
    double *dx = nullptr, *du_ = nullptr;
    IGA_CUDA(cudaMallocAsync(&dx, 3 * sizeof(double) * n_dir, st));
    IGA_CUDA(cudaMallocAsync(&du_, 2 * sizeof(double) * n_dir * n_rhs, st));
    IGA_CUDA(cudaMemcpyAsync(dx, xhat, 3 * sizeof(double) * n_dir, cudaMemcpyHostToDevice, st));
    launch_farfield(P->d, P->S, P->opt, n_rhs, dens, n_dir, dx, du_, P->d.gq, st);
    IGA_CUDA(cudaMemcpyAsync(uinf, du_, 2 * sizeof(double) * n_dir * n_rhs,
                             du ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaFreeAsync(dx, st));
    IGA_CUDA(cudaFreeAsync(du_, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    P->prof.flush();
  });
}

}  // extern "C"
