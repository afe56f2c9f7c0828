// Internal declarations shared by the host set-up, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/igabem.h"

namespace igabem {

// ----------------------------------------------------------------------------------------------
// errors

struct Error {
  int code;
  std::string msg;
};
void set_error(const std::string &msg);
[[noreturn]] void fail(int code, const std::string &msg);
// Runs the body of a C entry point: returns IGABEM_OK, or the code of a fail() (its message left for
// igabem_last_error), IGABEM_ENOMEM for a host allocation failure, IGABEM_EINVAL for another exception.
// No C++ exception crosses the C ABI.
int run_guarded(const std::function<void()> &f);

#define IGA_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      ::igabem::fail(IGABEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

// Opt-in shared memory: kernels are set once to the device's largest opt-in size (a per-kernel value,
// so concurrent host threads never lower it under each other's launches); the launch's own size must
// not exceed it.
int max_optin_smem();
template <class K> cudaError_t set_max_dynamic_smem(K kernel, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int mx = max_optin_smem() - (int)fa.sharedSizeBytes;  // the kernel's static shared memory counts too
  if (bytes > (size_t)mx) fail(IGABEM_EINVAL, "kernel needs more shared memory than the device offers");
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

// ----------------------------------------------------------------------------------------------
// geometry input (host copy)

struct Patch {
  int p1, p2, k1, k2;
  std::vector<double> kn1, kn2;  // knot vectors
  std::vector<double> hw;        // homogeneous control net (w x, w y, w z, w), index (j1*k2+j2)*4
};

// ----------------------------------------------------------------------------------------------
// device arena: one allocation per problem, bump-allocated in 256-byte steps

struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  void reserve(size_t bytes);
  void *take(size_t bytes);
  template <class T> T *get(size_t n) { return static_cast<T *>(take(n * sizeof(T))); }
  void release();
};

// ----------------------------------------------------------------------------------------------
// host set-up products (plain arrays, uploaded once)

struct Rule4 {  // a rule on [0,1]^4 for touching element pairs, canonical position
  std::vector<double> x1, x2, y1, y2, w;
  // Sharing tables over chunks of sing_ch consecutive points: per chunk 6 counts, 6 lists of sing_ch
  // offsets (the first point of each distinct x1, x2, (x1, x2), y1, y2, (y1, y2) in the chunk), and
  // for each side the chunk's points grouped by their distinct point (sing_ch + 1 group offsets, then
  // sing_ch point offsets); then per point its 6 indices into the lists.
  std::vector<unsigned char> share;
};

// bytes of one chunk header of Rule4::share
inline int sing_share_header(int ch) { return 8 + 10 * ch; }

// Shared-memory layout of the singular kernel, offsets in doubles.  Three regions, each reused by
// steps that do not overlap in time: (A) the geometry column partials, then the per-point kernel values
// and basis values; (B) the distinct points' geometry, then the group sums; (C) the grouped side's basis
// values (written with the geometry, read by the accumulation); then the two element nets.
struct SingLayout {
  int s3, psi, cur, T, T2, U, geo, phiG, curG, nets, total;
};
inline SingLayout sing_layout(int ch, int nloc, bool hard, int nv, int nd, int pg1) {
  auto al = [](int x) { return (x + 1) & ~1; };  // double2 alignment
  auto mx = [](int a, int b) { return a > b ? a : b; };
  const int h3 = hard ? 3 : 0;
  SingLayout L;
  L.s3 = 0;                        // w k(x,y), w k(y,x), w gc per point (complex)
  L.psi = 6 * ch;                  // basis values on the side that is not grouped
  L.cur = L.psi + ch * nloc;       // and their curls
  const int endA = al(mx(L.cur + h3 * ch * nloc, 2 * nv * pg1 * 8));
  L.geo = endA;                    // x, d_s x, d_t x, n, |n| of the distinct points
  L.T = endA;                      // group sums of w k(x,y) times the basis values (complex)
  L.T2 = L.T + 2 * nd * nloc;      // the same with w k(y,x)
  L.U = L.T2 + 2 * nd * nloc;      // group sums of w gc times the curls (complex)
  const int endB = al(mx(L.geo + 2 * nd * 13, L.U + 2 * h3 * nd * nloc));
  L.phiG = endB;                   // basis values (and curls) of the grouped side's distinct points
  L.curG = L.phiG + nd * nloc;
  L.nets = L.curG + h3 * nd * nloc;
  L.total = L.nets + 8 * 49;
  return L;
}

struct TreeLevel {
  int n;                            // clusters on the level (n_patches 4^l)
  std::vector<double> center;       // 3 per cluster
  std::vector<double> radius;
  std::vector<int> far_ptr, far_src;  // admissible pairs, CSR by target cluster
  // interpolation on this level: q points per direction, kappa cap of its admissible pairs
  int q = 0;
  double cap = 0;
  std::vector<double> cheb;         // the q Chebyshev points on [0,1]
  std::vector<double> T1;           // [2][q][q] transfer to the children (when they use the same q)
  std::vector<double> LG;           // band bottom: [2^(m-l)][ng][q] Lagrange values at the Gauss points
  bool band_bottom = false;         // expansions built from / evaluated at the Gauss points directly
};

struct HostSetup {
  // discretisation
  int np = 0, m = 0, n1 = 0, E = 0, p = 0, nb = 0, nloc = 0;
  long NX = 0, N = 0;
  double h = 0, scale = 0;
  bool hard = false;
  // per-element rational Bezier geometry
  std::vector<int> edeg;       // 2 per element
  std::vector<long> eoff;      // offset (in doubles) of the element's homogeneous net
  std::vector<double> ebez;    // nets, 4 doubles per control point, index (i*(pg2+1)+j)
  std::vector<double> corners; // 4 corners x 3 per element, local (0,0),(1,0),(0,1),(1,1)
  // quadrature
  int ng = 4, ns = 5;
  int sing_ch = 128, sing_nv = 0, sing_nd = 0;  // singular chunk; most distinct coordinates / points in one
  bool sing_fact = false;  // identical sound-soft pairs summed in factorised form (k_near_singular)
  std::vector<double> gx, gw;          // Gauss rule on [0,1] (ng points)
  Rule4 r_id, r_edge, r_vert;
  // ansatz basis: per element column ix, Gauss point q, function a: value and d/ds
  std::vector<double> phi1, dphi1;     // [n1][ng][p+1]
  std::vector<double> ext1;            // Bernstein extraction [n1][p+1 (fn)][p+1 (bern)]
  // touching pairs (e, f, kind 0/1/2, Te, Tf)
  std::vector<int> touch;              // 5 ints per pair
  // continuous space gluing
  std::vector<int> x2g;                // NX
  std::vector<int> g2x_ptr, g2x_idx;   // CSR N -> X
  // tree
  int L = 0, b = 0, q = 7, nL1 = 0, nL = 0, lmin = 0;
  bool no_fmm = false;
  std::vector<TreeLevel> lev;
  std::vector<int> near_ptr, near_src; // near leaf pairs, CSR by target leaf
  std::vector<int> touch_blk;          // per touching pair: index of its near leaf pair
  std::vector<int> nbr;                // [E][nbr_w]: elements touching each element (-1 padded)
  int nbr_w = 1;
  // work list of the singular quadrature: each unordered touching pair once,
  // (e, f, kind, Te, Tf, block of (e,f), block of (f,e) or -1 for identical pairs)
  std::vector<int> sing;
  std::vector<int> diag_blk;           // per leaf: index of its diagonal near block (t, t)
  long n_far = 0;
  // interpolation tables
  std::vector<double> cheb;            // normalised Chebyshev nodes t_a on [0,1]
  std::vector<double> T1;              // [2][q][q]: L_a(parent) at child node a'
  std::vector<double> LG1;             // [2^b][ng][q]: leaf Lagrange at Gauss points
};

// Host set-up products that depend on the geometry and the level m alone (and the cluster balls on the
// leaf level m - b): kept with the geometry, so that problems on it at other wavenumbers, precisions or
// right-hand-side counts (a frequency sweep, repeated serving requests) skip their construction.
struct GeoCache {
  int m = -1, L = -1;
  std::vector<int> edeg;
  std::vector<long> eoff;
  std::vector<double> ebez, corners;
  double scale = 0;
  std::vector<int> touch, nbr;
  int nbr_w = 0;
  std::vector<std::vector<double>> center, radius;  // cluster balls on levels 0..L
};

// hit: products of an earlier call for the same geometry and level m (or nullptr); fill: receives this
// call's products when hit does not apply (or nullptr)
void build_setup(const std::vector<Patch> &patches, const igabem_options &opt, HostSetup &S,
                 const GeoCache *hit = nullptr, GeoCache *fill = nullptr);

// Gauss-Legendre rule on [0,1] (Newton iteration on P_n).
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w);

}  // namespace igabem

// ----------------------------------------------------------------------------------------------
// handles

struct igabem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
};

struct igabem_geom {
  igabem_ctx *ctx = nullptr;
  std::vector<igabem::Patch> patches;
  std::mutex cache_mu;
  std::shared_ptr<const igabem::GeoCache> cache;  // the latest level's host set-up products
};

namespace igabem {

// Per-problem profile: launch counters (always) and per-phase CUDA-event timing (when enabled).
struct Profiler {
  bool on = false;
  long launches = 0;
  long phase_launches[IGABEM_NPHASE] = {};
  double ms[IGABEM_NPHASE] = {};
  long calls[IGABEM_NPHASE] = {};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t event();
  void flush();  // accumulates pending event pairs; call after the stream has been synchronised
  void reset();
  ~Profiler();
};

// Scope of one phase on a stream: records start/stop events when timing is on, and makes
// note_launch() count launches against this phase.
class Phase {
 public:
  Phase(Profiler *p, int phase, cudaStream_t st);
  ~Phase();

 private:
  Profiler *p_;
  int ph_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr;
  Profiler *prev_p_;
  int prev_ph_;
};
void note_launch();

// device copies of the set-up and the working buffers of a problem
struct DeviceProblem {
  Profiler *prof = nullptr;
  // element tables
  int *edeg;
  long *eoff;
  double *ebez;
  double *gpx, *gpn, *gpa, *gfs, *gft;    // Gauss-point geometry: [3][E*ng*ng] or [E*ng*ng]
  double *phi1, *dphi1, *ext1, *gx, *gw;
  float *phi1f, *gwqf;  // FP32 copies: B-spline values at the Gauss points, gw[q1] gw[q2] h^2 per point
  double *rule[3];                          // singular rules (5 arrays each, SoA)
  unsigned char *share[3];                  // their sharing tables (Rule4::share)
  int rule_n[3];
  double *corners;
  int *touch, *touch_blk, *sing;
  int *nbr = nullptr;                        // [E][nbr_w] touching elements
  void *near_tab = nullptr;                  // set-up scratch: element tables of the regular quadrature
  int *x2g, *g2x_ptr, *g2x_idx;
  // tree
  int *near_ptr, *near_src, *near_tgt;
  std::vector<int *> far_ptr, far_src;       // per level
  std::vector<double *> nodes;               // per level: [7][n*q*q] (x, n~, a) node geometry
  std::vector<float *> nodes32;              // per level: [7][n*q*q] (x - centre, n~, a) in FP32
  std::vector<double *> centers;             // per level: [n][3] cluster centres
  std::vector<float *> pairc;                // per level: [n_far][8] FP32 pair constants
  std::vector<double *> cext;                // per level: [n][2] node extent and largest Jacobian
  std::vector<double *> chebl;               // per level: its q Chebyshev points on [0,1]
  std::vector<double *> T1l;                 // per level: [2][q][q] transfer to the children (same q)
  std::vector<double *> m2ls;                // stored M2L blocks per level (m2l_stored): [n_far][types][q^2 b][q^2 a]
                                             // complex, FP32 (mixed) or FP64, pair phase factor folded in
  std::vector<double *> LGl;                 // per band-bottom level: [2^(m-l)][ng][q] Lagrange at Gauss points
  std::vector<uint8_t *> tc_bimg;            // per level: tensor-core M2L operands of the sources
  std::vector<float *> tc_bscale;            // per level: power-of-two scale of each cluster's operand
  int *status = nullptr;                     // device status word: non-zero after a timed-out wait
  double *lm64 = nullptr;                    // leaf moment matrices [n_leaf][nL][q^2 C] (FP64 precision)
  float *lm32 = nullptr;                     // the same in FP32 (mixed precision)
  double *T1, *LG1;
  // near-field blocks (column-major nL x nL per near pair)
  double *blk = nullptr;                     // complex FP64: 2 doubles per entry (FP64 precision)
  float *blk32 = nullptr;                    // complex FP32 copy used by the mixed precision SpMV
  // preconditioner: inverses of the diagonal leaf blocks (column-major, complex FP64), identity lists
  double *binv = nullptr;
  int *diag_blk = nullptr, *ident_ptr = nullptr, *ident_src = nullptr;
  // work buffers, sized for max_rhs columns
  int max_rhs = 0;
  double *xX = nullptr;                      // X-space input [NX][R] complex
  double *yleaf = nullptr;                   // leaf-local outputs [n_leaf][nL][R] complex
  double *gq = nullptr;                      // channel values at Gauss points [E][nq][C][R]
  std::vector<void *> xhat, yhat;            // expansions per level [n][q*q][C][R]
  // mixed precisions: FP32 copies made once per product for the kernels that compute in FP32 (the
  // expansions after the upward pass, the input vector, the leaf-level local expansions)
  std::vector<float2 *> xhat32;
  float2 *xX32 = nullptr, *y32 = nullptr;
  double *xin = nullptr, *yout = nullptr;    // device staging of caller vectors [N][R]
  double *red = nullptr;                     // reduction scratch
};

}  // namespace igabem

struct igabem_problem;
namespace igabem {
igabem_problem *problem_plan(igabem_geom *geom, const igabem_options *opt);
void problem_materialize(igabem_problem *P, cudaStream_t st);
void problem_release(igabem_problem *P);
size_t problem_work_bytes(const HostSetup &S, int R, int gmres_m, int precision);
double now_ms();
}  // namespace igabem

struct igabem_problem {
  igabem::Profiler prof;
  igabem_geom *geom = nullptr;
  cudaStream_t stream = nullptr;   // the stream all of the problem's work is issued on
  size_t arena_bytes = 0;          // device memory of the set-up arena
  size_t temp_bytes = 0;           // transient device memory during set-up
  double t_plan = 0;
  igabem_options opt{};
  igabem::HostSetup S;
  igabem::Arena arena;
  igabem::DeviceProblem d{};
  igabem_info info{};
};
