/*
 * igabem.h -- C ABI of the GB300 isogeometric boundary element library for acoustic scattering.
 *
 * The library solves the combined field integral equations of Doelz, Harbrecht and Multerer,
 * "Solving acoustic scattering problems by the isogeometric boundary element method" (2023):
 *
 *   sound-soft  (1/2 + K' - i eta V) du/dn = du_inc/dn - i eta u_inc           (Sec. 2, eq. D2N)
 *   sound-hard  (1/2 - K  - i eta W) u     = u_inc     - i eta du_inc/dn       (Sec. 4.1, eq. CFIEN2D)
 *
 * discretised by Galerkin's method on spline spaces over NURBS patches (Sec. 3), with the
 * hypersingular operator in Maue's regularised form (Sec. 4.3), the matrix-vector product applied by
 * an interpolation (black-box) fast multipole method on the reference domain (Sec. 4.4), the systems
 * solved by restarted GMRES (Sec. 5.1), and the far-field pattern u_inf (Sec. 1) of the result.
 *
 * Conventions (all entry points):
 *   - time dependence exp(-i omega t): G(x,y) = exp(i kappa |x-y|) / (4 pi |x-y|);
 *     u_inc(x) = exp(i kappa d.x) with |d| = 1;
 *   - normals d_s F x d_t F point out of the scatterer (the caller's patches must be oriented so);
 *   - complex numbers are pairs of doubles (re, im), i.e. C99 double _Complex / numpy complex128;
 *   - a block of R vectors of length N is stored row-major as [N][R] (the R values of one degree of
 *     freedom are contiguous);
 *   - array arguments may point to host memory or to device memory of the context's device (the
 *     library asks the CUDA driver which); host arrays are copied, device arrays are used in place;
 *   - unless stated otherwise, inputs are copied and the caller keeps ownership of every array;
 *     handles are owned by the library until the matching *_destroy call;
 *   - every entry point returns IGABEM_OK (0) or a negative error code and, on error, leaves a
 *     message for igabem_last_error() of the calling thread; outputs are then unspecified;
 *   - calls on one context are not thread safe; work is issued on the context's stream and every
 *     entry point returns after that work has finished, unless stated otherwise.
 */
#ifndef IGABEM_H
#define IGABEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IGABEM_OK 0
#define IGABEM_EINVAL (-1)          /* invalid argument */
#define IGABEM_ENOMEM (-2)          /* device memory exhausted or admission refused */
#define IGABEM_ECUDA (-3)           /* a CUDA call failed */
#define IGABEM_ENOT_CONVERGED (-4)  /* GMRES stopped at max_iter; the density is still written */
#define IGABEM_ENUMERIC (-5)        /* NaN or Inf met */
#define IGABEM_ETIMEOUT (-6)        /* a bounded wait ran out */

typedef struct igabem_ctx igabem_ctx;
typedef struct igabem_geom igabem_geom;
typedef struct igabem_problem igabem_problem;

typedef enum { IGABEM_SOUND_SOFT = 0, IGABEM_SOUND_HARD = 1 } igabem_bc;

typedef enum {
  IGABEM_FP64 = 0,        /* every step in FP64 */
  IGABEM_MIXED_FP32 = 1,  /* far field (M2L, moments), regular near-field quadrature and the stored
                             near-field blocks in FP32 with FP32 accumulation per block; singular
                             quadrature, GMRES and residuals in FP64 */
  IGABEM_MIXED_TC = 2     /* IGABEM_MIXED_FP32 with the M2L of R >= 16 right-hand sides (R a multiple
                             of 16; sound-hard R <= 64, sound-soft R <= 512) on the tensor cores:
                             operands scaled by exact powers of two and split into FP16 hi + lo,
                             three products per pair, FP32 accumulation rounded to nearest per pair;
                             other R as IGABEM_MIXED_FP32 */
} igabem_precision;

typedef struct {
  int degree_p;        /* ansatz degree p >= 0 (p >= 1 for sound-hard) (Sec. 3.3) */
  int level_m;         /* uniform refinement level m: 2^m x 2^m elements per patch (Sec. 3.3) */
  double kappa;        /* wavenumber kappa >= 0 */
  double eta_cfie;     /* CFIE coupling eta (Sec. 2), any real non-zero value; kappa is usual */
  int bc;              /* igabem_bc */
  int cheb_q;          /* interpolation points per direction and cluster (Sec. 4.4), 2..16 */
  int leaf_offset;     /* b: the cluster tree stops at level m - b (leaves of 2^b x 2^b elements) */
  double eta_adm;      /* admissibility parameter: max(2r_t, 2r_s) <= eta_adm (dist - r_t - r_s) */
  double kappa_cap;    /* additionally require kappa max(2r) <= kappa_cap (<= 0: no cap) */
  int gauss_regular;   /* Gauss points per direction on regular element pairs (4) */
  int gauss_singular;  /* Gauss points per transformed variable on touching pairs (5) */
  int precision;       /* igabem_precision */
  int gmres_restart;   /* restart length (30, Sec. 5.1) */
  int max_iter;        /* iteration limit per right-hand side */
  double tol;          /* relative residual ||b - A x|| <= tol ||b|| */
  int no_fmm;          /* 1: treat every element pair as near (dense Galerkin matrix; tests) */
  int profile;         /* 1: per-phase CUDA-event timing from problem creation on (igabem_profile_*) */
  int precond;         /* GMRES preconditioner (the paper uses none): 0 none; 1 right preconditioner by the
                          inverses of the leaf clusters' diagonal near-field blocks, summed over the
                          overlapping leaves (block Jacobi).  The stopping test stays ||b - A x|| <= tol ||b||. */
  int q_max;           /* level-adaptive interpolation (the paper uses one q everywhere, Sec. 4.4): 0 or
                          cheb_q: cheb_q points on every level.  cheb_q < q_max <= 16 (needs kappa_cap > 0):
                          with eps(q, w) = w^q / (2^(q-1) q!), the bound of q-point Chebyshev interpolation
                          of exp(i w t) on [-1,1], and eps_ref = eps(cheb_q, kappa_cap / 2), level l takes
                          the smallest q in [cheb_q, q_max] with eps(q, kappa D_l / 2) <= eps_ref (D_l the
                          level's largest cluster diameter bound), else q_max, and admits pairs with
                          kappa max(2r) <= cap_l, eps(q_l, cap_l / 2) = eps_ref (kappa_cap where q_l =
                          cheb_q).  Expansions of a level whose q differs from its children's are formed
                          from and evaluated at the Gauss points directly. */
  int m2l_stored;      /* 0: M2L coupling blocks generated on the fly in every product (default);
                          1: generated once at set-up and kept in device memory (each far pair's q^2 x q^2
                          block per kernel type, FP32 in the mixed precisions, FP64 otherwise, with the
                          pair phase factor folded in), streamed by every product: the paper's H^2
                          storage of the compressed operator (Sec. 5.1), reused across iterations and
                          right-hand sides; igabem_problem_info reports the bytes */
  int no_graph;        /* 0: each GMRES iteration (matrix-vector product, Gram-Schmidt, Givens update, next
                          basis vector) is captured once as a CUDA graph with its state on the device and
                          replayed, the host only reading the finished flags one iteration behind;
                          1: the same kernels launched one by one (per-phase timing of the solve's
                          products, igabem_profile_*) */
} igabem_options;

/* Fills the defaults: p = 2, m = 3, kappa = 1, eta_cfie = kappa, sound-soft, q = 7, b = 0,
   eta_adm = 0.5, no cap, 4 / 5 Gauss points, FP64, restart 30, 1000 iterations, tol 1e-6, one q on
   every level. */
void igabem_default_options(igabem_options *opt);

typedef struct {
  long n_dofs;               /* N: dimension of S^2_{p,m} (soft) or S^0_{p,m} (hard) */
  long n_patch_dofs;         /* n (2^m+p)^2, the patch-wise coefficient space */
  long n_elements;           /* n 4^m */
  long n_clusters;           /* clusters on levels 0 .. m-b */
  long n_near_pairs;         /* near leaf-cluster pairs */
  long n_near_element_pairs; /* element pairs inside them */
  long n_touching_pairs;     /* identical, common-edge and common-vertex element pairs */
  long n_far_pairs;          /* admissible cluster pairs (M2L) over all levels */
  size_t device_bytes;       /* device memory held by the problem */
  double setup_ms;           /* wall time of igabem_problem_create */
  double host_setup_ms;      /* of which host-side set-up (tree, lists, tables) */
  long n_singular_points;    /* 4-D quadrature points evaluated for the touching pairs (Sec. 4.3 rules;
                                identical pairs take half of their rule, each point in both orientations) */
  int n_levels;              /* tree levels 0 .. m - b (at most 24 reported below) */
  int level_q[24];           /* interpolation points per direction on each level */
  long level_far[24];        /* admissible pairs on each level */
  long n_singular_geo_points;  /* element points whose geometry the touching pairs evaluate (a point
                                  repeated inside a chunk of the rule is evaluated once) */
  long n_singular_geo_columns; /* element nets contracted along their second coordinate, once per
                                  distinct value of it in a chunk */
  long n_singular_groups;      /* groups of 4-D points sharing the point of one element (per chunk, on the
                                  side with fewer distinct points): block entries are accumulated once
                                  per group */
  long n_singular_factored_points; /* of the 4-D points, those of identical sound-soft pairs summed in
                                      factorised form (groups of gauss_singular^2 points with tensor
                                      structure: univariate basis values, two nested sums) */
} igabem_info;

typedef struct {
  int iterations;            /* largest iteration count over the right-hand sides */
  double rel_residual;       /* largest final ||b - A x|| / ||b|| (recomputed with A) */
  int n_matvecs;             /* operator applications (one per block of right-hand sides) */
  double solve_ms;           /* wall time of the call */
} igabem_solve_info;

/* Phases of the per-problem profile. */
enum {
  IGABEM_PH_SETUP_TABLES = 0,  /* geometry at Gauss points and interpolation nodes */
  IGABEM_PH_SETUP_NEAR,        /* near-field Galerkin quadrature of the regular element pairs */
  IGABEM_PH_GATHER,            /* global <-> patch-wise / leaf-local vector gathers */
  IGABEM_PH_NEAR,              /* near-field block SpMV */
  IGABEM_PH_P2M,               /* leaf moments */
  IGABEM_PH_M2M,               /* upward transfers */
  IGABEM_PH_M2L,               /* admissible-pair couplings with on-the-fly kernel samples */
  IGABEM_PH_L2L,               /* downward transfers */
  IGABEM_PH_L2P,               /* evaluation and testing at the Gauss points */
  IGABEM_PH_KRYLOV,            /* GMRES vector kernels */
  IGABEM_PH_RHS,               /* right-hand sides */
  IGABEM_PH_FARFIELD,          /* far-field pattern */
  IGABEM_PH_SETUP_SINGULAR,    /* near-field Galerkin quadrature of the touching element pairs */
  IGABEM_NPHASE
};

typedef struct {
  long launches;                 /* kernels launched for the problem (always counted) */
  double ms[IGABEM_NPHASE];      /* device time per phase, CUDA events (only while enabled) */
  long calls[IGABEM_NPHASE];     /* timed executions per phase */
  long phase_launches[IGABEM_NPHASE]; /* kernels launched per phase (always counted) */
} igabem_profile;

/* Turns per-phase timing with CUDA events on the context's stream on (1) or off (0). */
int igabem_profile_enable(igabem_problem *prob, int on);

/* Copies the problem's counters; reset != 0 clears them afterwards. */
int igabem_profile_get(igabem_problem *prob, igabem_profile *out, int reset);

/* Last error message of the calling thread ("" if none). */
const char *igabem_last_error(void);

/* Creates a context on CUDA device `device`.  `stream` is a cudaStream_t of that device (for example
   PyTorch's current stream) or NULL, in which case the context creates its own stream. */
int igabem_create(igabem_ctx **out, int device, void *stream);
void igabem_destroy(igabem_ctx *ctx);

/* Copies a NURBS geometry of n_patches patch maps F_j : [0,1]^2 -> R^3 (Sec. 3.2).  Per patch j:
     degrees[2j], degrees[2j+1]  = (p1, p2) geometry degrees, 1..6;
     counts[2j], counts[2j+1]    = (k1, k2) control points per direction;
     knots: k1+p1+1 values then k2+p2+1 values, p-open on [0,1]; the patches' knot arrays follow
            each other;
     ctrl:  k1*k2 control points (x,y,z), index j1*k2 + j2 (j1 along the first parameter);
     weights: k1*k2 positive weights, same order.
   All arrays are host memory.  Patches must meet conformingly (Sec. 3.2).  Element boundaries at
   level m must include every interior knot (knots at multiples of 2^-m); problem creation fails
   with IGABEM_EINVAL otherwise. */
int igabem_geometry_create(igabem_ctx *ctx, int n_patches, const int *degrees, const int *counts,
                           const double *knots, const double *ctrl, const double *weights,
                           igabem_geom **out);
void igabem_geometry_destroy(igabem_geom *geom);

/* Sets up a discretised CFIE problem (Sec. 4): spaces, geometry tables, cluster tree and block
   partition, near-field Galerkin blocks (quadrature of Sec. 4.2-4.3), interpolation data.  The
   geometry must outlive the problem. */
int igabem_problem_create(igabem_geom *geom, const igabem_options *opt, igabem_problem **out);
int igabem_problem_info(const igabem_problem *prob, igabem_info *out);
void igabem_problem_destroy(igabem_problem *prob);

/* Right-hand sides of the CFIE (Sec. 4.1) for n_rhs incident directions dirs (host, [n_rhs][3],
   unit vectors): b = [N][n_rhs] complex. */
int igabem_rhs(igabem_problem *prob, int n_rhs, const double *dirs, void *b);

/* y = A x for the discretised CFIE operator A (far field by the fast multipole method unless
   no_fmm), x and y = [N][n_rhs] complex; x and y must not overlap. */
int igabem_matvec(igabem_problem *prob, int n_rhs, const void *x, void *y);

/* Solves A x = b(d_r) for the n_rhs directions by GMRES(restart) from x0 = 0; density = [N][n_rhs]
   complex (du/dn for sound-soft, u for sound-hard).  Returns IGABEM_ENOT_CONVERGED (density
   written) if a right-hand side missed the tolerance within max_iter iterations. */
int igabem_solve(igabem_problem *prob, int n_rhs, const double *dirs, void *density,
                 igabem_solve_info *info);

/* As igabem_solve for incident spherical waves from point sources, u_inc(x) = G(x, z_r) =
   exp(i kappa |x - z_r|) / (4 pi |x - z_r|) at the points z ([n_rhs][3], host, outside the scatterer:
   the direct formulation of Sec. 2 needs an incident field that solves the Helmholtz equation inside
   it), instead of plane waves: the right-hand sides of Sec. 4.1 with these u_inc, grad u_inc =
   G (i kappa r - 1) / r^2 (x - z). */
int igabem_solve_sources(igabem_problem *prob, int n_rhs, const double *z, void *density,
                         igabem_solve_info *info);
/* Right-hand sides of igabem_solve_sources: b = [N][n_rhs] complex. */
int igabem_rhs_sources(igabem_problem *prob, int n_rhs, const double *z, void *b);

/* The scattered field at n_pts points outside the scatterer (pts [n_pts][3], host or device) for n_rhs
   <= 8 densities ([N][n_rhs] complex, host or device): sound-soft u_s = -SL(t), sound-hard u_s = DL(u)
   (the representations of Sec. 2), summed over the regular Gauss rule of every element, by an
   interpolation fast multipole method in physical space (Sec. 4.4, last part, and Sec. 5.3): an octree
   over the sources and points (leaves of at most 64 Gauss points), min(cheb_q, 10)^3 Chebyshev nodes
   per box, eta_adm and kappa_cap as for the surface tree, kernel samples generated on the fly (FP32 in
   the mixed precisions, FP64 otherwise), the near field summed directly; no_fmm = 1 sums everything
   directly.  u = [n_pts][n_rhs] complex (host or device).  Allocates its octree and expansions for the
   duration of the call. */
int igabem_potential(igabem_problem *prob, int n_rhs, const void *density, int n_pts, const double *pts,
                     void *u);

/* Far-field pattern (Sec. 1) of n_rhs densities at n_dir unit directions xhat ([n_dir][3], host):
     sound-soft u_inf(x^) = -1/(4 pi) int exp(-i kappa x^.y) t(y) dsigma_y,
     sound-hard u_inf(x^) = -i kappa/(4 pi) int (x^.n_y) exp(-i kappa x^.y) u(y) dsigma_y,
   with the regular Gauss rule on every element; uinf = [n_dir][n_rhs] complex. */
int igabem_farfield(igabem_problem *prob, int n_rhs, const void *density, int n_dir,
                    const double *xhat, void *uinf);

/* ------------------------------------------------------------------------------------------------
 * Serving loop.  A server solves independent scattering requests (different geometries, levels,
 * wavenumbers, boundary conditions, right-hand-side counts) concurrently on one device: up to
 * max_active requests run at once, each on its own CUDA stream, and a request is admitted only when
 * the exact device memory of its set-up plus its solve fits the server's budget alongside the
 * requests already running; a request that arrives while others run starts as soon as a slot and
 * memory are free.  Each request runs the whole path (set-up, right-hand sides for its incident
 * directions, GMRES, far field at its directions) with its own options; its result does not depend
 * on what else runs.  Requests for the same problem (same geometry handle and identical options) are
 * batched: those waiting together are merged into one multi-column GMRES solve (shared matrix-vector
 * products), and a finished problem stays resident (tree, near-field blocks) for later requests with
 * the same key, in a least-recently-used cache that counts against the memory budget.
 * ------------------------------------------------------------------------------------------------ */
typedef struct igabem_server igabem_server;
typedef struct igabem_request igabem_request;

typedef struct {
  long submitted, completed, failed;
  double p50_ms, p99_ms, mean_ms; /* latency from submission to completion of completed requests */
  double solves_per_s;            /* completed requests / (last completion - first submission) */
  size_t peak_bytes;              /* largest admitted device memory at one time (resident problems included) */
  size_t budget_bytes;
  int peak_active;                /* largest number of requests running at one time */
  long merged;                    /* requests that joined another request's solve (same problem) */
  long cache_hits;                /* requests served by a resident problem (no set-up) */
  long resident;                  /* problems resident now */
} igabem_server_stats;

/* Starts a server with max_active worker threads (1..64) on the context's device.  memory_budget in
   bytes (0: 90 % of the free device memory; never more than the free memory). */
int igabem_server_create(igabem_ctx *ctx, size_t memory_budget, int max_active, igabem_server **out);
/* Finishes every submitted request, then stops the workers and frees the server. */
int igabem_server_destroy(igabem_server *srv);
/* Queues a request: geometry (must outlive the request), options (copied), n_rhs incident directions
   dirs[n_rhs][3] and n_dir far-field directions xhat[n_dir][3] (host arrays, copied).  Returns at
   once; the request handle belongs to the caller until igabem_request_destroy. */
int igabem_submit(igabem_server *srv, igabem_geom *geom, const igabem_options *opt, int n_rhs,
                  const double *dirs, int n_dir, const double *xhat, igabem_request **out);
/* *done = 1 once the request has finished (successfully or not). */
int igabem_poll(igabem_request *req, int *done);
/* Blocks until the request finished or timeout_s seconds passed (IGABEM_ETIMEOUT); timeout_s < 0
   waits without limit. */
int igabem_wait(igabem_request *req, double timeout_s);
/* Copies the far field uinf[n_dir][n_rhs] (complex, host memory) and the solve information (its
   solve_ms is the request's latency from submission); returns the request's status: IGABEM_OK,
   IGABEM_ENOMEM if the request alone exceeds the memory budget, IGABEM_ENOT_CONVERGED (far field
   still written), or the error of a failed set-up or solve.  IGABEM_ETIMEOUT if not finished. */
int igabem_result(igabem_request *req, void *uinf, igabem_solve_info *info);
/* Waits for the request if it is still running, then frees it. */
void igabem_request_destroy(igabem_request *req);
int igabem_server_get_stats(igabem_server *srv, igabem_server_stats *out);

/* Far-field pattern without any device memory allocation.  The paper has no counterpart: this is a
   property of the library for callers that cannot allocate device memory -- a host program whose
   own caching allocator has reserved the device (a library cudaMalloc would fail or fragment its
   pool), or a serving loop that must not stall on the implicit device synchronisation of
   cudaMalloc/cudaFree.  Same result as igabem_farfield, but density ([N][n_rhs] complex), xhat
   ([n_dir][3] doubles) and uinf ([n_dir][n_rhs] complex) must all be device memory of the context's
   device or managed memory (host memory, page-locked or not, and another GPU's memory are refused
   with IGABEM_EINVAL); n_rhs <= 65535.  The work runs on the problem's stream.  The problem must already exist (creating it
   allocates).  Scratch: a fixed 32 MiB device array inside the library (2^21 complex values, one per
   element x Gauss point x right-hand side), held by every device that loads the library until the
   process exits; calls with n_elements * gauss_regular^2 * n_rhs > 2^21 are refused with
   IGABEM_EINVAL.  The first call on a device looks up the array's device address; make that first
   call before any stream capture on the device.  All calls share the array: calls whose GPU work
   overlaps (other host threads, other contexts or streams on the same device) race and give wrong
   results. */
int igabem_farfield_noalloc(igabem_problem *prob, int n_rhs, const void *density, int n_dir,
                            const double *xhat, void *uinf);

/* Self-test of the bounded device waits (the paper has no counterpart).  The tensor-core M2L waits on
   mbarriers for its copies and MMAs; every wait gives up after a time limit, after which the kernel
   releases what it holds, records the failure in the problem's status word and returns, and the call
   reports IGABEM_ETIMEOUT instead of hanging the device.  This call runs the same wait routine on a
   barrier that nothing arrives at, with limit_s seconds (0 < limit_s <= 10), on the context's stream:
   it returns IGABEM_ETIMEOUT (the expected result, with a message) when the wait gave up, IGABEM_OK if it
   completed, IGABEM_EINVAL for a bad limit, IGABEM_ECUDA on a CUDA error.  The context stays usable. */
int igabem_wait_selftest(igabem_ctx *ctx, double limit_s);

/* Autotuner of the problem layout (the paper has no counterpart; it tunes this library's own
   parameters).  For the geometry, options and n_rhs columns it sets up and times every candidate
   layout that fits 60 % of the free device memory -- leaf_offset b in 1..min(level_m, 3) (leaves of
   2^b x 2^b elements) with the M2L coupling blocks generated on the fly or stored -- scoring set-up time
   + matvecs_per_setup x the time of one product (CUDA events, 3 products after a warm-up), and writes
   the caller's options with the best leaf_offset and m2l_stored into *out.  Choices are cached in
   memory and, when cache_path is not NULL, appended to that text file (one line per key: discretisation,
   wavenumber, precision, column count, geometry fingerprint) and read from it on later calls, so a
   later call with the same key returns at once (info->from_cache = 1).  Allocates device memory for the
   candidates while it runs; IGABEM_ENOMEM if no candidate fits. */
typedef struct {
  int leaf_offset, m2l_stored;  /* the choice */
  double setup_ms, matvec_ms;   /* measured for the choice (0 when taken from the cache) */
  double score_ms;              /* setup_ms + matvecs_per_setup x matvec_ms */
  int candidates;               /* layouts timed */
  int from_cache;               /* 1: the choice came from the cache */
} igabem_tune_info;
int igabem_autotune(igabem_geom *geom, const igabem_options *opt, int n_rhs, int matvecs_per_setup,
                    const char *cache_path, igabem_options *out, igabem_tune_info *info);

/* Measured arithmetic rates of the context's device (the paper has no counterpart: these are the
   denominators against which the library's benchmark quotes the roofline fractions of its ALU-bound
   kernels).  Each rate is timed with CUDA events on the context's stream, best of five launches after
   a warm-up, over a grid of 8 x 256 threads per SM whose threads run 8 independent chains of the
   operation; no setting of the GPU is changed (the clocks are whatever the GPU runs at).  Takes about
   a tenth of a second; allocates 2 KiB of device memory for the duration of the call. */
typedef struct {
  double fp32_tflops;       /* FP32 fused multiply-add rate, 2 flops per FMA */
  double fp64_tflops;       /* FP64 fused multiply-add rate, 2 flops per FMA */
  double sincosf_gops;      /* __sincosf calls per second (a sine and a cosine each, special-function unit) */
  double rsqrtf_gops;       /* rsqrtf calls per second */
  double sincos_fp64_gops;  /* FP64 sincos calls per second (the CUDA math library routine) */
  int sm_count;             /* multiprocessors of the device */
  double sm_clock_mhz_attr; /* the device's reported SM clock attribute (MHz), for reference */
} igabem_peaks;
int igabem_measure_peaks(igabem_ctx *ctx, igabem_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* IGABEM_H */
