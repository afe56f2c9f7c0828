// Right-hand sides (Sec. 4.1), far-field pattern (Sec. 1) and the vector kernels of GMRES (Sec. 5.1).
#include <algorithm>

#include "internal.h"
#include "k_common.cuh"
#include "kernels.h"

namespace igabem {

namespace {

inline int grid_for(long n, int block = 256) {
  return (int)std::max<long>(1, std::min<long>((n + block - 1) / block, 152L * 32));
}

#define GRID_STRIDE(i, n) \
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

struct RhsArgs {
  const double *gpx, *gpn, *gpa, *phi1, *gw;
  const int *g2x_ptr, *g2x_idx;
  const double *dirs;     // per right-hand side: the direction d (plane wave) or the source point z
  long gst, N;
  int n1, nb, p, ng, R;
  double h, kappa, eta;
  bool hard;
  int kind;               // 0 plane waves exp(i kappa d.x); 1 point sources G(x, z)
};

// b[i][r] = sum over the elements of the supports of psi_i of sum_q w_q h^2 psi(q) f_r(q),
//   soft: f = grad u_inc . n~ - i eta a u_inc        (a (du_inc/dn - i eta u_inc))
//   hard: f = a u_inc - i eta grad u_inc . n~        (a (u_inc - i eta du_inc/dn))
// with u_inc = exp(i kappa d.x), grad u_inc = i kappa d u_inc (plane wave), or u_inc = G(x, z),
// grad u_inc = G (i kappa r - 1) / r^2 (x - z), r = |x - z| (point source at z).
__global__ void k_rhs(RhsArgs A, double2 *__restrict__ b) {
  const int p1 = A.p + 1, nq = A.ng * A.ng;
  GRID_STRIDE(o, A.N * A.R) {
    long gi = o / A.R;
    int r = int(o % A.R);
    const double *d = A.dirs + 3 * r;
    double2 acc = cmk(0, 0);
    for (int k = A.g2x_ptr[gi]; k < A.g2x_ptr[gi + 1]; ++k) {
      long X = A.g2x_idx[k];
      int j = int(X / ((long)A.nb * A.nb)), i1 = int((X / A.nb) % A.nb), i2 = int(X % A.nb);
      for (int ix = max(0, i1 - A.p); ix <= min(A.n1 - 1, i1); ++ix)
        for (int iy = max(0, i2 - A.p); iy <= min(A.n1 - 1, i2); ++iy) {
          long e = ((long)j * A.n1 + ix) * A.n1 + iy;
          int ka = i1 - ix, kb = i2 - iy;
          for (int q1 = 0; q1 < A.ng; ++q1)
            for (int q2 = 0; q2 < A.ng; ++q2) {
              long iq = e * nq + q1 * A.ng + q2;
              double x[3] = {A.gpx[iq], A.gpx[A.gst + iq], A.gpx[2 * A.gst + iq]};
              double n[3] = {A.gpn[iq], A.gpn[A.gst + iq], A.gpn[2 * A.gst + iq]};
              double2 f;
              if (A.kind == 0) {
                double dx = d[0] * x[0] + d[1] * x[1] + d[2] * x[2];
                double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
                double s, c;
                sincos(A.kappa * dx, &s, &c);
                f = A.hard ? cmk(A.gpa[iq] + A.eta * A.kappa * dn, 0.0) : cmk(0.0, A.kappa * dn - A.eta * A.gpa[iq]);
                f = cmul(f, cmk(c, s));
              } else {
                const double v[3] = {x[0] - d[0], x[1] - d[1], x[2] - d[2]};
                const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                double s, c;
                sincos(A.kappa * r, &s, &c);
                const double2 u = cmk(c / (4.0 * IGA_PI * r), s / (4.0 * IGA_PI * r));
                const double vn = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / (r * r);
                const double2 gn = cscale(cmul(u, cmk(-1.0, A.kappa * r)), vn);   // grad u_inc . n~
                const double2 ie_gn = cmk(-A.eta * gn.y, A.eta * gn.x);         // i eta grad u . n~
                const double2 ie_u = cmk(-A.eta * u.y * A.gpa[iq], A.eta * u.x * A.gpa[iq]);  // i eta a u
                f = A.hard ? csub(cscale(u, A.gpa[iq]), ie_gn) : csub(gn, ie_u);
              }
              double w = A.gw[q1] * A.gw[q2] * A.h * A.h *
                         A.phi1[(ix * A.ng + q1) * p1 + ka] * A.phi1[(iy * A.ng + q2) * p1 + kb];
              acc = cadd(acc, cscale(f, w));
            }
        }
    }
    b[o] = acc;
  }
}

// density at the Gauss points, weighted by w_q h^2: rho[e][q][r] = w_q h^2 sum_k psi_k(q) x[.][r]
__global__ void k_density(RhsArgs A, const int *__restrict__ x2g, const double2 *__restrict__ x,
                          long E, double2 *__restrict__ rho) {
  const int p1 = A.p + 1, nq = A.ng * A.ng;
  GRID_STRIDE(o, E * nq * A.R) {
    long e = o / (nq * A.R);
    int q = int((o / A.R) % nq), r = int(o % A.R), q1 = q / A.ng, q2 = q % A.ng;
    int j = int(e / ((long)A.n1 * A.n1)), ix = int((e / A.n1) % A.n1), iy = int(e % A.n1);
    double2 acc = cmk(0, 0);
    for (int ka = 0; ka < p1; ++ka)
      for (int kb = 0; kb < p1; ++kb) {
        long X = ((long)j * A.nb + ix + ka) * A.nb + iy + kb;
        double w = A.phi1[(ix * A.ng + q1) * p1 + ka] * A.phi1[(iy * A.ng + q2) * p1 + kb];
        acc = cadd(acc, cscale(x[(long)x2g[X] * A.R + r], w));
      }
    rho[o] = cscale(acc, A.gw[q1] * A.gw[q2] * A.h * A.h);
  }
}

// u_inf[k][r] = sum_points rho * exp(-i kappa x^_k . x) * (soft: -a/(4 pi); hard: -i kappa (x^.n~)/(4 pi))
__global__ void k_farfield(RhsArgs A, const double2 *__restrict__ rho, long npts,
                           const double *__restrict__ xhat, double2 *__restrict__ uinf) {
  __shared__ double2 red[256];
  const int k = blockIdx.x, r = blockIdx.y;
  const double *xh = xhat + 3 * k;
  double2 acc = cmk(0, 0);
  for (long i = threadIdx.x; i < npts; i += blockDim.x) {
    double x[3] = {A.gpx[i], A.gpx[A.gst + i], A.gpx[2 * A.gst + i]};
    double s, c;
    sincos(-A.kappa * (xh[0] * x[0] + xh[1] * x[1] + xh[2] * x[2]), &s, &c);
    double2 v = cmul(rho[i * A.R + r], cmk(c, s));
    if (A.hard) {
      double xn = xh[0] * A.gpn[i] + xh[1] * A.gpn[A.gst + i] + xh[2] * A.gpn[2 * A.gst + i];
      v = cmul(v, cmk(0.0, -A.kappa * xn));
    } else {
      v = cscale(v, -A.gpa[i]);
    }
    acc = cadd(acc, v);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) uinf[(long)k * gridDim.y + r] = cscale(red[0], 0.25 / IGA_PI);
}

// Far field in the mixed precisions, for many directions: the Gauss points are taken in groups of
// FE x FE elements with a reference point C (the group's first Gauss point, FP64); the phase
// kappa x^.y = kappa x^.C + kappa x^.(y - C) splits into a per-(direction, group) factor exp(-i kappa
// x^.C) in FP64 and per-point exponentials of the small offsets in FP32, summed in FP32 per group and
// direction, scaled by the FP64 factor and added over the groups in FP64.  Block: one group and 64
// directions, 4 point lanes per direction, up to 8 right-hand sides per pass.
constexpr int FF_DIRS = 64, FF_LANES = 4, FF_COLS = 8, FF_CHUNK = 256;

__global__ void __launch_bounds__(256) k_farfield32(RhsArgs A, const double2 *__restrict__ rho, int fe, int n_dir,
                                                    const double *__restrict__ xhat, double2 *__restrict__ uinf) {
  __shared__ float4 pts[FF_CHUNK];               // y - C (3), a
  __shared__ float4 nrm[FF_CHUNK];               // n~ (3)
  __shared__ float2 rs[FF_CHUNK * FF_COLS];      // weighted density (FP32)
  __shared__ float2 red[FF_LANES][FF_DIRS][FF_COLS];
  const int nq = A.ng * A.ng, ge = 1 << fe, ngr1 = A.n1 >> fe;
  const int g = blockIdx.x, j = g / (ngr1 * ngr1), gx = (g / ngr1) % ngr1, gy = g % ngr1;
  const int npts = ge * ge * nq;
  const int dl = threadIdx.x % FF_DIRS, lane = threadIdx.x / FF_DIRS;
  const int k = blockIdx.y * FF_DIRS + dl;
  const bool kv = k < n_dir;
  // reference point: the first Gauss point of the group
  const long e0 = ((long)j * A.n1 + gx * ge) * A.n1 + gy * ge;
  const double C0 = A.gpx[e0 * nq], C1 = A.gpx[A.gst + e0 * nq], C2v = A.gpx[2 * A.gst + e0 * nq];
  double xh[3] = {0.0, 0.0, 1.0};
  if (kv) {
    xh[0] = xhat[3 * k];
    xh[1] = xhat[3 * k + 1];
    xh[2] = xhat[3 * k + 2];
  }
  const float kx0 = (float)(-A.kappa * xh[0]), kx1 = (float)(-A.kappa * xh[1]), kx2 = (float)(-A.kappa * xh[2]);
  for (int c0 = 0; c0 < A.R; c0 += FF_COLS) {
    const int nc = min(FF_COLS, A.R - c0);
    float2 acc[FF_COLS];
#pragma unroll
    for (int c = 0; c < FF_COLS; ++c) acc[c] = make_float2(0.f, 0.f);
    for (int p0 = 0; p0 < npts; p0 += FF_CHUNK) {
      const int np = min(FF_CHUNK, npts - p0);
      __syncthreads();
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int pi = p0 + i, el = pi / nq, q = pi % nq;
        const long e = ((long)j * A.n1 + gx * ge + el / ge) * A.n1 + gy * ge + el % ge;
        const long iq = e * nq + q;
        pts[i] = make_float4((float)(A.gpx[iq] - C0), (float)(A.gpx[A.gst + iq] - C1),
                             (float)(A.gpx[2 * A.gst + iq] - C2v), (float)A.gpa[iq]);
        nrm[i] = make_float4((float)A.gpn[iq], (float)A.gpn[A.gst + iq], (float)A.gpn[2 * A.gst + iq], 0.f);
      }
      for (int i = threadIdx.x; i < np * FF_COLS; i += blockDim.x) {
        const int pi = i / FF_COLS, c = i % FF_COLS;
        const int el = (p0 + pi) / nq, q = (p0 + pi) % nq;
        const long e = ((long)j * A.n1 + gx * ge + el / ge) * A.n1 + gy * ge + el % ge;
        float2 v = make_float2(0.f, 0.f);
        if (c < nc) {
          const double2 r = rho[(e * nq + q) * A.R + c0 + c];
          v = make_float2((float)r.x, (float)r.y);
        }
        rs[i] = v;
      }
      __syncthreads();
      if (kv) {
        for (int i = lane; i < np; i += FF_LANES) {
          const float4 y = pts[i];
          float ph = fmaf(kx0, y.x, fmaf(kx1, y.y, kx2 * y.z));
          const float kq = rintf(ph * 0.15915494309189535f);
          ph = fmaf(-kq, 6.28318548202514648f, ph);
          ph = fmaf(-kq, -1.7484556e-07f, ph);
          float s, c;
          __sincosf(ph, &s, &c);
          float2 E;
          if (A.hard) {  // -i kappa (x^.n~) e
            const float4 n = nrm[i];
            const float xn = -fmaf(kx0, n.x, fmaf(kx1, n.y, kx2 * n.z));  // kappa x^.n~
            E = make_float2(xn * s, -xn * c);
          } else {       // -a e
            E = make_float2(-y.w * c, -y.w * s);
          }
#pragma unroll
          for (int cc = 0; cc < FF_COLS; ++cc) {
            const float2 r = rs[i * FF_COLS + cc];
            acc[cc].x = fmaf(E.x, r.x, fmaf(-E.y, r.y, acc[cc].x));
            acc[cc].y = fmaf(E.x, r.y, fmaf(E.y, r.x, acc[cc].y));
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < FF_COLS; ++c) red[lane][dl][c] = acc[c];
    __syncthreads();
    for (int i = threadIdx.x; i < FF_DIRS * FF_COLS; i += blockDim.x) {
      const int d = i / FF_COLS, c = i % FF_COLS, kk = blockIdx.y * FF_DIRS + d;
      if (kk >= n_dir || c >= nc) continue;
      double sx = 0.0, sy = 0.0;
      for (int l = 0; l < FF_LANES; ++l) {
        sx += (double)red[l][d][c].x;
        sy += (double)red[l][d][c].y;
      }
      // the group factor exp(-i kappa x^.C) of direction kk (recomputed by this thread)
      double s2, c2;
      sincos(-A.kappa * (xhat[3 * kk] * C0 + xhat[3 * kk + 1] * C1 + xhat[3 * kk + 2] * C2v), &s2, &c2);
      const double vx = (c2 * sx - s2 * sy) * (0.25 / IGA_PI), vy = (c2 * sy + s2 * sx) * (0.25 / IGA_PI);
      atomicAdd(&uinf[(long)kk * A.R + c0 + c].x, vx);
      atomicAdd(&uinf[(long)kk * A.R + c0 + c].y, vy);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------------------
// GMRES vector kernels; vectors are [N][R] complex, V_i = V + i N R

constexpr int RED_BLOCKS = 304;

// partial sums over chunks: red[(i*G + g)*R + r] = sum_{n in chunk g} conj(V_i[n][r]) w[n][r]
__global__ void k_multidot_partial(const double2 *__restrict__ V, const double2 *__restrict__ w,
                                   long N, int R, double2 *__restrict__ red) {
  extern __shared__ double2 sh[];
  const int i = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  const int nthr = (blockDim.x / R) * R;  // threads used: a multiple of R
  const double2 *Vi = V + (size_t)i * N * R;
  long chunk = (N + G - 1) / G, n0 = g * chunk, n1 = min(N, n0 + chunk);
  double2 acc = cmk(0, 0);
  if (threadIdx.x < nthr) {
    for (long idx = n0 * R + threadIdx.x; idx < n1 * R; idx += nthr) acc = cadd(acc, cconjmul(Vi[idx], w[idx]));
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < R) {
    double2 s = cmk(0, 0);
    for (int t = threadIdx.x; t < nthr; t += R) s = cadd(s, sh[t]);
    red[((size_t)i * G + g) * R + threadIdx.x] = s;
  }
}

__global__ void k_multidot_final(const double2 *__restrict__ red, int nv, int G, int R, double2 *__restrict__ h) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nv * R) return;
  int i = o / R, r = o % R;
  double2 s = cmk(0, 0);
  for (int g = 0; g < G; ++g) s = cadd(s, red[((size_t)i * G + g) * R + r]);
  h[o] = s;
}

__global__ void k_multiaxpy(const double2 *__restrict__ V, int nv, const double2 *__restrict__ h,
                            double2 *__restrict__ w, long N, int R, double sign) {
  GRID_STRIDE(o, N * R) {
    int r = int(o % R);
    double2 acc = w[o];
    for (int i = 0; i < nv; ++i) {
      double2 t = cmul(V[(size_t)i * N * R + o], h[i * R + r]);
      acc = cmk(acc.x + sign * t.x, acc.y + sign * t.y);
    }
    w[o] = acc;
  }
}

__global__ void k_scale(const double2 *__restrict__ w, const double *__restrict__ s, double2 *dst, long N, int R) {
  GRID_STRIDE(o, N * R) dst[o] = cscale(w[o], s[o % R]);
}

__global__ void k_sub(const double *__restrict__ b, const double *__restrict__ y, double *__restrict__ r, long n) {
  GRID_STRIDE(o, n) r[o] = b[o] - y[o];
}

__global__ void k_sqrt_re(const double2 *__restrict__ h, double *__restrict__ nrm, int R) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) nrm[r] = sqrt(fmax(h[r].x, 0.0));
}

// ---- device-side GMRES iteration: the Arnoldi index j lives on the device, so one captured graph
// serves every iteration of a cycle (the kernels read j; grids are sized for the whole cycle) ----

// partial sums of h[i][r] = sum_n conj(V_i[n][r]) w[n][r] for i <= j (blocks of i > j return)
__global__ void k_multidot_partial_dev(const double2 *__restrict__ V, const int *__restrict__ jdev,
                                       const double2 *__restrict__ w, long N, int R, double2 *__restrict__ red) {
  extern __shared__ double2 shd[];
  const int i = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  if (i > *jdev) return;
  const int nthr = (blockDim.x / R) * R;
  const double2 *Vi = V + (size_t)i * N * R;
  long chunk = (N + G - 1) / G, n0 = g * chunk, n1 = min(N, n0 + chunk);
  double2 acc = cmk(0, 0);
  if (threadIdx.x < nthr) {
    for (long idx = n0 * R + threadIdx.x; idx < n1 * R; idx += nthr) acc = cadd(acc, cconjmul(Vi[idx], w[idx]));
  }
  shd[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < R) {
    double2 sum = cmk(0, 0);
    for (int t = threadIdx.x; t < nthr; t += R) sum = cadd(sum, shd[t]);
    red[((size_t)i * G + g) * R + threadIdx.x] = sum;
  }
}

// h[i][r] for i <= j (zero above j), from the partial sums
__global__ void k_multidot_final_dev(const double2 *__restrict__ red, const int *__restrict__ jdev, int nmax, int G,
                                     int R, double2 *__restrict__ h) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nmax * R) return;
  int i = o / R, r = o % R;
  double2 sum = cmk(0, 0);
  if (i <= *jdev)
    for (int g = 0; g < G; ++g) sum = cadd(sum, red[((size_t)i * G + g) * R + r]);
  h[o] = sum;
}

// w[n][r] -= sum_{i <= j} V_i[n][r] h[i][r]
__global__ void k_multiaxpy_dev(const double2 *__restrict__ V, const int *__restrict__ jdev,
                                const double2 *__restrict__ h, double2 *__restrict__ w, long N, int R) {
  const int nv = *jdev + 1;
  GRID_STRIDE(o, N * R) {
    int r = int(o % R);
    double2 acc = w[o];
    for (int i = 0; i < nv; ++i) acc = csub(acc, cmul(V[(size_t)i * N * R + o], h[i * R + r]));
    w[o] = acc;
  }
}

// dst = V_j
__global__ void k_copy_vj(const double2 *__restrict__ V, const int *__restrict__ jdev, double2 *__restrict__ dst,
                          long NR) {
  const double2 *src = V + (size_t)(*jdev) * NR;
  GRID_STRIDE(o, NR) dst[o] = src[o];
}

// V_{j} = s w for the (already advanced) index j
__global__ void k_scale_vj(const double2 *__restrict__ w, const double *__restrict__ s, double2 *__restrict__ V,
                           const int *__restrict__ jdev, long N, int R) {
  double2 *dst = V + (size_t)(*jdev) * N * R;
  GRID_STRIDE(o, N * R) dst[o] = cscale(w[o], s[o % R]);
}

// cycle start: H, rotations and g cleared, g_0 = beta for the active columns, s = 1 / beta, j = 0
__global__ void k_gm_init(GmDev G, const double *__restrict__ beta, const int *__restrict__ active) {
  const int R = G.R, m = G.m;
  GRID_STRIDE(o, (long)(m + 1) * m * R) G.H[o] = cmk(0, 0);
  GRID_STRIDE(o, (long)m * R) {
    G.cs[o] = cmk(1, 0);
    G.sn[o] = cmk(0, 0);
  }
  GRID_STRIDE(o, (long)(m + 1) * R) G.g[o] = o < R && active[o] ? cmk(beta[o], 0) : cmk(0, 0);
  GRID_STRIDE(o, (long)R) {
    G.done[o] = active[o] ? 0 : 1;
    G.k[o] = 0;
    G.s[o] = active[o] ? 1.0 / beta[o] : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *G.j = 0;
    G.flags[0] = 0;
    G.flags[1] = 0;
  }
}

// Arnoldi column j of every active right-hand side: h = hA + hB (the two Gram-Schmidt passes), the
// new column of H rotated by the previous Givens rotations, the new rotation, g updated, the
// convergence test |g_{j+1}| <= tol ||b||; s = 1 / h_{j+1,j} for the next basis vector (0 for finished
// columns); then j advances.  One block; flags[0] = every column finished, flags[1] = non-finite met.
__global__ void k_gm_arnoldi(GmDev G) {
  const int R = G.R, m = G.m, j = *G.j;
  __shared__ int all_done, bad;
  if (threadIdx.x == 0) {
    all_done = 1;
    bad = 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (G.done[r]) {
      G.s[r] = 0.0;
      continue;
    }
    const double hn = G.nrm[r];
    double2 *Hc = G.H + (size_t)r;  // H[i][jj][r] at ((i * m) + jj) * R + r
    for (int i = 0; i <= j; ++i) Hc[((size_t)i * m + j) * R] = cadd(G.hA[i * R + r], G.hB[i * R + r]);
    Hc[((size_t)(j + 1) * m + j) * R] = cmk(hn, 0);
    for (int i = 0; i < j; ++i) {
      const double2 c = G.cs[i * R + r], sv = G.sn[i * R + r];
      const double2 a = Hc[((size_t)i * m + j) * R], b = Hc[((size_t)(i + 1) * m + j) * R];
      // [c, s; -conj(s), conj(c)] (a, b)
      Hc[((size_t)i * m + j) * R] = cadd(cmul(c, a), cmul(sv, b));
      Hc[((size_t)(i + 1) * m + j) * R] = cadd(cmul(cmk(-sv.x, sv.y), a), cmul(cmk(c.x, -c.y), b));
    }
    const double2 a = Hc[((size_t)j * m + j) * R], b = Hc[((size_t)(j + 1) * m + j) * R];
    const double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    const double2 c = den > 0 ? cmk(a.x / den, -a.y / den) : cmk(1, 0);
    const double2 sv = den > 0 ? cmk(b.x / den, -b.y / den) : cmk(0, 0);
    G.cs[j * R + r] = c;
    G.sn[j * R + r] = sv;
    Hc[((size_t)j * m + j) * R] = cmk(den, 0);
    Hc[((size_t)(j + 1) * m + j) * R] = cmk(0, 0);
    const double2 gj = G.g[j * R + r];
    G.g[(j + 1) * R + r] = cmul(cmk(-sv.x, sv.y), gj);
    G.g[j * R + r] = cmul(c, gj);
    G.k[r] = j + 1;
    const int its = ++G.its[r];
    const double2 gn = G.g[(j + 1) * R + r];
    const double res = sqrt(gn.x * gn.x + gn.y * gn.y);
    if (!isfinite(res) || !isfinite(hn)) atomicExch(&bad, 1);
    const bool done = res <= G.tol * G.bn[r] || its >= G.maxit || hn == 0.0 || j + 1 >= m;
    G.done[r] = done ? 1 : 0;
    G.s[r] = (!done && hn > 0) ? 1.0 / hn : 0.0;
    if (!done) atomicExch(&all_done, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    G.flags[0] = all_done;
    G.flags[1] = bad;
    *G.j = j + 1;
  }
}

// y = H^-1 g per column over its Krylov dimension k (zero beyond)
__global__ void k_gm_solve(GmDev G) {
  const int R = G.R, m = G.m;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const int kc = G.k[r];
    for (int i = m; i >= 0; --i) G.y[i * R + r] = cmk(0, 0);
    for (int i = kc - 1; i >= 0; --i) {
      double2 acc = G.g[i * R + r];
      for (int q = i + 1; q < kc; ++q) acc = csub(acc, cmul(G.H[((size_t)i * m + q) * R + r], G.y[q * R + r]));
      const double2 d = G.H[((size_t)i * m + i) * R + r];
      const double dd = d.x * d.x + d.y * d.y;
      G.y[i * R + r] = dd > 0 ? cmk((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd) : cmk(0, 0);
    }
  }
}

RhsArgs rhs_args(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R) {
  RhsArgs A;
  A.gpx = d.gpx; A.gpn = d.gpn; A.gpa = d.gpa; A.phi1 = d.phi1; A.gw = d.gw;
  A.g2x_ptr = d.g2x_ptr; A.g2x_idx = d.g2x_idx; A.dirs = nullptr;
  A.gst = (long)S.E * S.ng * S.ng; A.N = S.N;
  A.n1 = S.n1; A.nb = S.nb; A.p = S.p; A.ng = S.ng; A.R = R;
  A.h = S.h; A.kappa = o.kappa; A.eta = o.eta_cfie; A.hard = S.hard;
  A.kind = 0;
  return A;
}

}  // namespace

void launch_rhs(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                const double *dirs_dev, double *b, cudaStream_t st, int kind) {
  Phase ph(d.prof, IGABEM_PH_RHS, st);
  RhsArgs A = rhs_args(d, S, o, R);
  A.dirs = dirs_dev;
  A.kind = kind;
  k_rhs<<<grid_for(S.N * R), 256, 0, st>>>(A, reinterpret_cast<double2 *>(b));
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_density(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, const double *dens,
                    double *rho, cudaStream_t st) {
  RhsArgs A = rhs_args(d, S, o, R);
  const long npts = (long)S.E * S.ng * S.ng;
  k_density<<<grid_for(npts * R), 256, 0, st>>>(A, d.x2g, reinterpret_cast<const double2 *>(dens), S.E,
                                                 reinterpret_cast<double2 *>(rho));
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_farfield(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                     const double *dens, int n_dir, const double *xhat_dev, double *uinf, double *scratch,
                     cudaStream_t st) {
  if (R > 65535) fail(IGABEM_EINVAL, "the far field takes at most 65535 right-hand sides per call");
  Phase ph(d.prof, IGABEM_PH_FARFIELD, st);
  RhsArgs A = rhs_args(d, S, o, R);
  long npts = (long)S.E * S.ng * S.ng;
  double2 *rho = reinterpret_cast<double2 *>(scratch);  // E nq R complex values
  k_density<<<grid_for(npts * R), 256, 0, st>>>(A, d.x2g, reinterpret_cast<const double2 *>(dens), S.E, rho);
  note_launch();
  if (o.precision != IGABEM_FP64) {
    const int fe = std::min(S.m, 4);
    const long ngroups = (long)S.np << (2 * (S.m - fe));
    IGA_CUDA(cudaMemsetAsync(uinf, 0, sizeof(double2) * (size_t)n_dir * R, st));
    dim3 g32((unsigned)ngroups, (unsigned)((n_dir + FF_DIRS - 1) / FF_DIRS));
    k_farfield32<<<g32, 256, 0, st>>>(A, rho, fe, n_dir, xhat_dev, reinterpret_cast<double2 *>(uinf));
    note_launch();
    IGA_CUDA(cudaGetLastError());
    return;
  }
  dim3 grid(n_dir, R);
  k_farfield<<<grid, 256, 0, st>>>(A, rho, npts, xhat_dev, reinterpret_cast<double2 *>(uinf));
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_multidot(const double *V, int nv, const double *w, long N, int R, double *red,
                     double *h, cudaStream_t st) {
  int threads = std::max(R, (256 / R) * R);
  dim3 grid(RED_BLOCKS, nv);
  k_multidot_partial<<<grid, threads, threads * sizeof(double2), st>>>(
      reinterpret_cast<const double2 *>(V), reinterpret_cast<const double2 *>(w), N, R,
      reinterpret_cast<double2 *>(red));
  note_launch();
  k_multidot_final<<<(nv * R + 255) / 256, 256, 0, st>>>(reinterpret_cast<const double2 *>(red), nv,
                                                         RED_BLOCKS, R, reinterpret_cast<double2 *>(h));
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_gm_iteration_tail(const GmDev &G, double *red, long N, cudaStream_t st) {
  // two classical Gram-Schmidt passes against V_0..V_j, the norm, the Arnoldi update, the next basis vector
  const int R = G.R, threads = std::max(R, (256 / R) * R);
  for (int pass = 0; pass < 2; ++pass) {
    double2 *h = pass ? G.hB : G.hA;
    dim3 grid(RED_BLOCKS, G.m + 1);
    k_multidot_partial_dev<<<grid, threads, threads * sizeof(double2), st>>>(
        reinterpret_cast<const double2 *>(G.V), G.j, reinterpret_cast<const double2 *>(G.w), N, R,
        reinterpret_cast<double2 *>(red));
    note_launch();
    k_multidot_final_dev<<<((G.m + 1) * R + 255) / 256, 256, 0, st>>>(reinterpret_cast<const double2 *>(red), G.j,
                                                                     G.m + 1, RED_BLOCKS, R, h);
    note_launch();
    k_multiaxpy_dev<<<grid_for(N * R), 256, 0, st>>>(reinterpret_cast<const double2 *>(G.V), G.j, h,
                                                      reinterpret_cast<double2 *>(G.w), N, R);
    note_launch();
  }
  launch_norms(G.w, N, R, red, G.nrm, st);
  k_gm_arnoldi<<<1, 1024, 0, st>>>(G);
  note_launch();
  k_scale_vj<<<grid_for(N * R), 256, 0, st>>>(reinterpret_cast<const double2 *>(G.w), G.s,
                                               reinterpret_cast<double2 *>(G.V), G.j, N, R);
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_copy_vj(const GmDev &G, double *dst, long N, cudaStream_t st) {
  k_copy_vj<<<grid_for(N * G.R), 256, 0, st>>>(reinterpret_cast<const double2 *>(G.V), G.j,
                                                 reinterpret_cast<double2 *>(dst), N * G.R);
  note_launch();
}

void launch_gm_init(const GmDev &G, const double *beta, const int *active, cudaStream_t st) {
  k_gm_init<<<grid_for((long)(G.m + 1) * G.m * G.R), 256, 0, st>>>(G, beta, active);
  note_launch();
}

void launch_gm_solve(const GmDev &G, cudaStream_t st) {
  k_gm_solve<<<(G.R + 127) / 128, 128, 0, st>>>(G);
  note_launch();
}

void launch_multiaxpy(const double *V, int nv, const double *h, double *w, long N, int R, cudaStream_t st) {
  k_multiaxpy<<<grid_for(N * R), 256, 0, st>>>(reinterpret_cast<const double2 *>(V), nv,
                                                reinterpret_cast<const double2 *>(h),
                                                reinterpret_cast<double2 *>(w), N, R, -1.0);
  note_launch();
}

void launch_update(const double *V, int nv, const double *y, double *x, long N, int R, cudaStream_t st) {
  k_multiaxpy<<<grid_for(N * R), 256, 0, st>>>(reinterpret_cast<const double2 *>(V), nv,
                                                reinterpret_cast<const double2 *>(y),
                                                reinterpret_cast<double2 *>(x), N, R, 1.0);
  note_launch();
}

void launch_norms(const double *w, long N, int R, double *red, double *nrm, cudaStream_t st) {
  double *h = red + (size_t)2 * RED_BLOCKS * R * 2;  // past the partial sums of one vector
  launch_multidot(w, 1, w, N, R, red, h, st);
  k_sqrt_re<<<(R + 255) / 256, 256, 0, st>>>(reinterpret_cast<const double2 *>(h), nrm, R);
  note_launch();
}

void launch_scale(const double *w, const double *s, double *dst, long N, int R, cudaStream_t st) {
  k_scale<<<grid_for(N * R), 256, 0, st>>>(reinterpret_cast<const double2 *>(w), s,
                                            reinterpret_cast<double2 *>(dst), N, R);
  note_launch();
}

void launch_sub(const double *b, const double *y, double *r, long n, cudaStream_t st) {
  k_sub<<<grid_for(n), 256, 0, st>>>(b, y, r, n);
  note_launch();
}

}  // namespace igabem
