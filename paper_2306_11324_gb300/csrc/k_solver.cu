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
  const double *dirs;
  long gst, N;
  int n1, nb, p, ng, R;
  double h, kappa, eta;
  bool hard;
};

// b[i][r] = sum over the elements of the supports of psi_i of sum_q w_q h^2 psi(q) f_r(q),
//   soft: f = (i kappa d.n~ - i eta a) exp(i kappa d.x)   (a (du_inc/dn - i eta u_inc))
//   hard: f = (a + eta kappa d.n~) exp(i kappa d.x)         (a (u_inc - i eta du_inc/dn))
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
              double dx = d[0] * x[0] + d[1] * x[1] + d[2] * x[2];
              double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
              double s, c;
              sincos(A.kappa * dx, &s, &c);
              double2 f = A.hard ? cmk(A.gpa[iq] + A.eta * A.kappa * dn, 0.0)
                                 : cmk(0.0, A.kappa * dn - A.eta * A.gpa[iq]);
              f = cmul(f, cmk(c, s));
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

RhsArgs rhs_args(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R) {
  RhsArgs A;
  A.gpx = d.gpx; A.gpn = d.gpn; A.gpa = d.gpa; A.phi1 = d.phi1; A.gw = d.gw;
  A.g2x_ptr = d.g2x_ptr; A.g2x_idx = d.g2x_idx; A.dirs = nullptr;
  A.gst = (long)S.E * S.ng * S.ng; A.N = S.N;
  A.n1 = S.n1; A.nb = S.nb; A.p = S.p; A.ng = S.ng; A.R = R;
  A.h = S.h; A.kappa = o.kappa; A.eta = o.eta_cfie; A.hard = S.hard;
  return A;
}

}  // namespace

void launch_rhs(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                const double *dirs_dev, double *b, cudaStream_t st) {
  Phase ph(d.prof, IGABEM_PH_RHS, st);
  RhsArgs A = rhs_args(d, S, o, R);
  A.dirs = dirs_dev;
  k_rhs<<<grid_for(S.N * R), 256, 0, st>>>(A, reinterpret_cast<double2 *>(b));
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
