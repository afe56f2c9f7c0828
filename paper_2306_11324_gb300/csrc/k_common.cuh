// Device helpers shared by the kernels: complex arithmetic, rational Bezier evaluation, the
// Helmholtz kernel and its pull-backs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace igabem {

#define IGA_PI 3.14159265358979323846

// ----------------------------------------------------------------------------------------------
// complex numbers as (re, im) pairs

__host__ __device__ inline double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ inline double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return cmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline float2 fcmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ----------------------------------------------------------------------------------------------
// Bernstein polynomials B_k^n(u) and their derivatives, n <= 6

__device__ inline void bernstein_all(int n, double u, double *B, double *dB) {
  // B^0 = 1; B_k^d = (1-u) B_k^{d-1} + u B_{k-1}^{d-1}
  double Bl[8];
  B[0] = 1.0;
  for (int d = 1; d <= n; ++d) {
    if (d == n && dB) {
      for (int k = 0; k < d; ++k) Bl[k] = B[k];
    }
    double prev = 0.0;
    for (int k = 0; k < d; ++k) {
      double cur = B[k];
      B[k] = (1.0 - u) * cur + u * prev;
      prev = cur;
    }
    B[d] = u * prev;
  }
  if (dB) {
    if (n == 0) {
      dB[0] = 0.0;
      return;
    }
    // d/du B_k^n = n (B_{k-1}^{n-1} - B_k^{n-1})
    for (int k = 0; k <= n; ++k) {
      double a = k >= 1 ? Bl[k - 1] : 0.0;
      double b = k <= n - 1 ? Bl[k] : 0.0;
      dB[k] = n * (a - b);
    }
  }
}

// Rational Bezier patch with homogeneous net H[(i*(p2+1)+j)*4 + c]: F and dF/du, dF/dv.
__device__ inline void bez_eval(const double *__restrict__ H, int p1, int p2, double u, double v,
                                double F[3], double Fu[3], double Fv[3]) {
  double B1[8], dB1[8], B2[8], dB2[8];
  bernstein_all(p1, u, B1, dB1);
  bernstein_all(p2, v, B2, dB2);
  double h[4] = {0, 0, 0, 0}, hu[4] = {0, 0, 0, 0}, hv[4] = {0, 0, 0, 0};
  for (int i = 0; i <= p1; ++i)
    for (int j = 0; j <= p2; ++j) {
      const double *c = H + (i * (p2 + 1) + j) * 4;
      double bb = B1[i] * B2[j], bu = dB1[i] * B2[j], bv = B1[i] * dB2[j];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[k] += bb * c[k];
        hu[k] += bu * c[k];
        hv[k] += bv * c[k];
      }
    }
  double iw = 1.0 / h[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    F[k] = h[k] * iw;
    Fu[k] = (hu[k] - F[k] * hu[3]) * iw;
    Fv[k] = (hv[k] - F[k] * hv[3]) * iw;
  }
}

// The same evaluation done separably (contract the second parameter first); H may point to shared
// memory.
__device__ inline void bez_eval_sep(const double *__restrict__ H, int p1, int p2, double u, double v,
                                    double F[3], double Fu[3], double Fv[3]) {
  double B1[8], dB1[8], B2[8], dB2[8];
  bernstein_all(p1, u, B1, dB1);
  bernstein_all(p2, v, B2, dB2);
  double h[4] = {0, 0, 0, 0}, hu[4] = {0, 0, 0, 0}, hv[4] = {0, 0, 0, 0};
  for (int i = 0; i <= p1; ++i) {
    double r[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0};
    const double *c = H + i * (p2 + 1) * 4;
    for (int j = 0; j <= p2; ++j) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        r[k] += B2[j] * c[4 * j + k];
        rv[k] += dB2[j] * c[4 * j + k];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] += B1[i] * r[k];
      hu[k] += dB1[i] * r[k];
      hv[k] += B1[i] * rv[k];
    }
  }
  double iw = 1.0 / h[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    F[k] = h[k] * iw;
    Fu[k] = (hu[k] - F[k] * hu[3]) * iw;
    Fv[k] = (hv[k] - F[k] * hv[3]) * iw;
  }
}

__device__ inline void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// The square symmetry T_k (identity, rotations by 90/180/270 degrees, then the same after the
// diagonal reflection) applied to local coordinates.
__device__ inline void d4_apply(int k, double u, double v, double &ou, double &ov) {
  double a = u, b = v;
  if (k >= 4) {
    double t = a;
    a = b;
    b = t;
  }
  for (int r = 0; r < (k & 3); ++r) {
    double na = 1.0 - b, nb = a;
    a = na;
    b = nb;
  }
  ou = a;
  ov = b;
}

// ----------------------------------------------------------------------------------------------
// Helmholtz kernel pieces: G = exp(i kappa r)/(4 pi r), G'(r)/r = G (i kappa r - 1)/r^2

struct KernelVals {
  double2 G;     // G(r)
  double2 dGr;   // G'(r) / r
};

__device__ inline KernelVals helmholtz(double kappa, double r) {
  double s, c;
  sincos(kappa * r, &s, &c);
  double ir = 1.0 / r, f = ir * (0.25 / IGA_PI);
  KernelVals k;
  k.G = cmk(c * f, s * f);
  // G (i kappa r - 1) / r^2
  double2 t = cmk(-1.0, kappa * r);
  k.dGr = cscale(cmul(k.G, t), ir * ir);
  return k;
}

}  // namespace igabem
