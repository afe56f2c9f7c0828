// Kernel samples of the M2L coupling blocks (Sec. 4.4) between the Chebyshev nodes of a target
// and a source cluster, in FP64 or FP32, and the small complex type they are returned in.
#pragma once

#include <type_traits>

#include "k_common.cuh"

namespace igabem {

template <class T> struct C2 {
  T x, y;
};
template <class T> __device__ inline C2<T> c2(T a, T b) { return {a, b}; }
template <class T> __device__ inline C2<T> add(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __device__ inline C2<T> mul(C2<T> a, C2<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __device__ inline C2<T> fma2(C2<T> a, C2<T> b, C2<T> acc) {  // acc + a b
  return {acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x};
}

// Sample of one node pair in precision T: returns the kernel value of the requested type.
//   type 0: soft  a_y G'(r)/r (x-y).n~x - i eta a_x a_y G
//   type 1: hard  a_x G'(r)/r (y-x).n~y
//   type 2: hard  G
// x, y: FP64 absolute node positions (FP64 path) or offsets from the cluster centres (FP32 path,
// with the pair constants D, |D|, |D|^2; the pair factor exp(i kappa |D|) is applied by the caller).
template <class T>
__device__ inline C2<T> node_sample(int type, const T *x, const T *nx, T ax, const T *y, const T *ny, T ay,
                                    const T *D, T Dn, T D2, T kappa, T eta) {
  constexpr bool F32 = std::is_same<T, float>::value;
  T d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  T r2, ir, r, cph, sph, dn_x, dn_y;
  if constexpr (F32) {
    T Dd = D[0] * d0 + D[1] * d1 + D[2] * d2;
    T dd = d0 * d0 + d1 * d1 + d2 * d2;
    T num = (T)2 * Dd + dd;
    r2 = D2 + num;
    ir = rsqrtf(r2);
    r = r2 * ir;
    T ph = kappa * __fdividef(num, r + Dn);
    T kq = rintf(ph * 0.15915494309189535f);
    ph = fmaf(-kq, 6.28318548202514648f, ph);
    ph = fmaf(-kq, -1.7484556e-07f, ph);
    __sincosf(ph, &sph, &cph);
    dn_x = D[0] * nx[0] + D[1] * nx[1] + D[2] * nx[2] + d0 * nx[0] + d1 * nx[1] + d2 * nx[2];
    dn_y = D[0] * ny[0] + D[1] * ny[1] + D[2] * ny[2] + d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
  } else {
    r2 = d0 * d0 + d1 * d1 + d2 * d2;
    ir = rsqrt(r2);
    r = r2 * ir;
    sincos(kappa * r, &sph, &cph);
    dn_x = d0 * nx[0] + d1 * nx[1] + d2 * nx[2];
    dn_y = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
  }
  const T f = ir * (T)(0.25 / IGA_PI), kr = kappa * r, g2 = f * ir * ir;
  const C2<T> G = c2(cph * f, sph * f);
  if (type == 2) return G;
  const C2<T> dG = c2((-cph - sph * kr) * g2, (-sph + cph * kr) * g2);
  if (type == 1) {
    T w1 = -ax * dn_y;
    return c2(dG.x * w1, dG.y * w1);
  }
  T w1 = ay * dn_x, w2 = ax * ay * eta;
  return c2(dG.x * w1 + G.y * w2, dG.y * w1 - G.x * w2);
}

}  // namespace igabem
