// Set-up kernels: geometry tables at Gauss points and interpolation nodes, and the near-field
// Galerkin blocks (Sec. 4.2-4.3 with the quadrature rules for regular and touching element pairs).
#include <type_traits>

#include "internal.h"
#include "k_common.cuh"
#include "kernels.h"

namespace igabem {

// ----------------------------------------------------------------------------------------------
// geometry at the Gauss points of every element: x, n~ = d_s F x d_t F, a = |n~|, d_s F, d_t F

__global__ void k_gauss_geometry(const int *__restrict__ edeg, const long *__restrict__ eoff,
                                 const double *__restrict__ ebez, const double *__restrict__ gx,
                                 int E, int ng, double n1, double *gpx, double *gpn, double *gpa,
                                 double *gfs, double *gft) {
  long tot = (long)E * ng * ng;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
    int e = int(i / (ng * ng)), q = int(i % (ng * ng));
    double F[3], Fu[3], Fv[3], fs[3], ft[3], n[3];
    bez_eval(ebez + eoff[e], edeg[2 * e], edeg[2 * e + 1], gx[q / ng], gx[q % ng], F, Fu, Fv);
    for (int k = 0; k < 3; ++k) {
      fs[k] = Fu[k] * n1;  // d/ds = 2^m d/du
      ft[k] = Fv[k] * n1;
    }
    cross3(fs, ft, n);
    for (int k = 0; k < 3; ++k) {
      gpx[k * tot + i] = F[k];
      gpn[k * tot + i] = n[k];
      gfs[k * tot + i] = fs[k];
      gft[k * tot + i] = ft[k];
    }
    gpa[i] = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  }
}

// geometry at the Chebyshev nodes of every cluster of level l: [7][n_clusters*q*q] = x, n~, a
__global__ void k_node_geometry(const int *__restrict__ edeg, const long *__restrict__ eoff,
                                const double *__restrict__ ebez, const double *__restrict__ cheb,
                                const double *__restrict__ center, int n_clusters, int l, int q, int n1,
                                double *out, float *out32) {
  long tot = (long)n_clusters * q * q;
  int nl = 1 << l;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
    int t = int(i / (q * q)), a = int(i % (q * q));
    int j = t / (nl * nl), cx = (t / nl) % nl, cy = t % nl;
    double s = (cx + cheb[a / q]) / nl, tt = (cy + cheb[a % q]) / nl;
    int ix = min(int(s * n1), n1 - 1), iy = min(int(tt * n1), n1 - 1);
    int e = (j * n1 + ix) * n1 + iy;
    double F[3], Fu[3], Fv[3], fs[3], ft[3], n[3];
    bez_eval(ebez + eoff[e], edeg[2 * e], edeg[2 * e + 1], s * n1 - ix, tt * n1 - iy, F, Fu, Fv);
    for (int k = 0; k < 3; ++k) {
      fs[k] = Fu[k] * n1;
      ft[k] = Fv[k] * n1;
    }
    cross3(fs, ft, n);
    double v[7] = {F[0], F[1], F[2], n[0], n[1], n[2], sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2])};
    for (int k = 0; k < 7; ++k) {
      out[k * tot + i] = v[k];
      // FP32 copy: positions relative to the cluster centre
      out32[k * tot + i] = (float)(k < 3 ? v[k] - center[3 * t + k] : v[k]);
    }
  }
}

// ----------------------------------------------------------------------------------------------
// Kernel of the CFIE for one point pair, split as  ks psi_k(x) psi_l(y) + gc c_k(x) . c_l(y):
//   sound-soft  ks = a_y G'(r)/r (x-y).n~_x - i eta a_x a_y G,  gc = 0            (K' - i eta V)
//   sound-hard  ks = -a_x G'(r)/r (y-x).n~_y + i eta kappa^2 (n~_x.n~_y) G,  gc = -i eta G
//                                                                        (-K - i eta W, Maue)

struct PairKernel {
  double2 ks, gc;
};

__device__ inline PairKernel cfie_kernel(bool hard, double kappa, double eta, const double *x,
                                         const double *nx, double ax, const double *y,
                                         const double *ny, double ay) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  KernelVals kv = helmholtz(kappa, r);
  PairKernel pk;
  if (!hard) {
    double dn = d[0] * nx[0] + d[1] * nx[1] + d[2] * nx[2];
    double2 kp = cscale(kv.dGr, ay * dn);
    double2 v = cscale(kv.G, ax * ay);
    pk.ks = cmk(kp.x + eta * v.y, kp.y - eta * v.x);  // kp - i eta v
    pk.gc = cmk(0.0, 0.0);
  } else {
    double dn = -(d[0] * ny[0] + d[1] * ny[1] + d[2] * ny[2]);
    double2 kk = cscale(kv.dGr, ax * dn);
    double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double2 g = kv.G;
    double f = eta * kappa * kappa * nn;
    pk.ks = cmk(-kk.x - f * g.y, -kk.y + f * g.x);
    pk.gc = cmk(eta * g.y, -eta * g.x);  // -i eta G
  }
  return pk;
}

// Both orientations of a touching pair from one evaluation of G: the kernel at (x, y) and the ks part
// at (y, x) (gc is symmetric).
__device__ inline void cfie_kernel_both(bool hard, double kappa, double eta, const double *x, const double *nx,
                                        double ax, const double *y, const double *ny, double ay,
                                        PairKernel &xy, double2 &ks_yx) {
  double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  KernelVals kv = helmholtz(kappa, r);
  const double dnx = d[0] * nx[0] + d[1] * nx[1] + d[2] * nx[2];   // (x-y).n~x
  const double dny = d[0] * ny[0] + d[1] * ny[1] + d[2] * ny[2];   // (x-y).n~y
  if (!hard) {
    double2 v = cscale(kv.G, ax * ay);
    double2 kp = cscale(kv.dGr, ay * dnx);
    xy.ks = cmk(kp.x + eta * v.y, kp.y - eta * v.x);
    xy.gc = cmk(0.0, 0.0);
    double2 kq = cscale(kv.dGr, -ax * dny);                        // a_x G'/r (y-x).n~y
    ks_yx = cmk(kq.x + eta * v.y, kq.y - eta * v.x);
  } else {
    double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double f = eta * kappa * kappa * nn;
    double2 g = kv.G;
    double2 kk = cscale(kv.dGr, -ax * dny);                        // a_x G'/r (y-x).n~y
    xy.ks = cmk(-kk.x - f * g.y, -kk.y + f * g.x);
    xy.gc = cmk(eta * g.y, -eta * g.x);
    double2 kk2 = cscale(kv.dGr, ay * dnx);                        // a_y G'/r (x-y).n~x
    ks_yx = cmk(-kk2.x - f * g.y, -kk2.y + f * g.x);
  }
}

template <class T> struct PK {
  T ksx, ksy, gcx, gcy;
};

// the same kernel in precision T (FP32 for the regular pairs of the mixed precision set-up)
template <class T>
__device__ inline PK<T> cfie_kernel_t(bool hard, T kappa, T eta, const T *x, const T *nx, T ax, const T *y,
                                      const T *ny, T ay) {
  T d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  T r2 = d0 * d0 + d1 * d1 + d2 * d2;
  T ir, sn, cs;
  if constexpr (sizeof(T) == 4) {
    ir = rsqrtf(r2);
    sincosf(kappa * r2 * ir, &sn, &cs);
  } else {
    ir = rsqrt(r2);
    sincos(kappa * r2 * ir, &sn, &cs);
  }
  const T r = r2 * ir, f = ir * (T)(0.25 / IGA_PI), kr = kappa * r, g2 = f * ir * ir;
  const T Gx = cs * f, Gy = sn * f;
  const T dGx = (-cs - sn * kr) * g2, dGy = (-sn + cs * kr) * g2;
  PK<T> pk;
  if (!hard) {
    T w1 = ay * (d0 * nx[0] + d1 * nx[1] + d2 * nx[2]), w2 = ax * ay * eta;
    pk.ksx = dGx * w1 + Gy * w2;
    pk.ksy = dGy * w1 - Gx * w2;
    pk.gcx = 0;
    pk.gcy = 0;
  } else {
    T w1 = -ax * (d0 * ny[0] + d1 * ny[1] + d2 * ny[2]);
    T f2 = eta * kappa * kappa * (nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2]);
    pk.ksx = -dGx * w1 - f2 * Gy;
    pk.ksy = -dGy * w1 + f2 * Gx;
    pk.gcx = eta * Gy;
    pk.gcy = -eta * Gx;
  }
  return pk;
}

// ----------------------------------------------------------------------------------------------
// regular element pairs of the near field: tensor Gauss rule on both elements

struct NearArgs {
  const double *gpx, *gpn, *gpa, *gfs, *gft;  // Gauss-point geometry, SoA with stride gstride
  const double *phi1, *dphi1, *ext1, *gw, *corners;
  const int *edeg;
  const long *eoff;
  const double *ebez;
  const int *near_tgt, *near_src;
  long gstride;
  int n1, ng, p, nloc, b, nL1, nL, L;
  double h, kappa, eta, tol;
  bool hard;
  double2 *blk;
  // per-element tables of the regular quadrature (precision of the kernel): Gauss-point geometry
  // [E][nq][7] (x, n~, a), weighted basis values [E][nq][nloc], weighted curls [E][nq][nloc][3]
  const void *tab_pts, *tab_phw, *tab_cuw;
  const int *nbr;  // [E][nbr_w]: the elements touching each element (-1 padded)
  int nbr_w;
};

__device__ inline int leaf_local(int ix, int iy, int ka, int kb, int b, int nL1) {
  int mask = (1 << b) - 1;
  return ((ix & mask) + ka) * nL1 + (iy & mask) + kb;
}

__device__ inline void block_add(double2 *B, int nL, int row, int col, double2 v) {
  double2 *dst = B + (size_t)col * nL + row;
  atomicAdd(&dst->x, v.x);
  atomicAdd(&dst->y, v.y);
}

// basis value and d/ds, d/dt of local function k at Gauss point q of element column (ix, iy)
__device__ inline void basis_gp(const NearArgs &A, int ix, int iy, int k, int q, double &v,
                                double &ds, double &dt) {
  int p1 = A.p + 1, ka = k / p1, kb = k % p1, q1 = q / A.ng, q2 = q % A.ng;
  double b1 = A.phi1[(ix * A.ng + q1) * p1 + ka], b2 = A.phi1[(iy * A.ng + q2) * p1 + kb];
  v = b1 * b2;
  ds = A.dphi1[(ix * A.ng + q1) * p1 + ka] * b2;
  dt = b1 * A.dphi1[(iy * A.ng + q2) * p1 + kb];
}

// c_k = d_s psi_k d_t F - d_t psi_k d_s F at Gauss point q of element e
__device__ inline void curl_gp(const NearArgs &A, long iq, double ds, double dt, double c[3]) {
  for (int d = 0; d < 3; ++d)
    c[d] = ds * A.gft[d * A.gstride + iq] - dt * A.gfs[d * A.gstride + iq];
}

// e and f share a point (the pair is integrated by k_near_singular): the neighbour list of e
__device__ inline bool touching(const NearArgs &A, int e, int f) {
  if (e == f) return true;
  for (int c = 0; c < A.nbr_w; ++c)
    if (A.nbr[(long)e * A.nbr_w + c] == f) return true;
  return false;
}

// The per-element tables of the regular quadrature in precision T (one thread per Gauss point):
// they depend on the element alone, so every element pair reads them instead of re-evaluating the
// B-splines and curls.
template <class T>
__global__ void k_elem_tables(NearArgs A, long n_gp, T *__restrict__ pts, T *__restrict__ phw, T *__restrict__ cuw) {
  const int nq = A.ng * A.ng, nloc = A.nloc;
  for (long iq = blockIdx.x * (long)blockDim.x + threadIdx.x; iq < n_gp; iq += (long)gridDim.x * blockDim.x) {
    const long e = iq / nq;
    const int q = (int)(iq % nq), ix = (int)((e / A.n1) % A.n1), iy = (int)(e % A.n1);
    for (int c = 0; c < 3; ++c) {
      pts[iq * 7 + c] = (T)A.gpx[c * A.gstride + iq];
      pts[iq * 7 + 3 + c] = (T)A.gpn[c * A.gstride + iq];
    }
    pts[iq * 7 + 6] = (T)A.gpa[iq];
    const double w = A.gw[q / A.ng] * A.gw[q % A.ng];
    for (int k = 0; k < nloc; ++k) {
      double v, ds, dt;
      basis_gp(A, ix, iy, k, q, v, ds, dt);
      phw[iq * nloc + k] = (T)(v * w);
      if (A.hard) {
        double c[3];
        curl_gp(A, iq, ds, dt, c);
        for (int d = 0; d < 3; ++d) cuw[(iq * nloc + k) * 3 + d] = (T)(c[d] * w);
      }
    }
  }
}

// per-warp scratch of k_near_regular_t, in elements of its precision
__host__ __device__ inline int near_regular_scratch(int nq, int nloc, bool hard) {
  return 2 * nq * 7 + 2 * nq * nloc + 2 * nq * nq + 2 * nq * nloc + (hard ? 6 * nq * nloc + 2 * nq * nq + 6 * nq * nloc : 0);
}

// One block of threads per near leaf pair, one warp per element pair (touching pairs skipped:
// k_near_singular integrates them).  Block entry (k of e, l of f) +=
//   sum_{q,r} w_q w_r h^4 [ks(q,r) psi_k(q) psi_l(r) + gc(q,r) c_k(q) . c_l(r)],
// evaluated in precision T (FP64, or FP32 for the mixed precision set-up), the leaf-pair block summed
// in FP64 in shared memory when it fits (else with global FP64 atomics).
template <class T>
__global__ void k_near_regular_t(NearArgs A, int smem_block) {
  extern __shared__ __align__(16) unsigned char smr[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int nq = A.ng * A.ng, nloc = A.nloc, p1 = A.p + 1;
  // per-warp scratch (T): pts[2][nq][7], phi[2][nq][nloc], ks[nq*nq][2], Tm[nq][nloc][2], and for
  // sound-hard curl[2][nq][nloc][3], gc[nq*nq][2], Tc[3][nq][nloc][2] (near_regular_scratch)
  using BA = typename std::conditional<sizeof(T) == 4, float2, double2>::type;  // leaf-pair block sums
  const int hc = A.hard ? 1 : 0;
  const int per = near_regular_scratch(nq, nloc, A.hard);
  BA *Bs = reinterpret_cast<BA *>(smr);
  T *base = reinterpret_cast<T *>(smr + (smem_block ? (size_t)A.nL * A.nL * sizeof(BA) : 0));
  T *pts = base + warp * per;
  T *phe = pts + 2 * nq * 7, *phf = phe + nq * nloc;
  T *cue = phf + nq * nloc, *cuf = cue + hc * 3 * nq * nloc;
  T *ks = cuf + hc * 3 * nq * nloc, *gc = ks + 2 * nq * nq;
  T *Tm = gc + hc * 2 * nq * nq, *Tc = Tm + 2 * nq * nloc;
  const int bid = blockIdx.x;
  const int tgt = A.near_tgt[bid], src = A.near_src[bid];
  const int nlL = 1 << A.L, ne1 = 1 << A.b;
  const int jt = tgt / (nlL * nlL), cxt = (tgt / nlL) % nlL, cyt = tgt % nlL;
  const int js = src / (nlL * nlL), cxs = (src / nlL) % nlL, cys = src % nlL;
  double2 *Bg = A.blk + (size_t)bid * A.nL * A.nL;
  if (smem_block) {
    for (int i = threadIdx.x; i < A.nL * A.nL; i += blockDim.x) {
      Bs[i].x = 0;
      Bs[i].y = 0;
    }
    __syncthreads();
  }
  const T *tpts = static_cast<const T *>(A.tab_pts), *tphw = static_cast<const T *>(A.tab_phw),
          *tcuw = static_cast<const T *>(A.tab_cuw);
  const T h2 = (T)(A.h * A.h), kap = (T)A.kappa, eta = (T)A.eta;
  const int npair = ne1 * ne1 * ne1 * ne1;
  for (int pr = warp; pr < npair; pr += nwarp) {
    int et = pr / (ne1 * ne1), es = pr % (ne1 * ne1);
    int ixe = cxt * ne1 + et / ne1, iye = cyt * ne1 + et % ne1;
    int ixf = cxs * ne1 + es / ne1, iyf = cys * ne1 + es % ne1;
    int e = (jt * A.n1 + ixe) * A.n1 + iye, f = (js * A.n1 + ixf) * A.n1 + iyf;
    if (touching(A, e, f)) continue;  // warp-uniform
    // stage the Gauss points (x, n~, a) and the weighted basis values / curls of both elements from the
    // element tables
    for (int i = lane; i < 2 * nq * 7; i += 32) {
      const int side = i / (nq * 7), r = i % (nq * 7);
      pts[i] = tpts[(long)(side ? f : e) * nq * 7 + r];
    }
    for (int i = lane; i < 2 * nq * nloc; i += 32) {
      const int side = i / (nq * nloc), r = i % (nq * nloc);
      const long el = side ? f : e;
      (side ? phf : phe)[r] = tphw[el * nq * nloc + r];
      if (A.hard)
        for (int d = 0; d < 3; ++d) (side ? cuf : cue)[r * 3 + d] = tcuw[(el * nq * nloc + r) * 3 + d];
    }
    __syncwarp();
    for (int i = lane; i < nq * nq; i += 32) {
      int q = i / nq, r = i % nq;
      const T *X = pts + q * 7, *Y = pts + (nq + r) * 7;
      PK<T> pk = cfie_kernel_t<T>(A.hard, kap, eta, X, X + 3, X[6], Y, Y + 3, Y[6]);
      ks[2 * i] = pk.ksx * h2 * h2;
      ks[2 * i + 1] = pk.ksy * h2 * h2;
      if (A.hard) {
        gc[2 * i] = pk.gcx * h2 * h2;
        gc[2 * i + 1] = pk.gcy * h2 * h2;
      }
    }
    __syncwarp();
    // Tm[q][l] = sum_r ks[q][r] phi_l(r);  Tc[d][q][l] = sum_r gc[q][r] c_l,d(r)
    for (int i = lane; i < nq * nloc; i += 32) {
      int q = i / nloc, l = i % nloc;
      T tx = 0, ty = 0, c0x = 0, c0y = 0, c1x = 0, c1y = 0, c2x = 0, c2y = 0;
      for (int r = 0; r < nq; ++r) {
        T kx = ks[2 * (q * nq + r)], ky = ks[2 * (q * nq + r) + 1], ph = phf[r * nloc + l];
        tx += kx * ph;
        ty += ky * ph;
        if (A.hard) {
          T gx = gc[2 * (q * nq + r)], gy = gc[2 * (q * nq + r) + 1];
          const T *cl = cuf + (r * nloc + l) * 3;
          c0x += gx * cl[0]; c0y += gy * cl[0];
          c1x += gx * cl[1]; c1y += gy * cl[1];
          c2x += gx * cl[2]; c2y += gy * cl[2];
        }
      }
      Tm[2 * i] = tx;
      Tm[2 * i + 1] = ty;
      if (A.hard) {
        Tc[2 * i] = c0x; Tc[2 * i + 1] = c0y;
        Tc[2 * (nq * nloc + i)] = c1x; Tc[2 * (nq * nloc + i) + 1] = c1y;
        Tc[2 * (2 * nq * nloc + i)] = c2x; Tc[2 * (2 * nq * nloc + i) + 1] = c2y;
      }
    }
    __syncwarp();
    for (int i = lane; i < nloc * nloc; i += 32) {
      int k = i / nloc, l = i % nloc;
      T ax = 0, ay = 0;
      for (int q = 0; q < nq; ++q) {
        T ph = phe[q * nloc + k];
        ax += ph * Tm[2 * (q * nloc + l)];
        ay += ph * Tm[2 * (q * nloc + l) + 1];
        if (A.hard) {
          const T *ck = cue + (q * nloc + k) * 3;
          for (int d = 0; d < 3; ++d) {
            ax += ck[d] * Tc[2 * (d * nq * nloc + q * nloc + l)];
            ay += ck[d] * Tc[2 * (d * nq * nloc + q * nloc + l) + 1];
          }
        }
      }
      int row = leaf_local(ixe, iye, k / p1, k % p1, A.b, A.nL1);
      int col = leaf_local(ixf, iyf, l / p1, l % p1, A.b, A.nL1);
      if (smem_block) {
        BA *dst = Bs + (size_t)col * A.nL + row;
        atomicAdd(&dst->x, ax);
        atomicAdd(&dst->y, ay);
      } else {
        block_add(Bg, A.nL, row, col, cmk((double)ax, (double)ay));
      }
    }
    __syncwarp();
  }
  if (smem_block) {
    __syncthreads();
    for (int i = threadIdx.x; i < A.nL * A.nL; i += blockDim.x) {
      const BA v = Bs[i];
      atomicAdd(&Bg[i].x, (double)v.x);
      atomicAdd(&Bg[i].y, (double)v.y);
    }
  }
}

// per-warp scratch of k_near_regular_f, in elements of its precision (offsets rounded to pairs)
__host__ __device__ inline int near_fused_scratch(int nq, int nl, bool hard) {
  auto al = [](int x) { return (x + 1) & ~1; };
  const int base = al(2 * nq * 7) + al(2 * nq * nl) + (hard ? al(6 * nq * nl) : 0);
  return base + 2 * nq * nl + (hard ? 6 * nq * nl : 0);
}

// Regular element pairs with the kernel samples folded into the first contraction in registers:
// lane (q, half) of a warp evaluates the samples of target Gauss point q against every other source
// point (half selects which) and accumulates Tm[q][l] = sum_r ks(q, r) psi_l(r) (sound-hard also
// Tc[d][q][l] = sum_r gc(q, r) c_l,d(r)) without storing the samples; a shuffle adds the two halves.
// The block entries then contract Tm with the test side's weighted basis values (and curls).  Same
// sums as k_near_regular_t in another order; one block per near leaf pair, one warp per element pair.
template <class T, int NL, bool HARD>
__global__ void k_near_regular_f(NearArgs A, int smem_block) {
  extern __shared__ __align__(16) unsigned char smf[];
  using BA = typename std::conditional<sizeof(T) == 4, float2, double2>::type;  // leaf-pair block sums
  using TV = BA;                                                                  // complex in precision T
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int nq = A.ng * A.ng, p1 = A.p + 1;
  auto al = [](int x) { return (x + 1) & ~1; };
  const int per = near_fused_scratch(nq, NL, HARD);
  BA *Bs = reinterpret_cast<BA *>(smf);
  T *base = reinterpret_cast<T *>(smf + (smem_block ? (size_t)A.nL * A.nL * sizeof(BA) : 0));
  T *pts = base + warp * per;
  T *phe = pts + al(2 * nq * 7), *phf = phe + nq * NL;
  T *cue = phe + al(2 * nq * NL), *cuf = cue + 3 * nq * NL;
  TV *Tm = reinterpret_cast<TV *>(phe + al(2 * nq * NL) + (HARD ? al(6 * nq * NL) : 0));
  TV *Tc = Tm + nq * NL;
  const int bid = blockIdx.x;
  const int tgt = A.near_tgt[bid], src = A.near_src[bid];
  const int nlL = 1 << A.L, ne1 = 1 << A.b;
  const int jt = tgt / (nlL * nlL), cxt = (tgt / nlL) % nlL, cyt = tgt % nlL;
  const int js = src / (nlL * nlL), cxs = (src / nlL) % nlL, cys = src % nlL;
  double2 *Bg = A.blk + (size_t)bid * A.nL * A.nL;
  if (smem_block) {
    for (int i = threadIdx.x; i < A.nL * A.nL; i += blockDim.x) {
      Bs[i].x = 0;
      Bs[i].y = 0;
    }
    __syncthreads();
  }
  const T *tpts = static_cast<const T *>(A.tab_pts), *tphw = static_cast<const T *>(A.tab_phw),
          *tcuw = static_cast<const T *>(A.tab_cuw);
  const T h2 = (T)(A.h * A.h), h4 = h2 * h2, kap = (T)A.kappa, eta = (T)A.eta;
  const int npair = ne1 * ne1 * ne1 * ne1;
  for (int pr = warp; pr < npair; pr += nwarp) {
    int et = pr / (ne1 * ne1), es = pr % (ne1 * ne1);
    int ixe = cxt * ne1 + et / ne1, iye = cyt * ne1 + et % ne1;
    int ixf = cxs * ne1 + es / ne1, iyf = cys * ne1 + es % ne1;
    int e = (jt * A.n1 + ixe) * A.n1 + iye, f = (js * A.n1 + ixf) * A.n1 + iyf;
    if (touching(A, e, f)) continue;  // warp-uniform
    // stage the Gauss points (x, n~, a) and the weighted basis values / curls of both elements
    for (int i = lane; i < 2 * nq * 7; i += 32) {
      const int side = i / (nq * 7), r = i % (nq * 7);
      pts[i] = tpts[(long)(side ? f : e) * nq * 7 + r];
    }
    for (int i = lane; i < 2 * nq * NL; i += 32) {
      const int side = i / (nq * NL), r = i % (nq * NL);
      const long el = side ? f : e;
      (side ? phf : phe)[r] = tphw[el * nq * NL + r];
      if (HARD)
        for (int d = 0; d < 3; ++d) (side ? cuf : cue)[r * 3 + d] = tcuw[(el * nq * NL + r) * 3 + d];
    }
    __syncwarp();
    // samples and the first contraction, 16 target points per pass
    for (int q0 = 0; q0 < nq; q0 += 16) {
      const int q = q0 + (lane & 15), half = lane >> 4;
      TV tm[NL], tc[HARD ? 3 : 1][HARD ? NL : 1];
#pragma unroll
      for (int l = 0; l < NL; ++l) tm[l].x = tm[l].y = (T)0;
      if constexpr (HARD) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int l = 0; l < NL; ++l) tc[d][l].x = tc[d][l].y = (T)0;
      }
      if (q < nq) {
        T xr[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) xr[c] = pts[q * 7 + c];
        for (int r = half; r < nq; r += 2) {
          const T *Y = pts + (nq + r) * 7;
          const PK<T> pk = cfie_kernel_t<T>(HARD, kap, eta, xr, xr + 3, xr[6], Y, Y + 3, Y[6]);
          const T kx = pk.ksx * h4, ky = pk.ksy * h4;
          const T *ph = phf + r * NL;
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            tm[l].x += kx * ph[l];
            tm[l].y += ky * ph[l];
          }
          if constexpr (HARD) {
            const T gx = pk.gcx * h4, gy = pk.gcy * h4;
            const T *cl = cuf + r * NL * 3;
#pragma unroll
            for (int l = 0; l < NL; ++l)
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                tc[d][l].x += gx * cl[l * 3 + d];
                tc[d][l].y += gy * cl[l * 3 + d];
              }
          }
        }
      }
      // lanes q and q + 16 hold the two halves of the same target point
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        tm[l].x += __shfl_xor_sync(0xffffffffu, tm[l].x, 16);
        tm[l].y += __shfl_xor_sync(0xffffffffu, tm[l].y, 16);
      }
      if constexpr (HARD) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            tc[d][l].x += __shfl_xor_sync(0xffffffffu, tc[d][l].x, 16);
            tc[d][l].y += __shfl_xor_sync(0xffffffffu, tc[d][l].y, 16);
          }
      }
      if (half == 0 && q < nq) {
#pragma unroll
        for (int l = 0; l < NL; ++l) Tm[q * NL + l] = tm[l];
        if constexpr (HARD) {
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int l = 0; l < NL; ++l) Tc[(d * nq + q) * NL + l] = tc[d][l];
        }
      }
    }
    __syncwarp();
    for (int i = lane; i < NL * NL; i += 32) {
      const int k = i / NL, l = i % NL;
      T ax = 0, ay = 0;
      for (int q = 0; q < nq; ++q) {
        const T ph = phe[q * NL + k];
        const TV t = Tm[q * NL + l];
        ax += ph * t.x;
        ay += ph * t.y;
        if constexpr (HARD) {
          const T *ck = cue + (q * NL + k) * 3;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const TV c = Tc[(d * nq + q) * NL + l];
            ax += ck[d] * c.x;
            ay += ck[d] * c.y;
          }
        }
      }
      const int row = leaf_local(ixe, iye, k / p1, k % p1, A.b, A.nL1);
      const int col = leaf_local(ixf, iyf, l / p1, l % p1, A.b, A.nL1);
      if (smem_block) {
        BA *dst = Bs + (size_t)col * A.nL + row;
        atomicAdd(&dst->x, ax);
        atomicAdd(&dst->y, ay);
      } else {
        block_add(Bg, A.nL, row, col, cmk((double)ax, (double)ay));
      }
    }
    __syncwarp();
  }
  if (smem_block) {
    __syncthreads();
    for (int i = threadIdx.x; i < A.nL * A.nL; i += blockDim.x) {
      const BA v = Bs[i];
      atomicAdd(&Bg[i].x, (double)v.x);
      atomicAdd(&Bg[i].y, (double)v.y);
    }
  }
}

// ----------------------------------------------------------------------------------------------
// touching element pairs: regularising transforms (identical 8, common edge 6, common vertex 4
// regions) with the canonical position given by the square symmetries (Te, Tf) found on the host.
// For identical pairs the half mass matrix 1/2 M (regular Gauss rule) is added as well.

struct SingArgs {
  NearArgs A;
  const int *sing;        // 7 ints per unordered touching pair
  const double *rule[3];  // per kind: x1, x2, y1, y2, w arrays of n points, concatenated
  int rule_n[3];
  const unsigned char *share[3];  // per kind: sharing tables over chunks of ch points
  int ch, nv, nd, pg1;            // chunk; most distinct coordinates / points of a chunk; max degree + 1
  int ns;                         // Gauss points per transformed variable
  int fact;                       // sum factorisation of the identical pairs' sound-soft blocks
  SingLayout L;                   // shared-memory layout (offsets in doubles)
};

// values of the nloc local functions at local point (u, v) of element column (ix, iy) (Bernstein
// extraction) into val; with curl != nullptr also c_k = d_s psi_k d_t F - d_t psi_k d_s F
__device__ inline void basis_curl_at(const NearArgs &A, int ix, int iy, double u, double v, const double *fs,
                                     const double *ft, double *val, double *curl) {
  const int p = A.p, p1 = p + 1;
  double Bu[8], dBu[8], Bv[8], dBv[8];
  bernstein_all(p, u, Bu, curl ? dBu : nullptr);
  bernstein_all(p, v, Bv, curl ? dBv : nullptr);
  double fu[8], dfu[8], fv[8], dfv[8];
  for (int a = 0; a <= p; ++a) {
    double s0 = 0, s1 = 0, t0 = 0, t1 = 0;
    for (int c = 0; c <= p; ++c) {
      double ea = A.ext1[(ix * p1 + a) * p1 + c], eb = A.ext1[(iy * p1 + a) * p1 + c];
      s0 += ea * Bu[c];
      t0 += eb * Bv[c];
      if (curl) {
        s1 += ea * dBu[c];
        t1 += eb * dBv[c];
      }
    }
    fu[a] = s0; fv[a] = t0; dfu[a] = s1 * A.n1; dfv[a] = t1 * A.n1;
  }
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) {
      const int k = a * p1 + b;
      val[k] = fu[a] * fv[b];
      if (curl) {
        const double ds = dfu[a] * fv[b], dt = fu[a] * dfv[b];
        for (int d = 0; d < 3; ++d) curl[k * 3 + d] = ds * ft[d] - dt * fs[d];
      }
    }
}

constexpr int SING_MAXACC = 19;  // (p+1)^4 / 128 rounded up for p <= 6

// One block per unordered touching pair.  Points of the regularising rule of the pair's kind, mapped
// by the canonical square symmetries; for edge and vertex pairs the same points also give the block
// of (f, e) with the roles of x and y exchanged (the rules are symmetric under that exchange).  The
// rule is taken in chunks of ch points (whole groups of ns^2): (1) the element nets contracted along
// each distinct second coordinate of the chunk, (2) the geometry of each distinct element point,
// (3) the kernel values per point, (4) sums over the points sharing an element point (or, for
// identical sound-soft pairs, the factorised inner sums), (5) the block entries, one per thread.
template <int NSLOT>
__global__ void k_near_singular(SingArgs S) {
  const NearArgs &A = S.A;
  extern __shared__ double smd[];
  const int nloc = A.nloc, p1 = A.p + 1, ch = S.ch, hard = A.hard;
  // shared (SingLayout): (A) the column partials colp[2][nv][pg1][8] of the element geometries, then per
  // point S3[ch][3] (w k(x,y), w k(y,x), w gc) and the basis values psiO[ch][nloc] (and curls) of the side
  // that is not grouped; (B) geo[2][nd][13] (x, d_s x, d_t x, n, |n| of the chunk's distinct points), then
  // per group T, T2 [nd][nloc] and U [nd][nloc][3]; (C) the basis values (and curls) of the grouped
  // side's distinct points; the two element nets
  double *colp = smd;
  double2 *S3 = reinterpret_cast<double2 *>(smd + S.L.s3);
  double *psiO = smd + S.L.psi, *curO = smd + S.L.cur;
  double2 *T = reinterpret_cast<double2 *>(smd + S.L.T), *T2 = reinterpret_cast<double2 *>(smd + S.L.T2);
  double2 *Ug = reinterpret_cast<double2 *>(smd + S.L.U);
  double *geo = smd + S.L.geo, *phiG = smd + S.L.phiG, *curG = smd + S.L.curG;
  double *net_e = smd + S.L.nets, *net_f = net_e + 4 * 49;  // element nets (degree <= 6)
  const int *W = S.sing + 7 * blockIdx.x;
  const int e = W[0], f = W[1], kind = W[2], te = W[3], tf = W[4], blk_ef = W[5], blk_fe = W[6];
  const bool both = blk_fe >= 0;
  const int ri = kind == 0 ? 0 : (kind == 2 ? 1 : 2);
  const int npt = S.rule_n[ri];
  // identical pairs: the first half of the rule with both orientations of every point (the second
  // half is the first with x and y exchanged), accumulated into the same block
  const int nuse = kind == 0 ? npt / 2 : npt;
  const double *R = S.rule[ri];
  const unsigned char *SH = S.share[ri];
  const int hdr = 8 + 10 * ch;  // sing_share_header
  const unsigned char *PI = SH + (size_t)((npt + ch - 1) / ch) * hdr;
  const int n1 = A.n1;
  const int ixe = (e / n1) % n1, iye = e % n1, ixf = (f / n1) % n1, iyf = f % n1;
  const double h4 = A.h * A.h * A.h * A.h;
  double2 acc[NSLOT], accb[NSLOT];
#pragma unroll
  for (int i = 0; i < NSLOT; ++i) acc[i] = accb[i] = cmk(0, 0);
  const int pe1 = A.edeg[2 * e], pe2 = A.edeg[2 * e + 1], pf1 = A.edeg[2 * f], pf2 = A.edeg[2 * f + 1];
  for (int i = threadIdx.x; i < 4 * (pe1 + 1) * (pe2 + 1); i += blockDim.x) net_e[i] = A.ebez[A.eoff[e] + i];
  for (int i = threadIdx.x; i < 4 * (pf1 + 1) * (pf2 + 1); i += blockDim.x) net_f[i] = A.ebez[A.eoff[f] + i];
  // the rule coordinate (0: first, 1: second) that becomes an element's second local coordinate under
  // its square symmetry (rotations by 90 / 270 degrees and the diagonal reflection exchange them)
  const int vse = ((te & 1) != (te >= 4)) ? 0 : 1, vsf = ((tf & 1) != (tf >= 4)) ? 0 : 1;
  __syncthreads();
  for (int c0 = 0; c0 < nuse; c0 += ch) {
    const int cn = min(ch, nuse - c0);
    const unsigned char *H = SH + (size_t)(c0 / ch) * hdr;
    // the side whose points repeat most in this chunk is grouped: sum_t s_t phi_k(x_t) psi_l(y_t) =
    // sum_g phi_k(x_g) sum_{t in g} s_t psi_l(y_t) (grouping by x; by y with the roles exchanged)
    const int gs = H[5] < H[2] ? 1 : 0, ng = H[gs ? 5 : 2];
    // identical pairs, sound-soft: in each group of ns^2 consecutive points (Gauss indices c, d of the
    // last two variables) x = (X1(c), X2(d)) and y = (Y1(c), Y2(d)), and the basis functions are tensor
    // products phi_k = u_k1 v_k2, so sum_t s_t phi_k(x_t) phi_l(y_t) =
    // sum_c u_k1(X1c) u_l1(Y1c) sum_d s(c, d) v_k2(X2d) v_l2(Y2d) (sum factorisation)
    const bool fac = S.fact && kind == 0 && !hard;
    const int ns = S.ns, ns2 = ns * ns, pb = A.p + 1;
    const int ngrp = fac ? (cn + ns2 - 1) / ns2 : 0;
    const unsigned char *goff = H + 6 + 6 * ch + gs * (ch + 1), *gmem = H + 6 + 6 * ch + 2 * (ch + 1) + gs * ch;
    // geometry, step 1: for each distinct second local coordinate v of the chunk and each row i of the
    // net, the row contracted with the Bernstein polynomials of v and their derivatives
    {
      const int nve = H[vse], nvf = H[3 + vsf], re = pe1 + 1, rf = pf1 + 1;
      for (int w = threadIdx.x; w < nve * re + nvf * rf; w += blockDim.x) {
        const bool sf = w >= nve * re;
        const int ww = sf ? w - nve * re : w, rr = sf ? rf : re;
        const int k = ww / rr, i = ww % rr;
        const int ip = c0 + H[6 + (sf ? 3 + vsf : vse) * ch + k];
        double u, v;
        if (sf) d4_apply(tf, R[2 * npt + ip], R[3 * npt + ip], u, v);
        else d4_apply(te, R[ip], R[npt + ip], u, v);
        const int q2 = sf ? pf2 : pe2;
        double B2[8], dB2[8];
        bernstein_all(q2, v, B2, dB2);
        const double *c = (sf ? net_f : net_e) + i * (q2 + 1) * 4;
        double r[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0};
        for (int j = 0; j <= q2; ++j) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            r[kk] += B2[j] * c[4 * j + kk];
            rv[kk] += dB2[j] * c[4 * j + kk];
          }
        }
        double *o = colp + ((size_t)((sf ? S.nv : 0) + k) * S.pg1 + i) * 8;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          o[kk] = r[kk];
          o[4 + kk] = rv[kk];
        }
      }
    }
    __syncthreads();
    // geometry, step 2: each distinct point of the chunk (x, its tangents d_s x, d_t x, the normal
    // n = d_s x ^ d_t x and |n|) from the column partials of its second coordinate; on the grouped side
    // also the basis values (and curls) there
    {
      const int nde = H[2], ndf = H[5];
      for (int w = threadIdx.x; w < nde + ndf; w += blockDim.x) {
        const bool sf = w >= nde;
        const int k = sf ? w - nde : w;
        const int ip = c0 + H[6 + (sf ? 5 : 2) * ch + k];
        double u, v;
        if (sf) d4_apply(tf, R[2 * npt + ip], R[3 * npt + ip], u, v);
        else d4_apply(te, R[ip], R[npt + ip], u, v);
        const int kv = PI[(size_t)ip * 6 + (sf ? 3 + vsf : vse)];
        const int q1 = sf ? pf1 : pe1;
        double B1[8], dB1[8];
        bernstein_all(q1, u, B1, dB1);
        const double *cp = colp + (size_t)((sf ? S.nv : 0) + kv) * S.pg1 * 8;
        double h[4] = {0, 0, 0, 0}, hu[4] = {0, 0, 0, 0}, hv[4] = {0, 0, 0, 0};
        for (int i = 0; i <= q1; ++i) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            h[kk] += B1[i] * cp[i * 8 + kk];
            hu[kk] += dB1[i] * cp[i * 8 + kk];
            hv[kk] += B1[i] * cp[i * 8 + 4 + kk];
          }
        }
        const double iw = 1.0 / h[3];
        double *g = geo + (size_t)((sf ? S.nd : 0) + k) * 13;
        double fs[3], ft[3], nn[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          const double F = h[kk] * iw;
          g[kk] = F;
          fs[kk] = (hu[kk] - F * hu[3]) * iw * n1;
          ft[kk] = (hv[kk] - F * hv[3]) * iw * n1;
          g[3 + kk] = fs[kk];
          g[6 + kk] = ft[kk];
        }
        cross3(fs, ft, nn);
        g[9] = nn[0];
        g[10] = nn[1];
        g[11] = nn[2];
        g[12] = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        if ((int)sf == gs && !fac)
          basis_curl_at(A, sf ? ixf : ixe, sf ? iyf : iye, u, v, fs, ft, phiG + (size_t)k * nloc,
                        hard ? curG + (size_t)k * nloc * 3 : nullptr);
      }
    }
    __syncthreads();
    // per 4-D point: the kernel values times the weight, and the basis values (and curls) of the side
    // that is not grouped
    for (int t = threadIdx.x; t < cn; t += blockDim.x) {
      const int ip = c0 + t;
      double ue, ve, uf, vf;
      d4_apply(te, R[ip], R[npt + ip], ue, ve);
      d4_apply(tf, R[2 * npt + ip], R[3 * npt + ip], uf, vf);
      const double w = R[4 * npt + ip] * h4;
      const double *ge = geo + (size_t)PI[(size_t)ip * 6 + 2] * 13;
      const double *gf = geo + (size_t)(S.nd + PI[(size_t)ip * 6 + 5]) * 13;
      double X[3], Y[3], nx[3], ny[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        X[k] = ge[k]; nx[k] = ge[9 + k];
        Y[k] = gf[k]; ny[k] = gf[9 + k];
      }
      PairKernel pk;
      double2 kyx;
      cfie_kernel_both(hard, A.kappa, A.eta, X, nx, ge[12], Y, ny, gf[12], pk, kyx);
      S3[3 * t] = cscale(pk.ks, w);
      S3[3 * t + 1] = cscale(kyx, w);
      S3[3 * t + 2] = cscale(pk.gc, w);  // gc(y, x) = gc(x, y)
      if (fac) continue;
      const double *go = gs ? ge : gf;
      if (gs) basis_curl_at(A, ixe, iye, ue, ve, go + 3, go + 6, psiO + (size_t)t * nloc,
                            hard ? curO + (size_t)t * nloc * 3 : nullptr);
      else basis_curl_at(A, ixf, iyf, uf, vf, go + 3, go + 6, psiO + (size_t)t * nloc,
                         hard ? curO + (size_t)t * nloc * 3 : nullptr);
    }
    if (fac) {
      // univariate basis values per group: B1[g][w][j][a], w = 0: u_a(X1 at c = j), 1: v_a(X2 at d = j),
      // 2: u_a(Y1 at c = j), 3: v_a(Y2 at d = j)
      for (int w = threadIdx.x; w < ngrp * 4 * ns; w += blockDim.x) {
        const int g = w / (4 * ns), wh = (w / ns) % 4, j = w % ns;
        const int ip = c0 + g * ns2 + ((wh & 1) ? j : j * ns);
        const double u = R[wh * npt + ip];
        const int ix = wh == 0 ? ixe : wh == 1 ? iye : wh == 2 ? ixf : iyf;
        double Bu[8];
        bernstein_all(A.p, u, Bu, nullptr);
        double *o = phiG + ((size_t)(g * 4 + wh) * ns + j) * pb;
        for (int a = 0; a < pb; ++a) {
          double v = 0;
          for (int c = 0; c < pb; ++c) v += A.ext1[(ix * pb + a) * pb + c] * Bu[c];
          o[a] = v;
        }
      }
    }
    __syncthreads();
    // group sums: T[g][i] = sum_{t in g} w k(x_t, y_t) psiO_i(t), T2 the same with k(y, x), and for
    // sound-hard U[g][i] = sum_{t in g} w gc(t) curlO_i(t)
    if (fac) {
      // U[g][c][k2][l2] = sum_d s(c, d) v_k2(X2d) v_l2(Y2d), and U2 with the other orientation
      const int pp = pb * pb;
      for (int w = threadIdx.x; w < ngrp * ns * pp; w += blockDim.x) {
        const int g = w / (ns * pp), c = (w / pp) % ns, k2 = (w % pp) / pb, l2 = w % pb;
        const double *bx2 = phiG + (size_t)(g * 4 + 1) * ns * pb, *by2 = phiG + (size_t)(g * 4 + 3) * ns * pb;
        double2 u1 = cmk(0, 0), u2 = cmk(0, 0);
        for (int d = 0; d < ns; ++d) {
          const int t = g * ns2 + c * ns + d;
          if (t >= cn) break;
          const double fv = bx2[d * pb + k2] * by2[d * pb + l2];
          const double2 s1 = S3[3 * t], s2 = S3[3 * t + 1];
          u1.x = fma(s1.x, fv, u1.x);
          u1.y = fma(s1.y, fv, u1.y);
          u2.x = fma(s2.x, fv, u2.x);
          u2.y = fma(s2.y, fv, u2.y);
        }
        T[w] = u1;
        T2[w] = u2;
      }
    }
    for (int w = threadIdx.x; w < (fac ? 0 : ng * nloc); w += blockDim.x) {
      const int g = w / nloc, i = w % nloc;
      double2 t1 = cmk(0, 0), t2 = cmk(0, 0), u0 = cmk(0, 0), u1 = cmk(0, 0), u2 = cmk(0, 0);
      for (int m = goff[g]; m < goff[g + 1]; ++m) {
        const int t = gmem[m];
        if (t >= cn) break;  // members ascend: the rest lie past the chunk's used points
        const double ps = psiO[t * nloc + i];
        const double2 s1 = S3[3 * t];
        t1.x = fma(s1.x, ps, t1.x);
        t1.y = fma(s1.y, ps, t1.y);
        if (both) {
          const double2 s2 = S3[3 * t + 1];
          t2.x = fma(s2.x, ps, t2.x);
          t2.y = fma(s2.y, ps, t2.y);
        }
        if (hard) {
          const double2 gg = S3[3 * t + 2];
          const double *cu = curO + (t * nloc + i) * 3;
          u0.x = fma(gg.x, cu[0], u0.x); u0.y = fma(gg.y, cu[0], u0.y);
          u1.x = fma(gg.x, cu[1], u1.x); u1.y = fma(gg.y, cu[1], u1.y);
          u2.x = fma(gg.x, cu[2], u2.x); u2.y = fma(gg.y, cu[2], u2.y);
        }
      }
      T[w] = t1;
      T2[w] = t2;
      if (hard) {
        Ug[3 * w] = u0;
        Ug[3 * w + 1] = u1;
        Ug[3 * w + 2] = u2;
      }
    }
    __syncthreads();
    // block entries (k of x, l of y): a += sum_g phiG_kG(g) T[g][kO] (+ curlG . U), kG / kO the entry's
    // index on the grouped / other side
#pragma unroll
    for (int slot = 0; slot < NSLOT; ++slot) {
      const int i = threadIdx.x + slot * blockDim.x;
      if (i >= nloc * nloc) break;
      const int k = i / nloc, l = i % nloc;
      const int kG = gs ? l : k, kO = gs ? k : l;
      double2 a = acc[slot], b = accb[slot];
      if (fac) {
        // a += sum_g sum_c u_k1(X1c) u_l1(Y1c) U[g][c][k2][l2]
        const int k1 = k / pb, k2 = k % pb, l1 = l / pb, l2 = l % pb, pp = pb * pb;
        for (int g = 0; g < ngrp; ++g) {
          const double *bx1 = phiG + (size_t)(g * 4) * ns * pb, *by1 = phiG + (size_t)(g * 4 + 2) * ns * pb;
          for (int c = 0; c < ns; ++c) {
            const double fu = bx1[c * pb + k1] * by1[c * pb + l1];
            const int iu = (g * ns + c) * pp + k2 * pb + l2;
            const double2 u1 = T[iu], u2 = T2[iu];
            a.x = fma(fu, u1.x, a.x);
            a.y = fma(fu, u1.y, a.y);
            b.x = fma(fu, u2.x, b.x);
            b.y = fma(fu, u2.y, b.y);
          }
        }
      } else if (hard) {
        for (int g = 0; g < ng; ++g) {
          const double ph = phiG[g * nloc + kG];
          const double *cg = curG + (g * nloc + kG) * 3;
          const double2 *uu = Ug + 3 * (g * nloc + kO);
          const double2 tt = T[g * nloc + kO];
          double2 d;
          d.x = fma(cg[0], uu[0].x, fma(cg[1], uu[1].x, cg[2] * uu[2].x));
          d.y = fma(cg[0], uu[0].y, fma(cg[1], uu[1].y, cg[2] * uu[2].y));
          a.x = fma(ph, tt.x, a.x + d.x);
          a.y = fma(ph, tt.y, a.y + d.y);
          if (both) {
            const double2 t2 = T2[g * nloc + kO];
            b.x = fma(ph, t2.x, b.x + d.x);
            b.y = fma(ph, t2.y, b.y + d.y);
          }
        }
      } else if (both) {
        for (int g = 0; g < ng; ++g) {
          const double ph = phiG[g * nloc + kG];
          const double2 tt = T[g * nloc + kO], t2 = T2[g * nloc + kO];
          a.x = fma(ph, tt.x, a.x);
          a.y = fma(ph, tt.y, a.y);
          b.x = fma(ph, t2.x, b.x);
          b.y = fma(ph, t2.y, b.y);
        }
      } else {
        for (int g = 0; g < ng; ++g) {
          const double ph = phiG[g * nloc + kG];
          const double2 tt = T[g * nloc + kO];
          a.x = fma(ph, tt.x, a.x);
          a.y = fma(ph, tt.y, a.y);
        }
      }
      acc[slot] = a;
      accb[slot] = b;
    }
    __syncthreads();
  }
  const int nq = A.ng * A.ng;
#pragma unroll
  for (int slot = 0; slot < NSLOT; ++slot) {
    const int i = threadIdx.x + slot * blockDim.x;
    if (i >= nloc * nloc) break;
    const int k = i / nloc, l = i % nloc;
    double2 a = acc[slot];
    if (kind == 0) {  // + 1/2 M_kl = 1/2 sum_q w_q h^2 a_q psi_k psi_l
      double m = 0;
      for (int q = 0; q < nq; ++q) {
        double vk, vl, d1, d2;
        basis_gp(A, ixe, iye, k, q, vk, d1, d2);
        basis_gp(A, ixe, iye, l, q, vl, d1, d2);
        m += A.gw[q / A.ng] * A.gw[q % A.ng] * A.gpa[(long)e * nq + q] * vk * vl;
      }
      a.x += 0.5 * m * A.h * A.h;
    }
    const int re = leaf_local(ixe, iye, k / p1, k % p1, A.b, A.nL1);
    const int cf = leaf_local(ixf, iyf, l / p1, l % p1, A.b, A.nL1);
    block_add(A.blk + (size_t)blk_ef * A.nL * A.nL, A.nL, re, cf, a);
    if (both) block_add(A.blk + (size_t)blk_fe * A.nL * A.nL, A.nL, cf, re, accb[slot]);
  }
}

// ----------------------------------------------------------------------------------------------
// launchers

void launch_gauss_geometry(const DeviceProblem &d, const HostSetup &S, cudaStream_t st) {
  Phase ph(d.prof, IGABEM_PH_SETUP_TABLES, st);
  long tot = (long)S.E * S.ng * S.ng;
  int grid = (int)std::min<long>((tot + 255) / 256, 152L * 16);
  k_gauss_geometry<<<grid, 256, 0, st>>>(d.edeg, d.eoff, d.ebez, d.gx, S.E, S.ng, (double)S.n1,
                                         d.gpx, d.gpn, d.gpa, d.gfs, d.gft);
  note_launch();
}

void launch_node_geometry(const DeviceProblem &d, const HostSetup &S, cudaStream_t st) {
  Phase ph(d.prof, IGABEM_PH_SETUP_TABLES, st);
  for (int l = 0; l <= S.L; ++l) {
    const int q = S.lev[l].q;
    long tot = (long)S.lev[l].n * q * q;
    int grid = (int)std::min<long>((tot + 255) / 256, 152L * 16);
    k_node_geometry<<<grid, 256, 0, st>>>(d.edeg, d.eoff, d.ebez, d.chebl[l], d.centers[l], S.lev[l].n, l, q,
                                          S.n1, d.nodes[l], d.nodes32[l]);
    note_launch();
  }
}

static NearArgs near_args(const DeviceProblem &d, const HostSetup &S, const igabem_options &o) {
  NearArgs A;
  A.gpx = d.gpx; A.gpn = d.gpn; A.gpa = d.gpa; A.gfs = d.gfs; A.gft = d.gft;
  A.phi1 = d.phi1; A.dphi1 = d.dphi1; A.ext1 = d.ext1; A.gw = d.gw; A.corners = d.corners;
  A.edeg = d.edeg; A.eoff = d.eoff; A.ebez = d.ebez;
  A.near_tgt = d.near_tgt; A.near_src = d.near_src;
  A.gstride = (long)S.E * S.ng * S.ng;
  A.n1 = S.n1; A.ng = S.ng; A.p = S.p; A.nloc = S.nloc; A.b = S.b; A.nL1 = S.nL1; A.nL = S.nL;
  A.L = S.L; A.h = S.h; A.kappa = o.kappa; A.eta = o.eta_cfie; A.tol = 1e-10 * S.scale;
  A.hard = S.hard;
  A.blk = reinterpret_cast<double2 *>(d.blk);
  A.tab_pts = A.tab_phw = A.tab_cuw = nullptr;
  A.nbr = d.nbr;
  A.nbr_w = S.nbr_w;
  return A;
}

size_t near_table_bytes(const HostSetup &S, const igabem_options &o) {
  const size_t tsz = o.precision != IGABEM_FP64 ? sizeof(float) : sizeof(double);
  const size_t ngp = (size_t)S.E * S.ng * S.ng;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(ngp * 7 * tsz) + al(ngp * S.nloc * tsz) + (S.hard ? al(ngp * S.nloc * 3 * tsz) : 0);
}

void launch_near_field(const DeviceProblem &d, const HostSetup &S, const igabem_options &o,
                       cudaStream_t st) {
  NearArgs A = near_args(d, S, o);
  int nblk = (int)S.near_src.size();
  if (nblk > 0) {
    Phase ph(d.prof, IGABEM_PH_SETUP_NEAR, st);
    const int nq = S.ng * S.ng, nloc = S.nloc;
    const bool f32 = o.precision != IGABEM_FP64;
    const size_t tsz = f32 ? sizeof(float) : sizeof(double);
    // the element tables, in the scratch buffer given with the problem (near_table_bytes)
    {
      const long ngp = (long)S.E * nq;
      auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
      uint8_t *tb = static_cast<uint8_t *>(d.near_tab);
      A.tab_pts = tb;
      A.tab_phw = tb + al(ngp * 7 * tsz);
      A.tab_cuw = tb + al(ngp * 7 * tsz) + al(ngp * nloc * tsz);
      const int grid = (int)std::min<long>((ngp + 255) / 256, 152L * 16);
      if (f32)
        k_elem_tables<float><<<grid, 256, 0, st>>>(A, ngp, (float *)A.tab_pts, (float *)A.tab_phw, (float *)A.tab_cuw);
      else
        k_elem_tables<double><<<grid, 256, 0, st>>>(A, ngp, (double *)A.tab_pts, (double *)A.tab_phw,
                                                    (double *)A.tab_cuw);
      note_launch();
    }
    // the fused kernel keeps Tm (and Tc) in registers: p <= 2, and p = 3 for sound-soft
    const bool fused = nloc == 4 || nloc == 9 || (nloc == 16 && !S.hard);
    const size_t per = (size_t)(fused ? near_fused_scratch(nq, nloc, S.hard) : near_regular_scratch(nq, nloc, S.hard)) * tsz;
    const size_t bsm = (size_t)S.nL * S.nL * 2 * tsz;
    const int smem_block = bsm <= 48 * 1024 ? 1 : 0;
    int warps = 8;
    while (warps > 1 && per * warps + (smem_block ? bsm : 0) > 200 * 1024) warps /= 2;
    size_t smem = per * warps + (smem_block ? bsm : 0);
    auto go = [&](auto kfn) {
      IGA_CUDA(set_max_dynamic_smem(kfn, smem));
      kfn<<<nblk, 32 * warps, smem, st>>>(A, smem_block);
    };
    if (fused) {
      const bool h = S.hard;
      if (f32) {
        if (nloc == 4) h ? go(k_near_regular_f<float, 4, true>) : go(k_near_regular_f<float, 4, false>);
        else if (nloc == 9) h ? go(k_near_regular_f<float, 9, true>) : go(k_near_regular_f<float, 9, false>);
        else go(k_near_regular_f<float, 16, false>);
      } else {
        if (nloc == 4) h ? go(k_near_regular_f<double, 4, true>) : go(k_near_regular_f<double, 4, false>);
        else if (nloc == 9) h ? go(k_near_regular_f<double, 9, true>) : go(k_near_regular_f<double, 9, false>);
        else go(k_near_regular_f<double, 16, false>);
      }
    } else if (f32) {
      IGA_CUDA(set_max_dynamic_smem(k_near_regular_t<float>, smem));
      k_near_regular_t<float><<<nblk, 32 * warps, smem, st>>>(A, smem_block);
    } else {
      IGA_CUDA(set_max_dynamic_smem(k_near_regular_t<double>, smem));
      k_near_regular_t<double><<<nblk, 32 * warps, smem, st>>>(A, smem_block);
    }
    note_launch();
    IGA_CUDA(cudaGetLastError());
  }
  Phase ph(d.prof, IGABEM_PH_SETUP_SINGULAR, st);
  SingArgs SA;
  SA.A = A;
  SA.sing = d.sing;
  for (int k = 0; k < 3; ++k) {
    SA.rule[k] = d.rule[k];
    SA.rule_n[k] = d.rule_n[k];
  }
  const int nsing = (int)S.sing.size() / 7;
  if (S.nloc * S.nloc > SING_MAXACC * 128) fail(IGABEM_EINVAL, "degree_p too large for the singular kernel");
  int pg1 = 1;
  for (size_t i = 0; i < S.edeg.size(); ++i) pg1 = std::max(pg1, S.edeg[i] + 1);
  SA.ch = S.sing_ch;
  SA.nv = S.sing_nv;
  SA.nd = S.sing_nd;
  SA.pg1 = pg1;
  for (int k = 0; k < 3; ++k) SA.share[k] = d.share[k];
  SA.L = sing_layout(S.sing_ch, S.nloc, S.hard, S.sing_nv, S.sing_nd, pg1);
  SA.ns = S.ns;
  SA.fact = S.sing_fact ? 1 : 0;
  const size_t smem = (size_t)SA.L.total * sizeof(double);
  if (smem > 227 * 1024) fail(IGABEM_EINVAL, "gauss_singular and degree_p too large for the singular kernel");
  const int nslot = (S.nloc * S.nloc + 127) / 128;
  auto go = [&](auto kfn) {
    IGA_CUDA(set_max_dynamic_smem(kfn, smem));
    kfn<<<nsing, 128, smem, st>>>(SA);
  };
  if (nslot <= 1) go(k_near_singular<1>);
  else if (nslot <= 2) go(k_near_singular<2>);
  else if (nslot <= 5) go(k_near_singular<5>);
  else if (nslot <= 11) go(k_near_singular<11>);
  else go(k_near_singular<SING_MAXACC>);
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

}  // namespace igabem
