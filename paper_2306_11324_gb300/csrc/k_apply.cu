// Application of the discretised CFIE operator: near-field block SpMV plus the interpolation fast
// multipole method on the reference domain (Sec. 4.4): leaf moments (P2M), upward transfers (M2M),
// coupling of admissible cluster pairs with kernel samples generated on the fly (M2L), downward
// transfers (L2L), evaluation and testing at the Gauss points (L2P).
#include <algorithm>

#include "internal.h"
#include "k_common.cuh"
#include "kernels.h"

namespace igabem {

namespace {

struct Dims {
  int np, m, n1, p, nb, b, L, q, Q, nL1, nL, ng, nq, C, R, CR;
  long NX, N, E;
  double h, kappa, eta;
  bool hard;
};

Dims dims(const HostSetup &S, const igabem_options &o, int R) {
  Dims D;
  D.np = S.np; D.m = S.m; D.n1 = S.n1; D.p = S.p; D.nb = S.nb; D.b = S.b; D.L = S.L; D.q = S.q;
  D.Q = S.q * S.q; D.nL1 = S.nL1; D.nL = S.nL; D.ng = S.ng; D.nq = S.ng * S.ng;
  D.C = S.hard ? 7 : 1; D.R = R; D.CR = D.C * R;
  D.NX = S.NX; D.N = S.N; D.E = S.E; D.h = S.h; D.kappa = o.kappa; D.eta = o.eta_cfie;
  D.hard = S.hard;
  return D;
}

inline int grid_for(long n, int block = 256) {
  return (int)std::max<long>(1, std::min<long>((n + block - 1) / block, 152L * 32));
}

#define GRID_STRIDE(i, n) \
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

// x_X[X][r] = x[x2g[X]][r]
__global__ void k_gather_in(Dims D, const int *__restrict__ x2g, const double2 *__restrict__ x,
                            double2 *__restrict__ xX) {
  GRID_STRIDE(i, D.NX * D.R) {
    long X = i / D.R;
    int r = int(i % D.R);
    xX[i] = x[(long)x2g[X] * D.R + r];
  }
}

__device__ inline long xindex(const Dims &D, int j, int i1, int i2) {
  return ((long)j * D.nb + i1) * D.nb + i2;
}

struct Tables {
  const double *phi1, *dphi1, *gw, *LG1, *T1;
  const double *gpn, *gfs, *gft;  // Gauss-point geometry (SoA, stride E*nq)
};

// P2M: xhat[t][a][c][r] = sum_{e in t, q} L_a(q) f_c(q), with the channel fields (weighted by
// w_q h^2) of u = sum_l x_l psi_l:  soft c0 = u;  hard c0 = u, c1..3 = d_s u d_t F - d_t u d_s F,
// c4..6 = n~ u.
__global__ void k_p2m(Dims D, Tables T, const double2 *__restrict__ xX, double2 *__restrict__ xhat) {
  const int nlL = 1 << D.L, e1 = 1 << D.b, p1 = D.p + 1;
  const long nleaf = (long)D.np * nlL * nlL;
  const long gst = D.E * D.nq;
  GRID_STRIDE(o, nleaf * D.Q * D.CR) {
    long t = o / (D.Q * D.CR);
    int a = int((o / D.CR) % D.Q), cr = int(o % D.CR), c = cr / D.R, r = cr % D.R;
    int j = int(t / (nlL * nlL)), cx = int((t / nlL) % nlL), cy = int(t % nlL);
    int a1 = a / D.q, a2 = a % D.q;
    double2 acc = cmk(0, 0);
    for (int ox = 0; ox < e1; ++ox)
      for (int oy = 0; oy < e1; ++oy) {
        int ix = cx * e1 + ox, iy = cy * e1 + oy;
        long e = ((long)j * D.n1 + ix) * D.n1 + iy;
        for (int q1 = 0; q1 < D.ng; ++q1)
          for (int q2 = 0; q2 < D.ng; ++q2) {
            double Lq = T.LG1[(ox * D.ng + q1) * D.q + a1] * T.LG1[(oy * D.ng + q2) * D.q + a2];
            double W = T.gw[q1] * T.gw[q2] * D.h * D.h * Lq;
            double2 u = cmk(0, 0), us = cmk(0, 0), ut = cmk(0, 0);
            for (int ka = 0; ka < p1; ++ka) {
              double bs = T.phi1[(ix * D.ng + q1) * p1 + ka], ds = T.dphi1[(ix * D.ng + q1) * p1 + ka];
              for (int kb = 0; kb < p1; ++kb) {
                double bt = T.phi1[(iy * D.ng + q2) * p1 + kb], dt = T.dphi1[(iy * D.ng + q2) * p1 + kb];
                double2 xv = xX[xindex(D, j, ix + ka, iy + kb) * D.R + r];
                u = cadd(u, cscale(xv, bs * bt));
                if (c >= 1 && c <= 3) {
                  us = cadd(us, cscale(xv, ds * bt));
                  ut = cadd(ut, cscale(xv, bs * dt));
                }
              }
            }
            long iq = e * D.nq + q1 * D.ng + q2;
            double2 f;
            if (c == 0) {
              f = u;
            } else if (c <= 3) {
              int d = c - 1;
              f = csub(cscale(us, T.gft[d * gst + iq]), cscale(ut, T.gfs[d * gst + iq]));
            } else {
              f = cscale(u, T.gpn[(c - 4) * gst + iq]);
            }
            acc = cadd(acc, cscale(f, W));
          }
      }
    xhat[o] = acc;
  }
}

// M2M from level l+1 to level l: xhat_l[t][a][cr] = sum_children sum_b T(c, a, b) xhat_{l+1}[b]
__global__ void k_m2m(Dims D, int l, const double *__restrict__ T1, const double2 *__restrict__ child,
                      double2 *__restrict__ parent) {
  const int nl = 1 << l, nc = 2 * nl;
  const long n = (long)D.np * nl * nl;
  GRID_STRIDE(o, n * D.Q * D.CR) {
    long t = o / (D.Q * D.CR);
    int a = int((o / D.CR) % D.Q), cr = int(o % D.CR);
    int j = int(t / (nl * nl)), cx = int((t / nl) % nl), cy = int(t % nl);
    int a1 = a / D.q, a2 = a % D.q;
    double2 acc = cmk(0, 0);
    for (int c1 = 0; c1 < 2; ++c1)
      for (int c2 = 0; c2 < 2; ++c2) {
        long tc = ((long)j * nc + 2 * cx + c1) * nc + 2 * cy + c2;
        const double2 *src = child + tc * D.Q * D.CR;
        for (int b1 = 0; b1 < D.q; ++b1) {
          double t1 = T1[(c1 * D.q + a1) * D.q + b1];
          for (int b2 = 0; b2 < D.q; ++b2)
            acc = cadd(acc, cscale(src[(b1 * D.q + b2) * D.CR + cr], t1 * T1[(c2 * D.q + a2) * D.q + b2]));
        }
      }
    parent[o] = acc;
  }
}

// L2L from level l to level l+1: yhat_{l+1}[t][b][cr] += sum_a T(c, a, b) yhat_l[parent][a][cr]
__global__ void k_l2l(Dims D, int l, const double *__restrict__ T1, const double2 *__restrict__ parent,
                      double2 *__restrict__ child) {
  const int nc = 2 << l, nl = 1 << l;
  const long n = (long)D.np * nc * nc;
  GRID_STRIDE(o, n * D.Q * D.CR) {
    long t = o / (D.Q * D.CR);
    int b = int((o / D.CR) % D.Q), cr = int(o % D.CR);
    int j = int(t / (nc * nc)), x = int((t / nc) % nc), y = int(t % nc);
    int c1 = x & 1, c2 = y & 1;
    long tp = ((long)j * nl + (x >> 1)) * nl + (y >> 1);
    int b1 = b / D.q, b2 = b % D.q;
    const double2 *src = parent + tp * D.Q * D.CR;
    double2 acc = child[o];
    for (int a1 = 0; a1 < D.q; ++a1) {
      double t1 = T1[(c1 * D.q + a1) * D.q + b1];
      for (int a2 = 0; a2 < D.q; ++a2)
        acc = cadd(acc, cscale(src[(a1 * D.q + a2) * D.CR + cr], t1 * T1[(c2 * D.q + a2) * D.q + b2]));
    }
    child[o] = acc;
  }
}

// M2M and L2L for many columns with the separable transfer T(c, a, b) = T1(c1, a1, b1) T1(c2, a2, b2)
// (tensor Chebyshev interpolation, Sec. 4.4): the two 1-D contractions one after the other through
// shared memory, in precision T (FP32 for the mixed precisions), one block per (parent, 32 columns).
template <class T> struct CV;
template <> struct CV<float> { using type = float2; };
template <> struct CV<double> { using type = double2; };
constexpr int SEP_COLS = 32;

template <class T>
__global__ void __launch_bounds__(256) k_m2m_sep(Dims D, int l, const double *__restrict__ T1,
                                                 const double2 *__restrict__ child, double2 *__restrict__ parent) {
  using V = typename CV<T>::type;
  extern __shared__ __align__(16) unsigned char smx[];
  V *X = reinterpret_cast<V *>(smx);  // [b1][b2][col]
  V *Z = X + D.Q * SEP_COLS;          // [b1][a2][col]
  __shared__ T Ts[2 * 16 * 16];
  const int q = D.q, Q = q * q, CR = D.CR;
  const int t = blockIdx.x, c0 = blockIdx.y * SEP_COLS, cw = min(SEP_COLS, CR - c0);
  const int nl = 1 << l, nc = 2 * nl;
  const int j = t / (nl * nl), cx = (t / nl) % nl, cy = t % nl;
  for (int i = threadIdx.x; i < 2 * q * q; i += blockDim.x) Ts[i] = (T)T1[i];
  V acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k].x = acc[k].y = 0;
  for (int ch = 0; ch < 4; ++ch) {
    const int c1 = ch >> 1, c2 = ch & 1;
    const long tc = ((long)j * nc + 2 * cx + c1) * nc + 2 * cy + c2;
    __syncthreads();
    for (int i = threadIdx.x; i < Q * SEP_COLS; i += blockDim.x) {
      const int b = i / SEP_COLS, col = i % SEP_COLS;
      V v;
      v.x = v.y = 0;
      if (col < cw) {
        const double2 x = child[(tc * Q + b) * CR + c0 + col];
        v.x = (T)x.x;
        v.y = (T)x.y;
      }
      X[i] = v;
    }
    __syncthreads();
    // second direction: Z[b1][a2][col] = sum_b2 T(c2, a2, b2) X[b1][b2][col]
    for (int i = threadIdx.x; i < Q * SEP_COLS; i += blockDim.x) {
      const int b1 = i / (q * SEP_COLS), a2 = (i / SEP_COLS) % q, col = i % SEP_COLS;
      V sum;
      sum.x = sum.y = 0;
      for (int b2 = 0; b2 < q; ++b2) {
        const T w = Ts[(c2 * q + a2) * q + b2];
        const V x = X[(b1 * q + b2) * SEP_COLS + col];
        sum.x += w * x.x;
        sum.y += w * x.y;
      }
      Z[i] = sum;
    }
    __syncthreads();
    // first direction into the parent: acc[a1][a2][col] += sum_b1 T(c1, a1, b1) Z[b1][a2][col]
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = threadIdx.x + 256 * k;
      if (i >= Q * SEP_COLS) continue;
      const int a = i / SEP_COLS, col = i % SEP_COLS, a1 = a / q, a2 = a % q;
      for (int b1 = 0; b1 < q; ++b1) {
        const T w = Ts[(c1 * q + a1) * q + b1];
        const V x = Z[(b1 * q + a2) * SEP_COLS + col];
        acc[k].x += w * x.x;
        acc[k].y += w * x.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = threadIdx.x + 256 * k;
    if (i >= Q * SEP_COLS) continue;
    const int a = i / SEP_COLS, col = i % SEP_COLS;
    if (col < cw) parent[((long)t * Q + a) * CR + c0 + col] = make_double2((double)acc[k].x, (double)acc[k].y);
  }
}

// L2L: yhat_child[b][cr] += sum_a T(c, a, b) yhat_parent[a][cr] for the four children of the block's
// parent t on level l.
template <class T>
__global__ void __launch_bounds__(256) k_l2l_sep(Dims D, int l, const double *__restrict__ T1,
                                                 const double2 *__restrict__ parent, double2 *__restrict__ child) {
  using V = typename CV<T>::type;
  extern __shared__ __align__(16) unsigned char smy[];
  const int q = D.q, Q = q * q, CR = D.CR;
  V *P = reinterpret_cast<V *>(smy);  // [a1][a2][col]
  V *U = P + Q * SEP_COLS;            // [c2][a1][b2][col]
  __shared__ T Ts[2 * 16 * 16];
  const int t = blockIdx.x, c0 = blockIdx.y * SEP_COLS, cw = min(SEP_COLS, CR - c0);
  const int nl = 1 << l, nc = 2 * nl;
  const int j = t / (nl * nl), cx = (t / nl) % nl, cy = t % nl;
  for (int i = threadIdx.x; i < 2 * q * q; i += blockDim.x) Ts[i] = (T)T1[i];
  for (int i = threadIdx.x; i < Q * SEP_COLS; i += blockDim.x) {
    const int a = i / SEP_COLS, col = i % SEP_COLS;
    V v;
    v.x = v.y = 0;
    if (col < cw) {
      const double2 y = parent[((long)t * Q + a) * CR + c0 + col];
      v.x = (T)y.x;
      v.y = (T)y.y;
    }
    P[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * Q * SEP_COLS; i += blockDim.x) {
    const int c2 = i / (Q * SEP_COLS), r = i % (Q * SEP_COLS), a1 = r / (q * SEP_COLS), b2 = (r / SEP_COLS) % q,
              col = r % SEP_COLS;
    V sum;
    sum.x = sum.y = 0;
    for (int a2 = 0; a2 < q; ++a2) {
      const T w = Ts[(c2 * q + a2) * q + b2];
      const V v = P[(a1 * q + a2) * SEP_COLS + col];
      sum.x += w * v.x;
      sum.y += w * v.y;
    }
    U[i] = sum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * Q * SEP_COLS; i += blockDim.x) {
    const int ch = i / (Q * SEP_COLS), r = i % (Q * SEP_COLS), b = r / SEP_COLS, col = r % SEP_COLS;
    if (col >= cw) continue;
    const int c1 = ch >> 1, c2 = ch & 1, b1 = b / q, b2 = b % q;
    V sum;
    sum.x = sum.y = 0;
    for (int a1 = 0; a1 < q; ++a1) {
      const T w = Ts[(c1 * q + a1) * q + b1];
      const V u = U[((c2 * q + a1) * q + b2) * SEP_COLS + col];
      sum.x += w * u.x;
      sum.y += w * u.y;
    }
    const long tc = ((long)j * nc + 2 * cx + c1) * nc + 2 * cy + c2;
    double2 *dst = child + (tc * Q + b) * CR + c0 + col;
    *dst = make_double2(dst->x + (double)sum.x, dst->y + (double)sum.y);
  }
}

// M2L on level l: yhat[t][a][cr] = sum_{s in far(t)} sum_b S_ts(a, b) xhat[s][b][cr], with the kernel
// samples between the Chebyshev nodes generated on the fly:
//   soft: S = a_y G'(r)/r (x-y).n~_x - i eta a_x a_y G      (pull-back of K' - i eta V)
//   hard: channel 0: S = a_x G'(r)/r (y-x).n~_y  (pull-back of K);  channels 1..6: S = G.
constexpr int M2L_BT = 16;   // source nodes per tile
constexpr int M2L_MO = 4;    // outputs per thread

__global__ void k_m2l(Dims D, int ncl, const int *__restrict__ far_ptr, const int *__restrict__ far_src,
                      const double *__restrict__ nodes, const double2 *__restrict__ xhat,
                      double2 *__restrict__ yhat, int crc) {
  extern __shared__ double2 smem[];
  const int t = blockIdx.x;
  const int cr0 = blockIdx.y * crc, ncr = min(crc, D.CR - cr0);
  if (ncr <= 0) return;
  const int ntypes = D.hard ? 2 : 1;
  double2 *S = smem;                                   // [ntypes][Q][BT]
  double2 *Xs = S + ntypes * D.Q * M2L_BT;             // [BT][crc]
  const long NQ = (long)ncl * D.Q;
  double2 acc[M2L_MO];
  for (int k = 0; k < M2L_MO; ++k) acc[k] = cmk(0, 0);
  const int nout = D.Q * ncr;
  for (int k = far_ptr[t]; k < far_ptr[t + 1]; ++k) {
    const int s = far_src[k];
    for (int b0 = 0; b0 < D.Q; b0 += M2L_BT) {
      const int nbt = min(M2L_BT, D.Q - b0);
      for (int i = threadIdx.x; i < D.Q * nbt; i += blockDim.x) {
        int a = i / nbt, bb = i % nbt;
        long ia = (long)t * D.Q + a, ib = (long)s * D.Q + b0 + bb;
        double x[3] = {nodes[ia], nodes[NQ + ia], nodes[2 * NQ + ia]};
        double y[3] = {nodes[ib], nodes[NQ + ib], nodes[2 * NQ + ib]};
        double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        KernelVals kv = helmholtz(D.kappa, r);
        double ax = nodes[6 * NQ + ia], ay = nodes[6 * NQ + ib];
        if (!D.hard) {
          double dn = d[0] * nodes[3 * NQ + ia] + d[1] * nodes[4 * NQ + ia] + d[2] * nodes[5 * NQ + ia];
          double2 kp = cscale(kv.dGr, ay * dn), v = cscale(kv.G, ax * ay);
          S[a * M2L_BT + bb] = cmk(kp.x + D.eta * v.y, kp.y - D.eta * v.x);
        } else {
          double dn = -(d[0] * nodes[3 * NQ + ib] + d[1] * nodes[4 * NQ + ib] + d[2] * nodes[5 * NQ + ib]);
          S[a * M2L_BT + bb] = cscale(kv.dGr, ax * dn);
          S[D.Q * M2L_BT + a * M2L_BT + bb] = kv.G;
        }
      }
      for (int i = threadIdx.x; i < nbt * ncr; i += blockDim.x) {
        int bb = i / ncr, c = i % ncr;
        Xs[bb * crc + c] = xhat[((long)s * D.Q + b0 + bb) * D.CR + cr0 + c];
      }
      __syncthreads();
      for (int k2 = 0; k2 < M2L_MO; ++k2) {
        int o = threadIdx.x + k2 * blockDim.x;
        if (o >= nout) break;
        int a = o / ncr, c = o % ncr;
        int type = (D.hard && (cr0 + c) / D.R >= 1) ? 1 : 0;
        const double2 *Sr = S + type * D.Q * M2L_BT + a * M2L_BT;
        double2 v = acc[k2];
        for (int bb = 0; bb < nbt; ++bb) v = cadd(v, cmul(Sr[bb], Xs[bb * crc + c]));
        acc[k2] = v;
      }
      __syncthreads();
    }
  }
  for (int k2 = 0; k2 < M2L_MO; ++k2) {
    int o = threadIdx.x + k2 * blockDim.x;
    if (o >= nout) break;
    int a = o / ncr, c = o % ncr;
    yhat[((long)t * D.Q + a) * D.CR + cr0 + c] = acc[k2];
  }
}

// L2P, step 1: channel values at the Gauss points, g[e][q][cr] = sum_a L_a(q) yhat_leaf[a][cr]
__global__ void k_l2p_eval(Dims D, Tables T, const double2 *__restrict__ yhat, double2 *__restrict__ g) {
  const int nlL = 1 << D.L, e1 = 1 << D.b;
  GRID_STRIDE(o, D.E * D.nq * D.CR) {
    long e = o / (D.nq * D.CR);
    int q = int((o / D.CR) % D.nq), cr = int(o % D.CR);
    int j = int(e / (D.n1 * D.n1)), ix = int((e / D.n1) % D.n1), iy = int(e % D.n1);
    long t = ((long)j * nlL + (ix >> D.b)) * nlL + (iy >> D.b);
    int ox = ix & (e1 - 1), oy = iy & (e1 - 1), q1 = q / D.ng, q2 = q % D.ng;
    const double2 *src = yhat + t * D.Q * D.CR;
    double2 acc = cmk(0, 0);
    for (int a1 = 0; a1 < D.q; ++a1) {
      double l1 = T.LG1[(ox * D.ng + q1) * D.q + a1];
      for (int a2 = 0; a2 < D.q; ++a2)
        acc = cadd(acc, cscale(src[(a1 * D.q + a2) * D.CR + cr], l1 * T.LG1[(oy * D.ng + q2) * D.q + a2]));
    }
    g[o] = acc;
  }
}

// L2P, step 2: test against the leaf-local functions and add to y_leaf:
//   soft: y_i += sum_q w_q h^2 psi_i(q) g0(q)
//   hard: y_i += sum_q w_q h^2 [-psi_i g0 - i eta (c_i . g_curl - kappa^2 psi_i n~ . g_n)]
__global__ void k_l2p_test(Dims D, Tables T, const double2 *__restrict__ g, double2 *__restrict__ yleaf) {
  const int nlL = 1 << D.L, e1 = 1 << D.b, p1 = D.p + 1;
  const long nleaf = (long)D.np * nlL * nlL;
  const long gst = D.E * D.nq;
  GRID_STRIDE(o, nleaf * D.nL * D.R) {
    long t = o / (D.nL * D.R);
    int i = int((o / D.R) % D.nL), r = int(o % D.R);
    int j = int(t / (nlL * nlL)), cx = int((t / nlL) % nlL), cy = int(t % nlL);
    int i1 = cx * e1 + i / D.nL1, i2 = cy * e1 + i % D.nL1;
    double2 acc = cmk(0, 0);
    for (int ix = max(cx * e1, i1 - D.p); ix <= min(cx * e1 + e1 - 1, i1); ++ix)
      for (int iy = max(cy * e1, i2 - D.p); iy <= min(cy * e1 + e1 - 1, i2); ++iy) {
        long e = ((long)j * D.n1 + ix) * D.n1 + iy;
        int ka = i1 - ix, kb = i2 - iy;
        for (int q1 = 0; q1 < D.ng; ++q1)
          for (int q2 = 0; q2 < D.ng; ++q2) {
            double bs = T.phi1[(ix * D.ng + q1) * p1 + ka], bt = T.phi1[(iy * D.ng + q2) * p1 + kb];
            double W = T.gw[q1] * T.gw[q2] * D.h * D.h;
            long iq = e * D.nq + q1 * D.ng + q2;
            const double2 *gv = g + iq * D.CR;
            if (!D.hard) {
              acc = cadd(acc, cscale(gv[r], W * bs * bt));
            } else {
              double ds = T.dphi1[(ix * D.ng + q1) * p1 + ka] * bt;
              double dt = bs * T.dphi1[(iy * D.ng + q2) * p1 + kb];
              double2 w = cscale(gv[r], -bs * bt);  // -K
              double2 wc = cmk(0, 0);
              for (int d = 0; d < 3; ++d) {
                double cd = ds * T.gft[d * gst + iq] - dt * T.gfs[d * gst + iq];
                wc = cadd(wc, cscale(gv[(1 + d) * D.R + r], cd));
                wc = csub(wc, cscale(gv[(4 + d) * D.R + r], D.kappa * D.kappa * bs * bt * T.gpn[d * gst + iq]));
              }
              // - i eta wc
              w = cadd(w, cmk(D.eta * wc.y, -D.eta * wc.x));
              acc = cadd(acc, cscale(w, W));
            }
          }
      }
    yleaf[o] = cadd(yleaf[o], acc);
  }
}

// ----------------------------------------------------------------------------------------------
// Levels whose q differs from their children's ("band bottoms" of the level-adaptive interpolation):
// their expansions are formed from, and evaluated at, the Gauss points directly, since the child
// expansions of fewer points cannot carry the parent's Lagrange polynomials exactly.

// channel fields at the Gauss points, weighted by w_q h^2 (the integrand of the moments):
//   F[e][q][cr]: soft c0 = u;  hard c0 = u, c1..3 = d_s u d_t F - d_t u d_s F, c4..6 = n~ u
__global__ void k_gauss_channels(Dims D, Tables T, const double2 *__restrict__ xX, double2 *__restrict__ F) {
  const int p1 = D.p + 1;
  const long gst = D.E * D.nq;
  GRID_STRIDE(o, D.E * D.nq * D.CR) {
    const long e = o / (D.nq * D.CR);
    const int q = int((o / D.CR) % D.nq), cr = int(o % D.CR), c = cr / D.R, r = cr % D.R;
    const int q1 = q / D.ng, q2 = q % D.ng;
    const int j = int(e / ((long)D.n1 * D.n1)), ix = int((e / D.n1) % D.n1), iy = int(e % D.n1);
    double2 u = cmk(0, 0), us = cmk(0, 0), ut = cmk(0, 0);
    for (int ka = 0; ka < p1; ++ka) {
      const double bs = T.phi1[(ix * D.ng + q1) * p1 + ka], ds = T.dphi1[(ix * D.ng + q1) * p1 + ka];
      for (int kb = 0; kb < p1; ++kb) {
        const double bt = T.phi1[(iy * D.ng + q2) * p1 + kb], dt = T.dphi1[(iy * D.ng + q2) * p1 + kb];
        const double2 xv = xX[xindex(D, j, ix + ka, iy + kb) * D.R + r];
        u = cadd(u, cscale(xv, bs * bt));
        if (c >= 1 && c <= 3) {
          us = cadd(us, cscale(xv, ds * bt));
          ut = cadd(ut, cscale(xv, bs * dt));
        }
      }
    }
    const long iq = e * D.nq + q;
    double2 f;
    if (c == 0) {
      f = u;
    } else if (c <= 3) {
      f = csub(cscale(us, T.gft[(c - 1) * gst + iq]), cscale(ut, T.gfs[(c - 1) * gst + iq]));
    } else {
      f = cscale(u, T.gpn[(c - 4) * gst + iq]);
    }
    F[o] = cscale(f, T.gw[q1] * T.gw[q2] * D.h * D.h);
  }
}

constexpr int BAND_COLS = 16;

// FP32 forms for sound-soft problems in the mixed precisions (one channel, the density): the values at
// every Gauss point times the quadrature weight from the FP32 copy of the patch-wise coefficients (for
// k_p2m_band), and the band bottoms' fields tested against the basis (from k_l2p_band's FP32 output).
// GB300's FP64 pipe would bound the FP64 forms.
__global__ void k_gauss_channels32(Dims D, const float *__restrict__ phi1f, const float *__restrict__ gwq,
                                   const float2 *__restrict__ xX32, float2 *__restrict__ F) {
  const int p1 = D.p + 1;
  GRID_STRIDE(o, D.E * D.nq * D.R) {
    const long e = o / (D.nq * D.R);
    const int q = int((o / D.R) % D.nq), r = int(o % D.R);
    const int q1 = q / D.ng, q2 = q % D.ng;
    const int j = int(e / ((long)D.n1 * D.n1)), ix = int((e / D.n1) % D.n1), iy = int(e % D.n1);
    float ux = 0.f, uy = 0.f;
    for (int ka = 0; ka < p1; ++ka) {
      const float bs = phi1f[(ix * D.ng + q1) * p1 + ka];
      for (int kb = 0; kb < p1; ++kb) {
        const float w = bs * phi1f[(iy * D.ng + q2) * p1 + kb];
        const float2 xv = xX32[xindex(D, j, ix + ka, iy + kb) * D.R + r];
        ux += w * xv.x;
        uy += w * xv.y;
      }
    }
    const float w = gwq[q];
    F[o] = make_float2(ux * w, uy * w);
  }
}

__global__ void k_l2p_test32(Dims D, const float *__restrict__ phi1f, const float *__restrict__ gwq,
                             const float2 *__restrict__ g, double2 *__restrict__ yleaf) {
  const int nlL = 1 << D.L, e1 = 1 << D.b, p1 = D.p + 1;
  const long nleaf = (long)D.np * nlL * nlL;
  GRID_STRIDE(o, nleaf * D.nL * D.R) {
    long t = o / (D.nL * D.R);
    int i = int((o / D.R) % D.nL), r = int(o % D.R);
    int j = int(t / (nlL * nlL)), cx = int((t / nlL) % nlL), cy = int(t % nlL);
    int i1 = cx * e1 + i / D.nL1, i2 = cy * e1 + i % D.nL1;
    float ax = 0.f, ay = 0.f;
    for (int ix = max(cx * e1, i1 - D.p); ix <= min(cx * e1 + e1 - 1, i1); ++ix)
      for (int iy = max(cy * e1, i2 - D.p); iy <= min(cy * e1 + e1 - 1, i2); ++iy) {
        const long e = ((long)j * D.n1 + ix) * D.n1 + iy;
        const int ka = i1 - ix, kb = i2 - iy;
        for (int q1 = 0; q1 < D.ng; ++q1) {
          const float bs = phi1f[(ix * D.ng + q1) * p1 + ka];
          for (int q2 = 0; q2 < D.ng; ++q2) {
            const int q = q1 * D.ng + q2;
            const float w = gwq[q] * bs * phi1f[(iy * D.ng + q2) * p1 + kb];
            const float2 gv = g[(e * D.nq + q) * D.R + r];
            ax += w * gv.x;
            ay += w * gv.y;
          }
        }
      }
    yleaf[o] = make_double2(yleaf[o].x + (double)ax, yleaf[o].y + (double)ay);
  }
}

// P2M of a band bottom on level l (q = D.q): xhat[t][a1 q + a2][cr] = sum over the cluster's Gauss
// grid (i1, i2) of LG(i1, a1) LG(i2, a2) F(i1, i2, cr), separably: per row i1 of the grid
// Z[a2] = sum_i2 LG(i2, a2) F(i1, i2), then xhat[a1][a2] += LG(i1, a1) Z[a2].  One block per
// (cluster, 16 columns).
template <class T, class FT>
__global__ void __launch_bounds__(256) k_p2m_band(Dims D, int l, const double *__restrict__ LG,
                                                  const FT *__restrict__ F, double2 *__restrict__ xhat) {
  using V = typename CV<T>::type;
  extern __shared__ __align__(16) unsigned char smb[];
  const int q = D.q, Q = q * q, ne = 1 << (D.m - l), n1d = ne * D.ng;
  T *LGs = reinterpret_cast<T *>(smb);                               // [n1d][q]
  V *Fs = reinterpret_cast<V *>(LGs + ((n1d * q + 3) & ~3));         // [n1d][BAND_COLS]
  V *Z = Fs + n1d * BAND_COLS;                                       // [q][BAND_COLS]
  const int t = blockIdx.x, c0 = blockIdx.y * BAND_COLS, cw = min(BAND_COLS, D.CR - c0);
  const int nl = 1 << l, j = t / (nl * nl), cx = (t / nl) % nl, cy = t % nl;
  for (int i = threadIdx.x; i < n1d * q; i += blockDim.x) LGs[i] = (T)LG[i];
  constexpr int MO = 16;  // outputs per thread: Q * BAND_COLS <= 256 * 16
  V acc[MO];
#pragma unroll
  for (int k = 0; k < MO; ++k) acc[k].x = acc[k].y = 0;
  for (int i1 = 0; i1 < n1d; ++i1) {
    const int ix = cx * ne + i1 / D.ng, g1 = i1 % D.ng;
    __syncthreads();
    for (int i = threadIdx.x; i < n1d * BAND_COLS; i += blockDim.x) {
      const int i2 = i / BAND_COLS, col = i % BAND_COLS;
      const int iy = cy * ne + i2 / D.ng, g2 = i2 % D.ng;
      const long e = ((long)j * D.n1 + ix) * D.n1 + iy;
      V v;
      v.x = v.y = 0;
      if (col < cw) {
        const FT f = F[((e * D.nq) + g1 * D.ng + g2) * D.CR + c0 + col];
        v.x = (T)f.x;
        v.y = (T)f.y;
      }
      Fs[i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q * BAND_COLS; i += blockDim.x) {
      const int a2 = i / BAND_COLS, col = i % BAND_COLS;
      V sum;
      sum.x = sum.y = 0;
      for (int i2 = 0; i2 < n1d; ++i2) {
        const T w = LGs[i2 * q + a2];
        const V f = Fs[i2 * BAND_COLS + col];
        sum.x += w * f.x;
        sum.y += w * f.y;
      }
      Z[i] = sum;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MO; ++k) {
      const int i = threadIdx.x + 256 * k;
      if (i < Q * BAND_COLS) {
        const int a = i / BAND_COLS, col = i % BAND_COLS, a1 = a / q, a2 = a % q;
        const T w = LGs[i1 * q + a1];
        const V z = Z[a2 * BAND_COLS + col];
        acc[k].x += w * z.x;
        acc[k].y += w * z.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MO; ++k) {
    const int i = threadIdx.x + 256 * k;
    if (i < Q * BAND_COLS) {
      const int a = i / BAND_COLS, col = i % BAND_COLS;
      if (col < cw) xhat[((long)t * Q + a) * D.CR + c0 + col] = make_double2((double)acc[k].x, (double)acc[k].y);
    }
  }
}

// L2P of a band bottom on level l: G(i1, i2, cr) += sum_a1 LG(i1, a1) sum_a2 LG(i2, a2) yhat[t][a1 q + a2][cr]
// at every Gauss point of the cluster (G[e][q][cr], tested against the basis by k_l2p_test), separably:
// per grid row i1, U[a2] = sum_a1 LG(i1, a1) yhat[a1][a2], then G(i1, i2) += sum_a2 LG(i2, a2) U[a2].
template <class T, class FT>
__global__ void __launch_bounds__(256) k_l2p_band(Dims D, int l, const double *__restrict__ LG,
                                                  const double2 *__restrict__ yhat, FT *__restrict__ G) {
  using V = typename CV<T>::type;
  extern __shared__ __align__(16) unsigned char smb[];
  const int q = D.q, Q = q * q, ne = 1 << (D.m - l), n1d = ne * D.ng;
  T *LGs = reinterpret_cast<T *>(smb);                               // [n1d][q]
  V *Ys = reinterpret_cast<V *>(LGs + ((n1d * q + 3) & ~3));         // [Q][BAND_COLS]
  V *U = Ys + Q * BAND_COLS;                                         // [q][BAND_COLS]
  const int t = blockIdx.x, c0 = blockIdx.y * BAND_COLS, cw = min(BAND_COLS, D.CR - c0);
  const int nl = 1 << l, j = t / (nl * nl), cx = (t / nl) % nl, cy = t % nl;
  for (int i = threadIdx.x; i < n1d * q; i += blockDim.x) LGs[i] = (T)LG[i];
  for (int i = threadIdx.x; i < Q * BAND_COLS; i += blockDim.x) {
    const int a = i / BAND_COLS, col = i % BAND_COLS;
    V v;
    v.x = v.y = 0;
    if (col < cw) {
      const double2 y = yhat[((long)t * Q + a) * D.CR + c0 + col];
      v.x = (T)y.x;
      v.y = (T)y.y;
    }
    Ys[i] = v;
  }
  for (int i1 = 0; i1 < n1d; ++i1) {
    const int ix = cx * ne + i1 / D.ng, g1 = i1 % D.ng;
    __syncthreads();
    for (int i = threadIdx.x; i < q * BAND_COLS; i += blockDim.x) {
      const int a2 = i / BAND_COLS, col = i % BAND_COLS;
      V sum;
      sum.x = sum.y = 0;
      for (int a1 = 0; a1 < q; ++a1) {
        const T w = LGs[i1 * q + a1];
        const V y = Ys[(a1 * q + a2) * BAND_COLS + col];
        sum.x += w * y.x;
        sum.y += w * y.y;
      }
      U[i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n1d * BAND_COLS; i += blockDim.x) {
      const int i2 = i / BAND_COLS, col = i % BAND_COLS;
      if (col >= cw) continue;
      V sum;
      sum.x = sum.y = 0;
      for (int a2 = 0; a2 < q; ++a2) {
        const T w = LGs[i2 * q + a2];
        const V u = U[a2 * BAND_COLS + col];
        sum.x += w * u.x;
        sum.y += w * u.y;
      }
      const int iy = cy * ne + i2 / D.ng, g2 = i2 % D.ng;
      const long e = ((long)j * D.n1 + ix) * D.n1 + iy;
      FT *dst = G + ((e * D.nq) + g1 * D.ng + g2) * D.CR + c0 + col;
      dst->x += (decltype(dst->x))sum.x;
      dst->y += (decltype(dst->y))sum.y;
    }
  }
}

size_t band_smem(int n1d, int q, bool fp32, bool l2p) {
  const size_t ts = fp32 ? sizeof(float) : sizeof(double);
  const size_t lg = ((size_t)(n1d * q + 3) & ~size_t(3)) * ts;
  return lg + 2 * ts * BAND_COLS * (l2p ? ((size_t)q * q + q) : ((size_t)n1d + q));
}

// FP32 copy of a complex FP64 vector (the mixed precisions: one conversion per product instead of one
// per use inside the FP32 kernels; GB300 converts on its FP64 pipe)
__global__ void k_to_f32(const double2 *__restrict__ src, float2 *__restrict__ dst, long n) {
  GRID_STRIDE(i, n) {
    const double2 v = src[i];
    dst[i] = make_float2((float)v.x, (float)v.y);
  }
}

void to_f32(const void *src, float2 *dst, long n, cudaStream_t st) {
  if (n <= 0 || !dst) return;
  k_to_f32<<<grid_for(n), 256, 0, st>>>(reinterpret_cast<const double2 *>(src), dst, n);
  note_launch();
}

// y[i][r] = sum_{X in g2x(i)} sum_{leaves t containing X} y_leaf[t][local(X)][r]
__global__ void k_gather_out(Dims D, const int *__restrict__ g2x_ptr, const int *__restrict__ g2x_idx,
                             const double2 *__restrict__ yleaf, double2 *__restrict__ y) {
  const int nlL = 1 << D.L, e1 = 1 << D.b;
  GRID_STRIDE(o, D.N * D.R) {
    long gi = o / D.R;
    int r = int(o % D.R);
    double2 acc = cmk(0, 0);
    for (int k = g2x_ptr[gi]; k < g2x_ptr[gi + 1]; ++k) {
      long X = g2x_idx[k];
      int j = int(X / ((long)D.nb * D.nb)), i1 = int((X / D.nb) % D.nb), i2 = int(X % D.nb);
      int cx0 = max(0, (i1 - D.nL1 + e1) / e1), cx1 = min(nlL - 1, i1 / e1);
      int cy0 = max(0, (i2 - D.nL1 + e1) / e1), cy1 = min(nlL - 1, i2 / e1);
      for (int cx = cx0; cx <= cx1; ++cx)
        for (int cy = cy0; cy <= cy1; ++cy) {
          int li = (i1 - cx * e1) * D.nL1 + (i2 - cy * e1);
          long t = ((long)j * nlL + cx) * nlL + cy;
          acc = cadd(acc, yleaf[((size_t)t * D.nL + li) * D.R + r]);
        }
    }
    y[o] = acc;
  }
}

}  // namespace

void launch_precond(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                    const double *r, double *z, cudaStream_t st) {
  Dims D = dims(S, o, R);
  k_gather_in<<<grid_for(D.NX * R), 256, 0, st>>>(D, d.x2g, reinterpret_cast<const double2 *>(r),
                                                   reinterpret_cast<double2 *>(d.xX));
  note_launch();
  launch_block_apply(d, S, o, R, st);
  k_gather_out<<<grid_for(D.N * R), 256, 0, st>>>(D, d.g2x_ptr, d.g2x_idx,
                                                   reinterpret_cast<const double2 *>(d.yleaf),
                                                   reinterpret_cast<double2 *>(z));
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_matvec(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                   const double *x, double *y, cudaStream_t st) {
  Dims D = dims(S, o, R);
  const int nleaf = S.lev[S.L].n;
  {
    Phase ph(d.prof, IGABEM_PH_GATHER, st);
    k_gather_in<<<grid_for(D.NX * R), 256, 0, st>>>(D, d.x2g, reinterpret_cast<const double2 *>(x),
                                                     reinterpret_cast<double2 *>(d.xX));
    note_launch();
    if (o.precision != IGABEM_FP64) to_f32(d.xX, d.xX32, D.NX * R, st);
  }
  const bool leafk = leaf_kernels_supported(S);
  {
    Phase ph(d.prof, IGABEM_PH_NEAR, st);
    launch_near_spmv(d, S, o, R, st);
  }
  if (S.n_far > 0) {
    Tables T{d.phi1, d.dphi1, d.gw, d.LG1, d.T1, d.gpn, d.gfs, d.gft};
    auto X = [&](int l) { return reinterpret_cast<double2 *>(d.xhat[l]); };
    auto Y = [&](int l) { return reinterpret_cast<double2 *>(d.yhat[l]); };
    auto level_dims = [&](int l) {  // the dimensions with level l's interpolation points
      Dims Dl = D;
      Dl.q = S.lev[l].q;
      Dl.Q = Dl.q * Dl.q;
      return Dl;
    };
    const bool f32 = o.precision != IGABEM_FP64;
    bool bands = false;  // levels whose expansions come from the Gauss points directly
    for (int l = S.lmin; l < S.L; ++l) bands = bands || S.lev[l].band_bottom;
    double2 *gq = reinterpret_cast<double2 *>(d.gq);
    // sound-soft mixed precision: the band channels in FP32 (the same buffer, float2 entries)
    const bool f32s = f32 && !S.hard;
    float2 *gq32 = reinterpret_cast<float2 *>(d.gq);
    auto band_launch = [&](int l, bool l2p) {
      const Dims Dl = level_dims(l);
      const int n1d = (1 << (S.m - l)) * S.ng;
      const size_t smem = band_smem(n1d, Dl.q, f32, l2p);
      dim3 grid(S.lev[l].n, (D.CR + BAND_COLS - 1) / BAND_COLS);
      if (l2p) {
        if (f32s) {
          IGA_CUDA(set_max_dynamic_smem(k_l2p_band<float, float2>, smem));
          k_l2p_band<float, float2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], Y(l), gq32);
        } else if (f32) {
          IGA_CUDA(set_max_dynamic_smem(k_l2p_band<float, double2>, smem));
          k_l2p_band<float, double2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], Y(l), gq);
        } else {
          IGA_CUDA(set_max_dynamic_smem(k_l2p_band<double, double2>, smem));
          k_l2p_band<double, double2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], Y(l), gq);
        }
      } else {
        if (f32s) {
          IGA_CUDA(set_max_dynamic_smem(k_p2m_band<float, float2>, smem));
          k_p2m_band<float, float2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], gq32, X(l));
        } else if (f32) {
          IGA_CUDA(set_max_dynamic_smem(k_p2m_band<float, double2>, smem));
          k_p2m_band<float, double2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], gq, X(l));
        } else {
          IGA_CUDA(set_max_dynamic_smem(k_p2m_band<double, double2>, smem));
          k_p2m_band<double, double2><<<grid, 256, smem, st>>>(Dl, l, d.LGl[l], gq, X(l));
        }
      }
      note_launch();
    };
    long nleafQ = (long)nleaf * D.Q * D.CR;
    {
      Phase ph(d.prof, IGABEM_PH_P2M, st);
      if (leafk) {
        launch_p2m(d, S, o, R, st);
      } else {
        k_p2m<<<grid_for(nleafQ), 256, 0, st>>>(D, T, reinterpret_cast<const double2 *>(d.xX), X(S.L));
        note_launch();
      }
      if (bands) {
        if (f32s)
          k_gauss_channels32<<<grid_for(D.E * D.nq * D.R), 256, 0, st>>>(D, d.phi1f, d.gwqf, d.xX32, gq32);
        else
          k_gauss_channels<<<grid_for(D.E * D.nq * D.CR), 256, 0, st>>>(D, T, reinterpret_cast<const double2 *>(d.xX),
                                                                         gq);
        note_launch();
      }
    }
    const bool stored = !d.m2ls.empty() && d.m2ls[S.lmin];
    const bool tc = !stored && o.precision == IGABEM_MIXED_TC && m2l_tc_supported(S, R) && !d.tc_bimg.empty() &&
                    d.tc_bimg[S.L];
    {
      Phase ph(d.prof, IGABEM_PH_M2M, st);
      for (int l = S.L - 1; l >= S.lmin; --l) {
        if (S.lev[l].band_bottom) {
          band_launch(l, false);
          continue;
        }
        const Dims Dl = level_dims(l);  // the children have the same q
        long n = (long)S.lev[l].n * Dl.Q * D.CR;
        const bool sep = (D.CR >= 16 || (f32 && D.CR >= 4)) && Dl.q <= 16 && Dl.Q * SEP_COLS <= 256 * 8;
        const size_t smem = (size_t)2 * Dl.Q * SEP_COLS * (f32 ? sizeof(float2) : sizeof(double2));
        if (sep) {
          IGA_CUDA(f32 ? set_max_dynamic_smem(k_m2m_sep<float>, smem) : set_max_dynamic_smem(k_m2m_sep<double>, smem));
          dim3 grid(S.lev[l].n, (D.CR + SEP_COLS - 1) / SEP_COLS);
          if (f32)
            k_m2m_sep<float><<<grid, 256, smem, st>>>(Dl, l, d.T1l[l], X(l + 1), X(l));
          else
            k_m2m_sep<double><<<grid, 256, smem, st>>>(Dl, l, d.T1l[l], X(l + 1), X(l));
        } else {
          k_m2m<<<grid_for(n), 256, 0, st>>>(Dl, l, d.T1l[l], X(l + 1), X(l));
        }
        note_launch();
      }
      if (f32 && !tc)  // the upward pass's expansions in FP32 for the FP32 M2L kernels
        for (int l = S.lmin; l <= S.L; ++l)
          to_f32(d.xhat[l], d.xhat32[l], (long)S.lev[l].n * S.lev[l].q * S.lev[l].q * D.CR, st);
    }
    if (m2l_rows_supported(S, o, R)) {
      Phase ph(d.prof, IGABEM_PH_M2L, st);
      if (tc) launch_m2l_tc(d, S, o, R, st);
      else launch_m2l_rows(d, S, o, R, f32, st);
    } else {
      Phase ph(d.prof, IGABEM_PH_M2L, st);
      for (int l = S.lmin; l <= S.L; ++l) {
        const Dims Dl = level_dims(l);
        int crc = std::max(1, std::min(D.CR, (M2L_MO * 256) / Dl.Q));
        int ntypes = D.hard ? 2 : 1;
        size_t smem = (size_t)(ntypes * Dl.Q * M2L_BT + M2L_BT * crc) * sizeof(double2);
        IGA_CUDA(set_max_dynamic_smem(k_m2l, smem));
        dim3 grid(S.lev[l].n, (D.CR + crc - 1) / crc);
        k_m2l<<<grid, 256, smem, st>>>(Dl, S.lev[l].n, d.far_ptr[l], d.far_src[l], d.nodes[l], X(l), Y(l), crc);
        note_launch();
      }
    }
    {
      Phase ph(d.prof, IGABEM_PH_L2L, st);
      if (bands) IGA_CUDA(cudaMemsetAsync(gq, 0, sizeof(double2) * D.E * D.nq * D.CR, st));
      for (int l = S.lmin; l < S.L; ++l) {
        if (S.lev[l].band_bottom) {
          band_launch(l, true);
          continue;
        }
        const Dims Dl = level_dims(l);
        long n = (long)S.lev[l + 1].n * Dl.Q * D.CR;
        const bool sep = (D.CR >= 16 || (f32 && D.CR >= 4)) && Dl.q <= 16;
        const size_t smem = (size_t)3 * Dl.Q * SEP_COLS * (f32 ? sizeof(float2) : sizeof(double2));
        if (sep && smem <= (size_t)max_optin_smem() - 4096) {
          IGA_CUDA(f32 ? set_max_dynamic_smem(k_l2l_sep<float>, smem) : set_max_dynamic_smem(k_l2l_sep<double>, smem));
          dim3 grid(S.lev[l].n, (D.CR + SEP_COLS - 1) / SEP_COLS);
          if (f32)
            k_l2l_sep<float><<<grid, 256, smem, st>>>(Dl, l, d.T1l[l], Y(l), Y(l + 1));
          else
            k_l2l_sep<double><<<grid, 256, smem, st>>>(Dl, l, d.T1l[l], Y(l), Y(l + 1));
        } else {
          k_l2l<<<grid_for(n), 256, 0, st>>>(Dl, l, d.T1l[l], Y(l), Y(l + 1));
        }
        note_launch();
      }
    }
    {
      Phase ph(d.prof, IGABEM_PH_L2P, st);
      if (f32) to_f32(d.yhat[S.L], d.y32, (long)nleaf * D.Q * D.CR, st);
      if (bands) {  // the band bottoms' fields at the Gauss points, tested (before gq is reused below)
        if (f32s)
          k_l2p_test32<<<grid_for((long)nleaf * D.nL * R), 256, 0, st>>>(D, d.phi1f, d.gwqf, gq32,
                                                                          reinterpret_cast<double2 *>(d.yleaf));
        else
          k_l2p_test<<<grid_for((long)nleaf * D.nL * R), 256, 0, st>>>(D, T, gq, reinterpret_cast<double2 *>(d.yleaf));
        note_launch();
      }
      if (leafk) {
        launch_l2p(d, S, o, R, st);
      } else {
        k_l2p_eval<<<grid_for(D.E * D.nq * D.CR), 256, 0, st>>>(D, T, Y(S.L), reinterpret_cast<double2 *>(d.gq));
        note_launch();
        k_l2p_test<<<grid_for((long)nleaf * D.nL * R), 256, 0, st>>>(D, T, reinterpret_cast<const double2 *>(d.gq),
                                                                      reinterpret_cast<double2 *>(d.yleaf));
        note_launch();
      }
    }
  }
  {
    Phase ph(d.prof, IGABEM_PH_GATHER, st);
    k_gather_out<<<grid_for(D.N * R), 256, 0, st>>>(D, d.g2x_ptr, d.g2x_idx,
                                                     reinterpret_cast<const double2 *>(d.yleaf),
                                                     reinterpret_cast<double2 *>(y));
    note_launch();
  }
  IGA_CUDA(cudaGetLastError());
}

}  // namespace igabem
