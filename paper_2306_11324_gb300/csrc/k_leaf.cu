// Leaf-level kernels of the matrix-vector product, one thread block per leaf cluster:
//   * near-field SpMV over the leaf's near blocks (HBM-bound);
//   * P2M: channel fields of u = sum x_l psi_l at the leaf's Gauss points, projected onto the
//     leaf's tensor Chebyshev basis (Sec. 4.4);
//   * L2P: local expansions evaluated at the Gauss points and tested against the leaf's B-splines.
// The leaf's Gauss points form a tensor grid of nG = 2^b ng points per direction; basis values,
// derivatives and Lagrange values are separable, so both passes are pairs of small 1-D contractions
// through shared memory.
#include <algorithm>

#include "internal.h"
#include "k_common.cuh"
#include "kernels.h"

namespace igabem {

namespace {

struct LeafArgs {
  const double *phi1, *dphi1, *gw, *LG1;
  const double *gpn, *gfs, *gft;  // Gauss-point geometry SoA, stride gst
  long gst;
  int np, n1, nb, p, b, L, q, ng, nL1, R, C;
  double h, kappa, eta;
  bool hard;
};

// Phi[g][alpha] of the leaf (g = o*ng + q over the leaf's element offset o): the value (or d/ds) of
// the leaf-local B-spline alpha at Gauss abscissa g; zero off the element's p+1 functions.
__device__ inline double leaf_phi(const LeafArgs &A, const double *tab, int c0, int g, int alpha) {
  int o = g / A.ng, qq = g % A.ng, ka = alpha - o;
  if (ka < 0 || ka > A.p) return 0.0;
  int ix = c0 + o;
  return tab[(ix * A.ng + qq) * (A.p + 1) + ka];
}

// near-field SpMV: y_leaf[t][i][r] = sum_{(t,s) near} sum_j B[j][i] x_s[j][r], block k column-major
template <class BT>
__global__ void k_near_spmv2(LeafArgs A, const int *__restrict__ near_ptr, const int *__restrict__ near_src,
                             const BT *__restrict__ blk, const double2 *__restrict__ xX,
                             double2 *__restrict__ yleaf, int nL) {
  extern __shared__ double2 ysm[];
  const int t = blockIdx.x;
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int nout = nL * A.R;
  const int G = nout <= (int)blockDim.x / 2 ? (int)blockDim.x / nout : 1;
  const int GS = G > 1 ? nout : (int)blockDim.x;
  const int g = threadIdx.x / GS, lt = threadIdx.x % GS;
  // this block's share of the target's near list (blockIdx.y of gridDim.y chunks)
  const int kb = near_ptr[t], ke = near_ptr[t + 1];
  const int chunk = (ke - kb + gridDim.y - 1) / gridDim.y;
  const int k0 = kb + blockIdx.y * chunk, k1 = min(ke, k0 + chunk);
  if (g < G) {
    for (int o = lt; o < nout; o += GS) {
      const int i = o / A.R, r = o % A.R;
      // one block's sum in the storage precision (FP32 blocks: FP32 arithmetic), the blocks summed
      // in FP64
      using RT = decltype(BT::x);
      double ax = 0.0, ay = 0.0;
      for (int k = k0 + g; k < k1; k += G) {
        const int s = near_src[k];
        const int js = s / (nlL * nlL), cx = (s / nlL) % nlL, cy = s % nlL;
        const BT *B = blk + (size_t)k * nL * nL + i;
        const long base = ((long)js * A.nb + cx * e1) * A.nb + cy * e1;
        int jj = 0;
        RT bx = 0, by = 0;
        for (int al = 0; al < A.nL1; ++al) {
          const double2 *xr = xX + (base + (long)al * A.nb) * A.R + r;
#pragma unroll 4
          for (int be = 0; be < A.nL1; ++be, ++jj) {
            const BT bv = B[(size_t)jj * nL];
            const double2 xd = xr[(long)be * A.R];
            const RT xvx = (RT)xd.x, xvy = (RT)xd.y;
            bx += bv.x * xvx - bv.y * xvy;
            by += bv.x * xvy + bv.y * xvx;
          }
        }
        ax += (double)bx;
        ay += (double)by;
      }
      if (G > 1) {
        ysm[g * nout + o] = make_double2(ax, ay);
      } else if (gridDim.y == 1) {
        yleaf[(size_t)t * nout + o] = make_double2(ax, ay);
      } else {
        atomicAdd(&yleaf[(size_t)t * nout + o].x, ax);
        atomicAdd(&yleaf[(size_t)t * nout + o].y, ay);
      }
    }
  }
  if (G > 1) {
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      double2 s = make_double2(0, 0);
      for (int gg = 0; gg < G; ++gg) {
        s.x += ysm[gg * nout + o].x;
        s.y += ysm[gg * nout + o].y;
      }
      if (gridDim.y == 1) {
        yleaf[(size_t)t * nout + o] = s;
      } else {
        atomicAdd(&yleaf[(size_t)t * nout + o].x, s.x);
        atomicAdd(&yleaf[(size_t)t * nout + o].y, s.y);
      }
    }
  }
}

// P2M for the columns [r0, r0 + Rc) of every channel.
// shared: X[nL1][nL1][Rc], U[nG][nL1][Rc] (and dU), f[nG][nG][C][Rc], T[q][nG][C][Rc]
__global__ void k_p2m2(LeafArgs A, const double2 *__restrict__ xX, double2 *__restrict__ xhat, int r0, int Rc) {
  extern __shared__ double2 sm2[];
  const int t = blockIdx.x;
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int j = t / (nlL * nlL), cx = (t / nlL) % nlL, cy = t % nlL;
  const int c0x = cx * e1, c0y = cy * e1;
  const int nG = e1 * A.ng, nL1 = A.nL1, q = A.q, C = A.C;
  double2 *X = sm2;                          // [nL1][nL1][Rc]
  double2 *U = X + nL1 * nL1 * Rc;           // [nG][nL1][Rc]
  double2 *dU = U + nG * nL1 * Rc;           // [nG][nL1][Rc]
  double2 *f = dU + nG * nL1 * Rc;           // [nG][nG][C][Rc]
  double2 *T = f + nG * nG * C * Rc;         // [q][nG][C][Rc]
  for (int i = threadIdx.x; i < nL1 * nL1 * Rc; i += blockDim.x) {
    int al = i / (nL1 * Rc), be = (i / Rc) % nL1, r = i % Rc;
    X[i] = xX[(((long)j * A.nb + c0x + al) * A.nb + c0y + be) * A.R + r0 + r];
  }
  __syncthreads();
  // U[g1][be] = sum_al Phi[g1][al] X[al][be];  dU with d/ds Phi
  for (int i = threadIdx.x; i < nG * nL1 * Rc; i += blockDim.x) {
    int g1 = i / (nL1 * Rc), be = (i / Rc) % nL1, r = i % Rc;
    double2 u = cmk(0, 0), du = cmk(0, 0);
    for (int al = 0; al < nL1; ++al) {
      double ph = leaf_phi(A, A.phi1, c0x, g1, al);
      double dph = A.hard ? leaf_phi(A, A.dphi1, c0x, g1, al) : 0.0;
      double2 xv = X[(al * nL1 + be) * Rc + r];
      u = cadd(u, cscale(xv, ph));
      du = cadd(du, cscale(xv, dph));
    }
    U[i] = u;
    dU[i] = du;
  }
  __syncthreads();
  // channel fields at (g1, g2), weighted by w_q1 w_q2 h^2
  for (int i = threadIdx.x; i < nG * nG * Rc; i += blockDim.x) {
    int g1 = i / (nG * Rc), g2 = (i / Rc) % nG, r = i % Rc;
    double2 u = cmk(0, 0), us = cmk(0, 0), ut = cmk(0, 0);
    for (int be = 0; be < nL1; ++be) {
      double ph = leaf_phi(A, A.phi1, c0y, g2, be);
      u = cadd(u, cscale(U[(g1 * nL1 + be) * Rc + r], ph));
      if (A.hard) {
        us = cadd(us, cscale(dU[(g1 * nL1 + be) * Rc + r], ph));
        ut = cadd(ut, cscale(U[(g1 * nL1 + be) * Rc + r], leaf_phi(A, A.dphi1, c0y, g2, be)));
      }
    }
    double W = A.gw[g1 % A.ng] * A.gw[g2 % A.ng] * A.h * A.h;
    double2 *fo = f + ((g1 * nG + g2) * C) * Rc + r;
    fo[0] = cscale(u, W);
    if (A.hard) {
      long e = ((long)j * A.n1 + c0x + g1 / A.ng) * A.n1 + c0y + g2 / A.ng;
      long iq = e * A.ng * A.ng + (g1 % A.ng) * A.ng + g2 % A.ng;
      for (int d = 0; d < 3; ++d) {
        double fs = A.gfs[d * A.gst + iq], ft = A.gft[d * A.gst + iq], nn = A.gpn[d * A.gst + iq];
        fo[(1 + d) * Rc] = cscale(csub(cscale(us, ft), cscale(ut, fs)), W);
        fo[(4 + d) * Rc] = cscale(u, nn * W);
      }
    }
  }
  __syncthreads();
  // T[a1][g2][cr] = sum_g1 L[g1][a1] f[g1][g2][cr]
  const int CRc = C * Rc;
  for (int i = threadIdx.x; i < q * nG * CRc; i += blockDim.x) {
    int a1 = i / (nG * CRc), g2 = (i / CRc) % nG, cr = i % CRc;
    double2 s = cmk(0, 0);
    for (int g1 = 0; g1 < nG; ++g1)
      s = cadd(s, cscale(f[(g1 * nG + g2) * CRc + cr], A.LG1[((g1 / A.ng) * A.ng + g1 % A.ng) * q + a1]));
    T[i] = s;
  }
  __syncthreads();
  // xhat[t][a1 q + a2][c][r0 + r] = sum_g2 L[g2][a2] T[a1][g2][cr]
  for (int i = threadIdx.x; i < q * q * CRc; i += blockDim.x) {
    int a1 = i / (q * CRc), a2 = (i / CRc) % q, cr = i % CRc, c = cr / Rc, r = cr % Rc;
    double2 s = cmk(0, 0);
    for (int g2 = 0; g2 < nG; ++g2)
      s = cadd(s, cscale(T[(a1 * nG + g2) * CRc + cr], A.LG1[((g2 / A.ng) * A.ng + g2 % A.ng) * q + a2]));
    xhat[(((long)t * q * q + a1 * q + a2) * C + c) * A.R + r0 + r] = s;
  }
}

// L2P for the columns [r0, r0 + Rc): y_leaf[t][alpha beta][r] += tested local expansion.
// shared: Y[Q][C][Rc], V[nG][q][C][Rc], g[nG][nG][C][Rc] (reused for h0/hs/ht), Z[nL1][nG][Rc] x2
__global__ void k_l2p2(LeafArgs A, const double2 *__restrict__ yhat, double2 *__restrict__ yleaf, int r0, int Rc) {
  extern __shared__ double2 sm3[];
  const int t = blockIdx.x;
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int j = t / (nlL * nlL), cx = (t / nlL) % nlL, cy = t % nlL;
  const int c0x = cx * e1, c0y = cy * e1;
  const int nG = e1 * A.ng, nL1 = A.nL1, q = A.q, C = A.C, CRc = C * Rc;
  double2 *Y = sm3;                          // [q][q][C][Rc]
  double2 *V = Y + q * q * CRc;              // [nG][q][C][Rc]
  double2 *g = V + nG * q * CRc;             // [nG][nG][C][Rc]
  double2 *H = g + nG * nG * CRc;            // [3][nG][nG][Rc]: h0, hs, ht
  double2 *Z = H + 3 * nG * nG * Rc;         // [2][nL1][nG][Rc]
  for (int i = threadIdx.x; i < q * q * CRc; i += blockDim.x) {
    int a = i / CRc, c = (i % CRc) / Rc, r = i % Rc;
    Y[i] = yhat[(((long)t * q * q + a) * C + c) * A.R + r0 + r];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nG * q * CRc; i += blockDim.x) {
    int g1 = i / (q * CRc), a2 = (i / CRc) % q, cr = i % CRc;
    double2 s = cmk(0, 0);
    for (int a1 = 0; a1 < q; ++a1) s = cadd(s, cscale(Y[(a1 * q + a2) * CRc + cr], A.LG1[g1 * q + a1]));
    V[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nG * nG * CRc; i += blockDim.x) {
    int g1 = i / (nG * CRc), g2 = (i / CRc) % nG, cr = i % CRc;
    double2 s = cmk(0, 0);
    for (int a2 = 0; a2 < q; ++a2) s = cadd(s, cscale(V[(g1 * q + a2) * CRc + cr], A.LG1[g2 * q + a2]));
    g[i] = s;
  }
  __syncthreads();
  // test functionals at the Gauss points: y = sum Phi Phi h0 + dPhi Phi hs + Phi dPhi ht
  for (int i = threadIdx.x; i < nG * nG * Rc; i += blockDim.x) {
    int g1 = i / (nG * Rc), g2 = (i / Rc) % nG, r = i % Rc;
    double W = A.gw[g1 % A.ng] * A.gw[g2 % A.ng] * A.h * A.h;
    const double2 *gv = g + (g1 * nG + g2) * CRc + r;
    double2 h0, hs = cmk(0, 0), ht = cmk(0, 0);
    if (!A.hard) {
      h0 = cscale(gv[0], W);
    } else {
      long e = ((long)j * A.n1 + c0x + g1 / A.ng) * A.n1 + c0y + g2 / A.ng;
      long iq = e * A.ng * A.ng + (g1 % A.ng) * A.ng + g2 % A.ng;
      // -K part and the normal part of -i eta W (+ i eta kappa^2 n~ . g_n)
      double2 nn = cmk(0, 0), cs = cmk(0, 0), ct = cmk(0, 0);
      for (int d = 0; d < 3; ++d) {
        double fs = A.gfs[d * A.gst + iq], ft = A.gft[d * A.gst + iq], n = A.gpn[d * A.gst + iq];
        nn = cadd(nn, cscale(gv[(4 + d) * Rc], n));
        cs = cadd(cs, cscale(gv[(1 + d) * Rc], ft));
        ct = cadd(ct, cscale(gv[(1 + d) * Rc], -fs));
      }
      double k2e = A.kappa * A.kappa * A.eta;
      h0 = cscale(cadd(cscale(gv[0], -1.0), cmk(-k2e * nn.y, k2e * nn.x)), W);
      // -i eta (curl test): multiplies d_s psi with cs and d_t psi with ct
      hs = cscale(cmk(A.eta * cs.y, -A.eta * cs.x), W);
      ht = cscale(cmk(A.eta * ct.y, -A.eta * ct.x), W);
    }
    H[(0 * nG * nG) * Rc + i] = h0;
    H[(1 * nG * nG) * Rc + i] = hs;
    H[(2 * nG * nG) * Rc + i] = ht;
  }
  __syncthreads();
  // Z0[al][g2] = sum_g1 Phi[g1][al] h0 + dPhi[g1][al] hs;  Z1[al][g2] = sum_g1 Phi[g1][al] ht
  for (int i = threadIdx.x; i < nL1 * nG * Rc; i += blockDim.x) {
    int al = i / (nG * Rc), g2 = (i / Rc) % nG, r = i % Rc;
    double2 z0 = cmk(0, 0), z1 = cmk(0, 0);
    for (int g1 = 0; g1 < nG; ++g1) {
      double ph = leaf_phi(A, A.phi1, c0x, g1, al);
      if (ph == 0.0 && !A.hard) continue;
      long o = (g1 * nG + g2) * Rc + r;
      z0 = cadd(z0, cscale(H[o], ph));
      if (A.hard) {
        z0 = cadd(z0, cscale(H[nG * nG * Rc + o], leaf_phi(A, A.dphi1, c0x, g1, al)));
        z1 = cadd(z1, cscale(H[2 * nG * nG * Rc + o], ph));
      }
    }
    Z[i] = z0;
    Z[nL1 * nG * Rc + i] = z1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nL1 * nL1 * Rc; i += blockDim.x) {
    int al = i / (nL1 * Rc), be = (i / Rc) % nL1, r = i % Rc;
    double2 s = cmk(0, 0);
    for (int g2 = 0; g2 < nG; ++g2) {
      double ph = leaf_phi(A, A.phi1, c0y, g2, be);
      s = cadd(s, cscale(Z[(al * nG + g2) * Rc + r], ph));
      if (A.hard) s = cadd(s, cscale(Z[nL1 * nG * Rc + (al * nG + g2) * Rc + r], leaf_phi(A, A.dphi1, c0y, g2, be)));
    }
    double2 *dst = yleaf + ((size_t)t * A.nL1 * A.nL1 + al * nL1 + be) * A.R + r0 + r;
    *dst = cadd(*dst, s);
  }
}

LeafArgs leaf_args(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R) {
  LeafArgs A;
  A.phi1 = d.phi1; A.dphi1 = d.dphi1; A.gw = d.gw; A.LG1 = d.LG1;
  A.gpn = d.gpn; A.gfs = d.gfs; A.gft = d.gft;
  A.gst = (long)S.E * S.ng * S.ng;
  A.np = S.np; A.n1 = S.n1; A.nb = S.nb; A.p = S.p; A.b = S.b; A.L = S.L; A.q = S.q; A.ng = S.ng;
  A.nL1 = S.nL1; A.R = R; A.C = S.hard ? 7 : 1;
  A.h = S.h; A.kappa = o.kappa; A.eta = o.eta_cfie; A.hard = S.hard;
  return A;
}

size_t p2m_smem(const HostSetup &S, int C, int Rc) {
  int nG = (1 << S.b) * S.ng;
  return sizeof(double2) * ((size_t)S.nL1 * S.nL1 * Rc + 2 * (size_t)nG * S.nL1 * Rc + (size_t)nG * nG * C * Rc +
                            (size_t)S.q * nG * C * Rc);
}

size_t l2p_smem(const HostSetup &S, int C, int Rc) {
  int nG = (1 << S.b) * S.ng;
  return sizeof(double2) * ((size_t)S.q * S.q * C * Rc + (size_t)nG * S.q * C * Rc + (size_t)nG * nG * C * Rc +
                            3 * (size_t)nG * nG * Rc + 2 * (size_t)S.nL1 * nG * Rc);
}

int column_chunk(size_t (*smem)(const HostSetup &, int, int), const HostSetup &S, int C, int R) {
  int Rc = R;
  while (Rc > 1 && smem(S, C, Rc) > 200 * 1024) Rc = (Rc + 1) / 2;
  return Rc;
}

}  // namespace

namespace {
// Preconditioner blocks: for every leaf t, the near-field part of the operator restricted to the
// leaf's own functions (the principal submatrix A[I_t, I_t]: every leaf-pair block (t', s') whose
// leaves carry both functions contributes its entry), inverted by Gauss-Jordan elimination with
// partial pivoting in FP64.  A numerically singular block is replaced by the identity.
struct InvArgs {
  const int *near_ptr, *near_src;
  const int *x2g, *g2x_ptr, *g2x_idx;
  int L, b, nL1, nL, nb;
};

// near-field entry A^near[X_r, X_c] between two patch-wise functions (possibly of different patches):
// the sum over the leaf pairs whose leaves carry the two functions
template <class BT>
__device__ double2 near_entry(const InvArgs &A, const BT *__restrict__ blk, int Xr, int Xc) {
  const int nlL = 1 << A.L, e1 = 1 << A.b, nb2 = A.nb * A.nb;
  const int jr = Xr / nb2, r1 = (Xr / A.nb) % A.nb, r2 = Xr % A.nb;
  const int jc = Xc / nb2, c1 = (Xc / A.nb) % A.nb, c2 = Xc % A.nb;
  double2 sum = make_double2(0, 0);
  auto lo = [&](int i) { return max(0, (i - A.nL1 + e1) / e1); };
  auto hi = [&](int i) { return min(nlL - 1, i / e1); };
  for (int x1 = lo(r1); x1 <= hi(r1); ++x1)
    for (int y1 = lo(r2); y1 <= hi(r2); ++y1) {
      const int tp = (jr * nlL + x1) * nlL + y1;
      const int rl = (r1 - x1 * e1) * A.nL1 + (r2 - y1 * e1);
      const int k0 = A.near_ptr[tp], k1 = A.near_ptr[tp + 1];
      for (int x2 = lo(c1); x2 <= hi(c1); ++x2)
        for (int y2 = lo(c2); y2 <= hi(c2); ++y2) {
          const int sp = (jc * nlL + x2) * nlL + y2;
          int a = k0, z = k1;  // binary search for the near block (tp, sp)
          while (a < z) {
            int mid = (a + z) >> 1;
            if (A.near_src[mid] < sp) a = mid + 1; else z = mid;
          }
          if (a < k1 && A.near_src[a] == sp) {
            const int cl = (c1 - x2 * e1) * A.nL1 + (c2 - y2 * e1);
            const BT v = blk[(size_t)a * A.nL * A.nL + (size_t)cl * A.nL + rl];
            sum.x += (double)v.x;
            sum.y += (double)v.y;
          }
        }
    }
  return sum;
}

// entry (al, be) of the principal submatrix of leaf t in global numbering: the basis functions of
// the (continuous) space are sums of their patch-wise copies
template <class BT>
__device__ double2 principal_entry(const InvArgs &A, const BT *__restrict__ blk, int t, int al, int be) {
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int j = t / (nlL * nlL), cx = (t / nlL) % nlL, cy = t % nlL;
  const int Xa = (j * A.nb + cx * e1 + al / A.nL1) * A.nb + cy * e1 + al % A.nL1;
  const int Xb = (j * A.nb + cx * e1 + be / A.nL1) * A.nb + cy * e1 + be % A.nL1;
  const int ga = A.x2g[Xa], gb = A.x2g[Xb];
  double2 sum = make_double2(0, 0);
  for (int u = A.g2x_ptr[ga]; u < A.g2x_ptr[ga + 1]; ++u)
    for (int v = A.g2x_ptr[gb]; v < A.g2x_ptr[gb + 1]; ++v) {
      double2 e = near_entry(A, blk, A.g2x_idx[u], A.g2x_idx[v]);
      sum.x += e.x;
      sum.y += e.y;
    }
  return sum;
}

template <class BT>
__global__ void k_block_inverse(InvArgs IA, const BT *__restrict__ blk, double2 *__restrict__ binv) {
  extern __shared__ double2 gj[];
  const int nL = IA.nL;
  double2 *M = gj, *I = gj + nL * nL, *fac = I + nL * nL;
  __shared__ int piv;
  __shared__ bool bad;
  const int t = blockIdx.x;
  for (int o = threadIdx.x; o < nL * nL; o += blockDim.x) {
    int i = o / nL, j = o % nL;                       // row-major M[i][j] = A[I_t(i), I_t(j)]
    M[o] = principal_entry(IA, blk, t, i, j);
    I[o] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (threadIdx.x == 0) bad = false;
  __syncthreads();
  for (int c = 0; c < nL; ++c) {
    if (threadIdx.x == 0) {
      int best = c;
      double bv = -1.0;
      for (int r = c; r < nL; ++r) {
        double2 v = M[r * nL + c];
        double a = v.x * v.x + v.y * v.y;
        if (a > bv) {
          bv = a;
          best = r;
        }
      }
      piv = best;
      if (!(bv > 1e-280)) bad = true;
    }
    __syncthreads();
    if (bad) break;
    const int pr = piv;
    if (pr != c)
      for (int j = threadIdx.x; j < nL; j += blockDim.x) {
        double2 a = M[c * nL + j], b = M[pr * nL + j];
        M[c * nL + j] = b; M[pr * nL + j] = a;
        a = I[c * nL + j]; b = I[pr * nL + j];
        I[c * nL + j] = b; I[pr * nL + j] = a;
      }
    __syncthreads();
    const double2 d = M[c * nL + c];
    const double den = d.x * d.x + d.y * d.y;
    const double2 inv = make_double2(d.x / den, -d.y / den);
    __syncthreads();
    for (int j = threadIdx.x; j < nL; j += blockDim.x) {
      M[c * nL + j] = cmul(M[c * nL + j], inv);
      I[c * nL + j] = cmul(I[c * nL + j], inv);
    }
    for (int r = threadIdx.x; r < nL; r += blockDim.x) fac[r] = M[r * nL + c];
    __syncthreads();
    for (int o = threadIdx.x; o < nL * nL; o += blockDim.x) {
      int r = o / nL, j = o % nL;
      if (r == c) continue;
      M[o] = csub(M[o], cmul(fac[r], M[c * nL + j]));
      I[o] = csub(I[o], cmul(fac[r], I[c * nL + j]));
    }
    __syncthreads();
  }
  double2 *out = binv + (size_t)t * nL * nL;
  for (int o = threadIdx.x; o < nL * nL; o += blockDim.x) {
    int i = o / nL, j = o % nL;                       // column-major out[j][i] = Inv[i][j]
    out[(size_t)j * nL + i] = bad ? make_double2(i == j ? 1.0 : 0.0, 0.0) : I[o];
  }
}

__global__ void k_to_fp32(const double *__restrict__ src, float *__restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
}  // namespace

void launch_blocks_to_fp32(const double *src, float *dst, size_t n, cudaStream_t st) {
  k_to_fp32<<<152 * 8, 256, 0, st>>>(src, dst, n);
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_block_inverse(const DeviceProblem &d, const HostSetup &S, cudaStream_t st) {
  const int nleaf = S.lev[S.L].n;
  const size_t smem = (2 * (size_t)S.nL * S.nL + S.nL) * sizeof(double2);
  InvArgs IA{d.near_ptr, d.near_src, d.x2g, d.g2x_ptr, d.g2x_idx, S.L, S.b, S.nL1, S.nL, S.nb};
  if (d.blk) {
    IGA_CUDA(set_max_dynamic_smem(k_block_inverse<double2>, smem));
    k_block_inverse<double2><<<nleaf, 256, smem, st>>>(IA, reinterpret_cast<const double2 *>(d.blk),
                                                       reinterpret_cast<double2 *>(d.binv));
  } else {
    IGA_CUDA(set_max_dynamic_smem(k_block_inverse<float2>, smem));
    k_block_inverse<float2><<<nleaf, 256, smem, st>>>(IA, reinterpret_cast<const float2 *>(d.blk32),
                                                      reinterpret_cast<double2 *>(d.binv));
  }
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

// z_leaf[t] = Binv_t x_t for every leaf t (the same product as the near-field SpMV, one block per leaf)
void launch_block_apply(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                        cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, R);
  const int nleaf = S.lev[S.L].n, nout = S.nL * R, threads = 256;
  const int G = nout <= threads / 2 ? threads / nout : 1;
  size_t smem = G > 1 ? (size_t)G * nout * sizeof(double2) : 0;
  k_near_spmv2<double2><<<dim3(nleaf, 1), threads, smem, st>>>(A, d.ident_ptr, d.ident_src,
                                                               reinterpret_cast<const double2 *>(d.binv),
                                                               reinterpret_cast<const double2 *>(d.xX),
                                                               reinterpret_cast<double2 *>(d.yleaf), S.nL);
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

bool leaf_kernels_supported(const HostSetup &S) {
  int C = S.hard ? 7 : 1;
  return p2m_smem(S, C, 1) <= 200 * 1024 && l2p_smem(S, C, 1) <= 200 * 1024;
}

void launch_near_spmv(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                      cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, R);
  const int nleaf = S.lev[S.L].n, nout = S.nL * R, threads = 256;
  const int G = nout <= threads / 2 ? threads / nout : 1;
  size_t smem = G > 1 ? (size_t)G * nout * sizeof(double2) : 0;
  // enough blocks to keep HBM busy: split long near lists over gridDim.y blocks that add atomically
  int maxlen = 0;
  for (int t = 0; t < nleaf; ++t) maxlen = std::max(maxlen, S.near_ptr[t + 1] - S.near_ptr[t]);
  int split = std::max(1, std::min(maxlen / std::max(1, 2 * G), (4 * 152 + nleaf - 1) / nleaf));
  if (split > 1) {
    IGA_CUDA(cudaMemsetAsync(d.yleaf, 0, (size_t)nleaf * nout * sizeof(double2), st));
  }
  dim3 grid(nleaf, split);
  if (d.blk32) {
    k_near_spmv2<float2><<<grid, threads, smem, st>>>(A, d.near_ptr, d.near_src,
                                                       reinterpret_cast<const float2 *>(d.blk32),
                                                       reinterpret_cast<const double2 *>(d.xX),
                                                       reinterpret_cast<double2 *>(d.yleaf), S.nL);
  } else {
    k_near_spmv2<double2><<<grid, threads, smem, st>>>(A, d.near_ptr, d.near_src,
                                                        reinterpret_cast<const double2 *>(d.blk),
                                                        reinterpret_cast<const double2 *>(d.xX),
                                                        reinterpret_cast<double2 *>(d.yleaf), S.nL);
  }
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_p2m(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, R);
  const int nleaf = S.lev[S.L].n;
  int Rc = column_chunk(p2m_smem, S, A.C, R);
  size_t smem = p2m_smem(S, A.C, Rc);
  IGA_CUDA(set_max_dynamic_smem(k_p2m2, smem));
  for (int r0 = 0; r0 < R; r0 += Rc) {
    k_p2m2<<<nleaf, 256, smem, st>>>(A, reinterpret_cast<const double2 *>(d.xX),
                                     reinterpret_cast<double2 *>(d.xhat[S.L]), r0, std::min(Rc, R - r0));
    note_launch();
  }
  IGA_CUDA(cudaGetLastError());
}

void launch_l2p(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, R);
  const int nleaf = S.lev[S.L].n;
  int Rc = column_chunk(l2p_smem, S, A.C, R);
  size_t smem = l2p_smem(S, A.C, Rc);
  IGA_CUDA(set_max_dynamic_smem(k_l2p2, smem));
  for (int r0 = 0; r0 < R; r0 += Rc) {
    k_l2p2<<<nleaf, 256, smem, st>>>(A, reinterpret_cast<const double2 *>(d.yhat[S.L]),
                                     reinterpret_cast<double2 *>(d.yleaf), r0, std::min(Rc, R - r0));
    note_launch();
  }
  IGA_CUDA(cudaGetLastError());
}

}  // namespace igabem
