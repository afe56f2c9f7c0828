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

// Near-field SpMV for many columns: one thread block per (target leaf, chunk of 64 columns).  Each
// near block and the source leaf's coefficients (converted to the block's precision) are staged in
// shared memory; each thread owns a 4 x 4 tile of (local function, column) outputs.  One block's sum
// is formed in the storage precision, the blocks are summed in FP64, as in k_near_spmv2.
constexpr int NM_COLS = 64;

template <class BT>
__global__ void __launch_bounds__(256) k_near_mrhs(LeafArgs A, const int *__restrict__ near_ptr,
                                                   const int *__restrict__ near_src, const BT *__restrict__ blk,
                                                   const double2 *__restrict__ xX, double2 *__restrict__ yleaf,
                                                   int nL) {
  using RT = decltype(BT::x);
  extern __shared__ __align__(16) unsigned char smn[];
  BT *Bs = reinterpret_cast<BT *>(smn);  // [nL (source)][nL (target)]
  BT *Xs = Bs + nL * nL;                 // [nL][NM_COLS]
  const int t = blockIdx.x, r0 = blockIdx.y * NM_COLS, Rc = min(NM_COLS, A.R - r0);
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int ti = threadIdx.x >> 4, tr = threadIdx.x & 15;
  double2 acc[4][4];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) acc[m][n] = make_double2(0.0, 0.0);
  for (int k = near_ptr[t]; k < near_ptr[t + 1]; ++k) {
    const int s = near_src[k];
    const int js = s / (nlL * nlL), cx = (s / nlL) % nlL, cy = s % nlL;
    const long base = ((long)js * A.nb + cx * e1) * A.nb + cy * e1;
    __syncthreads();  // the previous block's products are done
    const BT *Bk = blk + (size_t)k * nL * nL;
    for (int e = threadIdx.x; e < nL * nL; e += blockDim.x) Bs[e] = Bk[e];
    for (int e = threadIdx.x; e < nL * NM_COLS; e += blockDim.x) {
      const int jj = e / NM_COLS, c = e % NM_COLS, al = jj / A.nL1, be = jj % A.nL1;
      BT v;
      v.x = 0;
      v.y = 0;
      if (c < Rc) {
        const double2 xd = xX[(base + (long)al * A.nb + be) * A.R + r0 + c];
        v.x = (RT)xd.x;
        v.y = (RT)xd.y;
      }
      Xs[e] = v;
    }
    __syncthreads();
    RT px[4][4], py[4][4];
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) px[m][n] = py[m][n] = 0;
    for (int jj = 0; jj < nL; ++jj) {
      BT bv[4], xv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int i = ti + 16 * m;
        if (i < nL) {
          bv[m] = Bs[jj * nL + i];
        } else {
          bv[m].x = 0;
          bv[m].y = 0;
        }
      }
#pragma unroll
      for (int n = 0; n < 4; ++n) xv[n] = Xs[jj * NM_COLS + tr + 16 * n];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          px[m][n] += bv[m].x * xv[n].x - bv[m].y * xv[n].y;
          py[m][n] += bv[m].x * xv[n].y + bv[m].y * xv[n].x;
        }
    }
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n) {
        acc[m][n].x += (double)px[m][n];
        acc[m][n].y += (double)py[m][n];
      }
  }
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      const int i = ti + 16 * m, c = tr + 16 * n;
      if (i < nL && c < Rc) yleaf[((size_t)t * nL + i) * A.R + r0 + c] = acc[m][n];
    }
}

// Near-field SpMV for up to 16 columns per block: one thread block per (target leaf, column chunk),
// one thread per (local function i, CPT adjacent columns).  The near blocks of the target's list are
// staged in shared memory by asynchronous copies (cp.async), double buffered: block k + 1 is in flight
// while block k is multiplied, one barrier per block; the source coefficients (converted to the block
// precision) go through registers.  One block's sum is formed in the storage precision, the blocks
// are summed in FP64 (as in k_near_spmv2).
template <int BYTES>
__device__ inline void cp_async(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <class BT, int CPT>
__global__ void __launch_bounds__(576) k_near_cols(LeafArgs A, const int *__restrict__ near_ptr,
                                                   const int *__restrict__ near_src, const BT *__restrict__ blk,
                                                   const double2 *__restrict__ xX, const float2 *__restrict__ x32,
                                                   double2 *__restrict__ yleaf, int nL, int Rc) {
  using RT = decltype(BT::x);
  extern __shared__ __align__(16) unsigned char smk[];
  BT *Bs = reinterpret_cast<BT *>(smk);              // [2][nL * nL] (block column-major: [j][i])
  BT *Xs = Bs + 2 * nL * nL;                         // [2][nL][Rc]
  const int t = blockIdx.x, r0 = blockIdx.y * Rc, rc = min(Rc, A.R - r0);
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int nthr = blockDim.x, nB = nL * nL, nX = nL * Rc;
  const int i = threadIdx.x % nL, cg = threadIdx.x / nL, c0 = cg * CPT;
  const bool active = cg * CPT < Rc;
  const int kb = near_ptr[t], ke = near_ptr[t + 1];
  BT rx[2];
  auto issue_block = [&](int k, int buf) {  // asynchronous copy of near block k into buffer buf
    const BT *Bk = blk + (size_t)k * nB;
    BT *dst = Bs + buf * nB;
    for (int e = threadIdx.x; e < nB; e += nthr) cp_async<sizeof(BT)>(dst + e, Bk + e);
    cp_async_commit();
  };
  auto fetch_x = [&](int k) {  // this thread's share of block k's source coefficients
    const int s = near_src[k];
    const int js = s / (nlL * nlL), cx = (s / nlL) % nlL, cy = s % nlL;
    const long base = ((long)js * A.nb + cx * e1) * A.nb + cy * e1;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = threadIdx.x + u * nthr;
      rx[u].x = 0;
      rx[u].y = 0;
      if (e < nX) {
        const int jj = e / Rc, c = e % Rc, al = jj / A.nL1, be = jj % A.nL1;
        if (c < rc) {
          const long ix = (base + (long)al * A.nb + be) * A.R + r0 + c;
          if constexpr (sizeof(RT) == 4) {  // FP32 blocks: the FP32 copy of the input
            const float2 xf = x32[ix];
            rx[u].x = xf.x;
            rx[u].y = xf.y;
          } else {
            const double2 xd = xX[ix];
            rx[u].x = xd.x;
            rx[u].y = xd.y;
          }
        }
      }
    }
  };
  auto store_x = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = threadIdx.x + u * nthr;
      if (e < nX) Xs[buf * nX + e] = rx[u];
    }
  };
  // the blocks' sums: FP64 for FP64 blocks; for FP32 blocks an FP32 sum with a compensation term
  // (Neumaier), as accurate as an FP64 sum here without FP64 arithmetic
  double2 acc[CPT];
  float2 sh[CPT], sl[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    acc[c] = make_double2(0.0, 0.0);
    sh[c] = sl[c] = make_float2(0.f, 0.f);
  }
  auto nsum = [](float &hi, float &lo, float v) {
    const float t = hi + v;
    lo += fabsf(hi) >= fabsf(v) ? (hi - t) + v : (v - t) + hi;
    hi = t;
  };
  if (kb < ke) {
    issue_block(kb, 0);
    fetch_x(kb);
    store_x(0);
    cp_async_wait_all();
  }
  __syncthreads();
  if (kb + 1 < ke) {
    issue_block(kb + 1, 1);
    fetch_x(kb + 1);
  }
  for (int k = kb; k < ke; ++k) {
    const int cur = (k - kb) & 1;
    if (active) {
      RT px[CPT], py[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) px[c] = py[c] = 0;
      const BT *B = Bs + cur * nB + i;
      const BT *X = Xs + cur * nX + c0;
      for (int jj = 0; jj < nL; ++jj) {
        const BT bv = B[jj * nL];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          if (c0 + c >= Rc) break;  // odd chunk width: the last thread of a row has one column
          const BT xv = X[jj * Rc + c];
          px[c] += bv.x * xv.x - bv.y * xv.y;
          py[c] += bv.x * xv.y + bv.y * xv.x;
        }
      }
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        if constexpr (sizeof(RT) == 4) {
          nsum(sh[c].x, sl[c].x, (float)px[c]);
          nsum(sh[c].y, sl[c].y, (float)py[c]);
        } else {
          acc[c].x += (double)px[c];
          acc[c].y += (double)py[c];
        }
      }
    }
    if (k + 1 < ke) store_x(cur ^ 1);  // coefficients of block k + 1
    cp_async_wait_all();                // block k + 1 has landed
    __syncthreads();                    // ... for every thread; buffer cur is free
    if (k + 2 < ke) {
      issue_block(k + 2, cur);
      fetch_x(k + 2);
    }
  }
  if (active) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (sizeof(RT) == 4) acc[c] = make_double2((double)sh[c].x + (double)sl[c].x, (double)sh[c].y + (double)sl[c].y);
      if (c0 + c < rc) yleaf[((size_t)t * nL + i) * A.R + r0 + c0 + c] = acc[c];
    }
  }
}

// launch of k_near_cols: columns per thread 2 (1 for a single column), chunks of up to 16 columns
template <class BT>
bool launch_near_cols(const LeafArgs &A, const int *near_ptr, const int *near_src, const BT *blk, const double2 *xX,
                      const float2 *x32, double2 *yleaf, int nleaf, int nL, int R, cudaStream_t st) {
  const int Rc = std::min(R, 16), cpt = Rc >= 2 ? 2 : 1;
  const int threads = ((nL * ((Rc + cpt - 1) / cpt) + 31) / 32) * 32;
  if (threads > 576 || (size_t)nL * Rc > 2 * (size_t)threads) return false;
  const size_t smem = sizeof(BT) * 2 * ((size_t)nL * nL + (size_t)nL * Rc);
  dim3 grid(nleaf, (R + Rc - 1) / Rc);
  if (cpt == 2) {
    IGA_CUDA(set_max_dynamic_smem(k_near_cols<BT, 2>, smem));
    k_near_cols<BT, 2><<<grid, threads, smem, st>>>(A, near_ptr, near_src, blk, xX, x32, yleaf, nL, Rc);
  } else {
    IGA_CUDA(set_max_dynamic_smem(k_near_cols<BT, 1>, smem));
    k_near_cols<BT, 1><<<grid, threads, smem, st>>>(A, near_ptr, near_src, blk, xX, x32, yleaf, nL, Rc);
  }
  note_launch();
  return true;
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

// Leaf moment matrices (Sec. 4.4), set up once per problem: M_t[k][a C + c] = sum over the leaf's
// Gauss points g of L_a(g) w_c(g, k) for the leaf-local B-spline k = al nL1 + be, with
//   w_0 = W phi_k,  w_{1+d} = W (ft_d d_s phi_k - fs_d d_t phi_k),  w_{4+d} = W n~_d phi_k
// (W = w_1 w_2 h^2; channels 1..6 only for sound-hard).  P2M applies M_t to the leaf's coefficients;
// L2P applies its transpose with the channel factors of the tested operator, so both passes are dense
// products over many columns.  Tensor form: the a1 sum first (shared memory Tq[k][a1][g2]).
template <class T>
__global__ void k_leaf_moments(LeafArgs A, T *__restrict__ M) {
  extern __shared__ double smm[];
  const int t = blockIdx.x;
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int j = t / (nlL * nlL), cx = (t / nlL) % nlL, cy = t % nlL;
  const int c0x = cx * e1, c0y = cy * e1;
  const int nG = e1 * A.ng, q = A.q, Q = q * q, C = A.C, nL1 = A.nL1, nL = nL1 * nL1, QC = Q * C;
  double *Tq = smm;  // [nL][q][nG]
  for (int c = 0; c < C; ++c) {
    for (int i = threadIdx.x; i < nL * q * nG; i += blockDim.x) {
      const int k = i / (q * nG), a1 = (i / nG) % q, g2 = i % nG;
      const int al = k / nL1, be = k % nL1;
      const double pb = leaf_phi(A, A.phi1, c0y, g2, be);
      const double dpb = A.hard ? leaf_phi(A, A.dphi1, c0y, g2, be) : 0.0;
      double sum = 0.0;
      if (pb != 0.0 || dpb != 0.0) {
        for (int g1 = 0; g1 < nG; ++g1) {
          const double pa = leaf_phi(A, A.phi1, c0x, g1, al);
          const double dpa = A.hard ? leaf_phi(A, A.dphi1, c0x, g1, al) : 0.0;
          if (pa == 0.0 && dpa == 0.0) continue;
          const double W = A.gw[g1 % A.ng] * A.gw[g2 % A.ng] * A.h * A.h;
          double w;
          if (c == 0) {
            w = W * pa * pb;
          } else {
            const long e = ((long)j * A.n1 + c0x + g1 / A.ng) * A.n1 + c0y + g2 / A.ng;
            const long iq = e * A.ng * A.ng + (g1 % A.ng) * A.ng + g2 % A.ng;
            if (c <= 3)
              w = W * (A.gft[(c - 1) * A.gst + iq] * dpa * pb - A.gfs[(c - 1) * A.gst + iq] * pa * dpb);
            else
              w = W * A.gpn[(c - 4) * A.gst + iq] * pa * pb;
          }
          sum += A.LG1[g1 * q + a1] * w;
        }
      }
      Tq[i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nL * Q; i += blockDim.x) {
      const int k = i / Q, a = i % Q, a1 = a / q, a2 = a % q;
      double sum = 0.0;
      for (int g2 = 0; g2 < nG; ++g2) sum += A.LG1[g2 * q + a2] * Tq[(k * q + a1) * nG + g2];
      M[((size_t)t * nL + k) * QC + a * C + c] = (T)sum;
    }
    __syncthreads();
  }
}

// complex value type of the moment products
template <class T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };

// P2M for many columns: xhat_t[a C + c][r] = sum_k M_t[k][a C + c] x_t[k][r], one thread block per
// (leaf, chunk of 16 NN columns), 64-row chunks of the output with a 4 x NN register tile per thread.
template <class T, int NN>
__global__ void __launch_bounds__(256) k_p2m_mrhs(LeafArgs A, const T *__restrict__ M, const double2 *__restrict__ xX,
                                                  const float2 *__restrict__ x32, double2 *__restrict__ xhat) {
  using V = typename CT<T>::type;
  constexpr int NC = 16 * NN;
  extern __shared__ __align__(16) unsigned char smp[];
  const int nL1 = A.nL1, nL = nL1 * nL1, QC = A.q * A.q * A.C;
  V *Xs = reinterpret_cast<V *>(smp);        // [nL][NC]
  T *Ms = reinterpret_cast<T *>(Xs + nL * NC);  // [nL][64]
  const int t = blockIdx.x, r0 = blockIdx.y * NC, Rc = min(NC, A.R - r0);
  const int nlL = 1 << A.L, e1 = 1 << A.b;
  const int j = t / (nlL * nlL), cx = (t / nlL) % nlL, cy = t % nlL;
  const long base = ((long)j * A.nb + cx * e1) * A.nb + cy * e1;
  const int ti = threadIdx.x >> 4, tr = threadIdx.x & 15;
  for (int e = threadIdx.x; e < nL * NC; e += blockDim.x) {
    const int k = e / NC, c = e % NC, al = k / nL1, be = k % nL1;
    V v;
    v.x = 0;
    v.y = 0;
    if (c < Rc) {
      const long ix = (base + (long)al * A.nb + be) * A.R + r0 + c;
      if constexpr (sizeof(T) == 4) {
        const float2 xf = x32[ix];
        v.x = xf.x;
        v.y = xf.y;
      } else {
        const double2 xd = xX[ix];
        v.x = xd.x;
        v.y = xd.y;
      }
    }
    Xs[e] = v;
  }
  for (int i0 = 0; i0 < QC; i0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < nL * 64; e += blockDim.x) {
      const int k = e / 64, i = i0 + e % 64;
      Ms[e] = i < QC ? M[((size_t)t * nL + k) * QC + i] : (T)0;
    }
    __syncthreads();
    T px[4][NN], py[4][NN];
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < NN; ++n) px[m][n] = py[m][n] = 0;
    for (int k = 0; k < nL; ++k) {
      T mv[4];
      V xv[NN];
#pragma unroll
      for (int m = 0; m < 4; ++m) mv[m] = Ms[k * 64 + ti + 16 * m];
#pragma unroll
      for (int n = 0; n < NN; ++n) xv[n] = Xs[k * NC + tr + 16 * n];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          px[m][n] += mv[m] * xv[n].x;
          py[m][n] += mv[m] * xv[n].y;
        }
    }
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < NN; ++n) {
        const int i = i0 + ti + 16 * m, c = tr + 16 * n;
        if (i < QC && c < Rc) xhat[((size_t)t * QC + i) * A.R + r0 + c] = make_double2((double)px[m][n], (double)py[m][n]);
      }
  }
}

// L2P for many columns: y_leaf[t][k][r] += sum_{a, c} M_t[k][a C + c] sigma_c yhat_t[a C + c][r] with the
// channel factors of the tested operator: soft sigma_0 = 1; hard sigma_0 = -1 (the -K part),
// sigma_{1..3} = -i eta (curl test of -i eta W), sigma_{4..6} = i eta kappa^2 (its normal part).
// One thread block per (leaf, chunk of 16 NN columns), a 4 x NN register tile per thread.
template <class T, int NN>
__global__ void __launch_bounds__(256) k_l2p_mrhs(LeafArgs A, const T *__restrict__ M, const double2 *__restrict__ yhat,
                                                  const float2 *__restrict__ y32, double2 *__restrict__ yleaf) {
  using V = typename CT<T>::type;
  constexpr int NC = 16 * NN;
  extern __shared__ __align__(16) unsigned char smq[];
  const int nL1 = A.nL1, nL = nL1 * nL1, C = A.C, QC = A.q * A.q * C;
  V *Ys = reinterpret_cast<V *>(smq);           // [64 rows a C + c][NC]
  T *Ms = reinterpret_cast<T *>(Ys + 64 * NC);  // [nL][64 rows]
  const int t = blockIdx.x, r0 = blockIdx.y * NC, Rc = min(NC, A.R - r0);
  const int ti = threadIdx.x >> 4, tr = threadIdx.x & 15;
  const T k2e = (T)(A.kappa * A.kappa * A.eta), eta = (T)A.eta;
  T px[4][NN], py[4][NN];
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < NN; ++n) px[m][n] = py[m][n] = 0;
  for (int i0 = 0; i0 < QC; i0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * NC; e += blockDim.x) {
      const int i = i0 + e / NC, c = e % NC;
      V v;
      v.x = 0;
      v.y = 0;
      if (i < QC && c < Rc) {
        const size_t iy = ((size_t)t * QC + i) * A.R + r0 + c;
        V yv;
        if constexpr (sizeof(T) == 4) {
          const float2 f = y32[iy];
          yv.x = f.x;
          yv.y = f.y;
        } else {
          const double2 f = yhat[iy];
          yv.x = f.x;
          yv.y = f.y;
        }
        const int ch = i % C;
        if (!A.hard) {
          v = yv;
        } else if (ch == 0) {
          v.x = -yv.x;
          v.y = -yv.y;
        } else if (ch <= 3) {
          v.x = eta * yv.y;
          v.y = -eta * yv.x;
        } else {
          v.x = -k2e * yv.y;
          v.y = k2e * yv.x;
        }
      }
      Ys[e] = v;
    }
    for (int e = threadIdx.x; e < nL * 64; e += blockDim.x) {
      const int k = e / 64, i = i0 + e % 64;
      Ms[e] = i < QC ? M[((size_t)t * nL + k) * QC + i] : (T)0;
    }
    __syncthreads();
    const int iw = min(64, QC - i0);
    for (int i = 0; i < iw; ++i) {
      T mv[4];
      V yv[NN];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int k = ti + 16 * m;
        mv[m] = k < nL ? Ms[k * 64 + i] : (T)0;
      }
#pragma unroll
      for (int n = 0; n < NN; ++n) yv[n] = Ys[i * NC + tr + 16 * n];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          px[m][n] += mv[m] * yv[n].x;
          py[m][n] += mv[m] * yv[n].y;
        }
    }
  }
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < NN; ++n) {
      const int k = ti + 16 * m, c = tr + 16 * n;
      if (k < nL && c < Rc) {
        double2 *dst = yleaf + ((size_t)t * nL + k) * A.R + r0 + c;
        *dst = make_double2(dst->x + (double)px[m][n], dst->y + (double)py[m][n]);
      }
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
  if (R <= 16 && launch_near_cols<double2>(A, d.ident_ptr, d.ident_src, reinterpret_cast<const double2 *>(d.binv),
                                           reinterpret_cast<const double2 *>(d.xX), nullptr,
                                           reinterpret_cast<double2 *>(d.yleaf), nleaf, S.nL, R, st)) {
    IGA_CUDA(cudaGetLastError());
    return;
  }
  if (R >= 8 && S.nL <= 64) {
    dim3 grid(nleaf, (R + NM_COLS - 1) / NM_COLS);
    const size_t smem = sizeof(double2) * ((size_t)S.nL * S.nL + (size_t)S.nL * NM_COLS);
    IGA_CUDA(set_max_dynamic_smem(k_near_mrhs<double2>, smem));
    k_near_mrhs<double2><<<grid, threads, smem, st>>>(A, d.ident_ptr, d.ident_src,
                                                      reinterpret_cast<const double2 *>(d.binv),
                                                      reinterpret_cast<const double2 *>(d.xX),
                                                      reinterpret_cast<double2 *>(d.yleaf), S.nL);
    note_launch();
    IGA_CUDA(cudaGetLastError());
    return;
  }
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
  if (R <= 16) {  // staged, double-buffered blocks with one thread per (function, column pair)
    const bool ok = d.blk32 ? launch_near_cols<float2>(A, d.near_ptr, d.near_src, reinterpret_cast<const float2 *>(d.blk32),
                                                       reinterpret_cast<const double2 *>(d.xX), d.xX32,
                                                       reinterpret_cast<double2 *>(d.yleaf), nleaf, S.nL, R, st)
                            : launch_near_cols<double2>(A, d.near_ptr, d.near_src, reinterpret_cast<const double2 *>(d.blk),
                                                        reinterpret_cast<const double2 *>(d.xX), nullptr,
                                                        reinterpret_cast<double2 *>(d.yleaf), nleaf, S.nL, R, st);
    if (ok) {
      IGA_CUDA(cudaGetLastError());
      return;
    }
  }
  if (R >= 8 && S.nL <= 64) {
    dim3 grid(nleaf, (R + NM_COLS - 1) / NM_COLS);
    if (d.blk32) {
      const size_t smem = sizeof(float2) * ((size_t)S.nL * S.nL + (size_t)S.nL * NM_COLS);
      IGA_CUDA(set_max_dynamic_smem(k_near_mrhs<float2>, smem));
      k_near_mrhs<float2><<<grid, threads, smem, st>>>(A, d.near_ptr, d.near_src,
                                                       reinterpret_cast<const float2 *>(d.blk32),
                                                       reinterpret_cast<const double2 *>(d.xX),
                                                       reinterpret_cast<double2 *>(d.yleaf), S.nL);
    } else {
      const size_t smem = sizeof(double2) * ((size_t)S.nL * S.nL + (size_t)S.nL * NM_COLS);
      IGA_CUDA(set_max_dynamic_smem(k_near_mrhs<double2>, smem));
      k_near_mrhs<double2><<<grid, threads, smem, st>>>(A, d.near_ptr, d.near_src,
                                                        reinterpret_cast<const double2 *>(d.blk),
                                                        reinterpret_cast<const double2 *>(d.xX),
                                                        reinterpret_cast<double2 *>(d.yleaf), S.nL);
    }
    note_launch();
    IGA_CUDA(cudaGetLastError());
    return;
  }
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

size_t leaf_moment_entries(const HostSetup &S) {
  return (size_t)S.lev[S.L].n * S.nL1 * S.nL1 * S.q * S.q * (S.hard ? 7 : 1);
}

bool leaf_moments_supported(const HostSetup &S) { return S.nL1 * S.nL1 <= 64; }

void launch_leaf_moments(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, 1);
  const int nG = (1 << S.b) * S.ng;
  const size_t smem = sizeof(double) * (size_t)S.nL1 * S.nL1 * S.q * nG;
  if (d.lm32) {
    IGA_CUDA(set_max_dynamic_smem(k_leaf_moments<float>, smem));
    k_leaf_moments<float><<<S.lev[S.L].n, 256, smem, st>>>(A, d.lm32);
  } else {
    IGA_CUDA(set_max_dynamic_smem(k_leaf_moments<double>, smem));
    k_leaf_moments<double><<<S.lev[S.L].n, 256, smem, st>>>(A, d.lm64);
  }
  note_launch();
  IGA_CUDA(cudaGetLastError());
}

void launch_p2m(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st) {
  LeafArgs A = leaf_args(d, S, o, R);
  const int nleaf = S.lev[S.L].n;
  if (R >= 8 && (d.lm32 || d.lm64)) {
    const int nn = R <= 16 ? 1 : 4, nc = 16 * nn;
    dim3 grid(nleaf, (R + nc - 1) / nc);
    const size_t nl = (size_t)S.nL1 * S.nL1;
    auto go = [&](auto kfn, const auto *M, size_t smem) {
      IGA_CUDA(set_max_dynamic_smem(kfn, smem));
      kfn<<<grid, 256, smem, st>>>(A, M, reinterpret_cast<const double2 *>(d.xX), d.xX32,
                                   reinterpret_cast<double2 *>(d.xhat[S.L]));
    };
    if (d.lm32) {
      const size_t smem = nl * nc * sizeof(float2) + nl * 64 * sizeof(float);
      if (nn == 1) go(k_p2m_mrhs<float, 1>, d.lm32, smem);
      else go(k_p2m_mrhs<float, 4>, d.lm32, smem);
    } else {
      const size_t smem = nl * nc * sizeof(double2) + nl * 64 * sizeof(double);
      if (nn == 1) go(k_p2m_mrhs<double, 1>, d.lm64, smem);
      else go(k_p2m_mrhs<double, 4>, d.lm64, smem);
    }
    note_launch();
    IGA_CUDA(cudaGetLastError());
    return;
  }
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
  if (R >= 8 && (d.lm32 || d.lm64)) {
    const int nn = R <= 16 ? 1 : 4, nc = 16 * nn;
    dim3 grid(nleaf, (R + nc - 1) / nc);
    const size_t nl = (size_t)S.nL1 * S.nL1 * 64;
    auto go = [&](auto kfn, const auto *M, size_t smem) {
      IGA_CUDA(set_max_dynamic_smem(kfn, smem));
      kfn<<<grid, 256, smem, st>>>(A, M, reinterpret_cast<const double2 *>(d.yhat[S.L]), d.y32,
                                   reinterpret_cast<double2 *>(d.yleaf));
    };
    if (d.lm32) {
      const size_t smem = 64 * (size_t)nc * sizeof(float2) + nl * sizeof(float);
      if (nn == 1) go(k_l2p_mrhs<float, 1>, d.lm32, smem);
      else go(k_l2p_mrhs<float, 4>, d.lm32, smem);
    } else {
      const size_t smem = 64 * (size_t)nc * sizeof(double2) + nl * sizeof(double);
      if (nn == 1) go(k_l2p_mrhs<double, 1>, d.lm64, smem);
      else go(k_l2p_mrhs<double, 4>, d.lm64, smem);
    }
    note_launch();
    IGA_CUDA(cudaGetLastError());
    return;
  }
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
