// M2L: couplings of admissible cluster pairs (Sec. 4.4) with the kernel samples between the
// Chebyshev nodes generated on the fly, FP64 and FP32.
//
// Layout: one thread block per target cluster (all levels in one launch), its warps share the
// target's interaction list; lane l owns target nodes a0 + l and a0 + l + 32 of a chunk of 64 target
// nodes (levels with q*q > 64 take several chunks, each streaming the interaction list again) and
// generates their rows of the coupling block in registers while streaming the source nodes of one pair
// from shared memory (broadcast reads).  Accumulation is blocked: q source nodes per partial sum, q
// partial sums per pair, then the pairs; the warps are reduced through shared memory at the end of a
// chunk.  Each level has its own q (level-adaptive interpolation).
//
// FP32 phase split: the sample phase kappa r is formed as kappa |D| (D = c_t - c_s, the distance of
// the two cluster centres, taken in FP64 once per pair and reduced mod 2 pi) plus kappa (r - |D|),
// with r - |D| = (2 D.delta + |delta|^2)/(r + |D|) computed in FP32 from the node offsets
// delta = (x_a - c_t) - (y_b - c_s).  The FP32 error of the phase is then of the order of the
// cluster size times the unit roundoff instead of kappa r times it, and the factor
// exp(i kappa |D|) multiplies the pair's partial sums once.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "k_common.cuh"
#include "kernels.h"
#include "k_m2l.cuh"

namespace igabem {

namespace {

constexpr int M2L_WARPS = 8;
constexpr double TWO_PI = 6.283185307179586476925286766559;

struct M2LLevel {
  const int *far_ptr, *far_src;
  const double *nodes;   // FP64 [7][n q^2]: x, n~, a
  const float *nodes32;  // FP32 [7][n q^2]: x - c, n~, a
  const float *pc;       // FP32 pair constants [n_far][8]: D, |D|, |D|^2, cos, sin of kappa|D| (FP32 path)
  const double2 *xhat;
  const float2 *xhat32;  // FP32 copy of xhat (the FP32 kernels read it)
  const void *stored;    // stored coupling blocks of the level (m2l_stored) or nullptr
  double2 *yhat;
  int n;                 // clusters on the level
  int first;             // first block index of the level in the flattened grid
  int q, Q;              // interpolation points per direction / per cluster on the level
};

struct M2LArgs {
  M2LLevel lev[16];
  int nlev;
  int QS;                // source nodes per warp in shared memory (the largest Q of the launch)
  int CR, R;
  double kappa, eta;
  bool hard;
};

// per-source-node data in shared memory
template <class T> struct SrcNode {
  T dy[3], ny[3], ay, Ddy, Dny, pad;
};

// Kernel sample(s) between target node (x, n~x, ax) and source node (y, n~y, ay).
//   soft: ks = a_y G'(r)/r (x-y).n~x - i eta a_x a_y G                       (K' - i eta V)
//   hard: kk = a_x G'(r)/r (y-x).n~y (K),  g = G (the six W channels)
// e = (cos, sin) of the phase carried by the sample; for FP32 the pair factor exp(i kappa |D|) is
// applied by the caller.
template <class T, int NCR, bool HARD>
__global__ void __launch_bounds__(32 * M2L_WARPS) k_m2l_rows(M2LArgs A, int cr0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr bool F32 = std::is_same<T, float>::value;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // locate the level of this block
  int li = 0;
  while (li + 1 < A.nlev && (int)blockIdx.x >= A.lev[li + 1].first) ++li;
  const M2LLevel &L = A.lev[li];
  const int t = blockIdx.x - L.first;
  const int Q = L.Q, q = L.q, QS = A.QS;
  const long NQ = (long)L.n * Q;
  const int ncr = min(NCR, A.CR - cr0);
  // shared memory: per warp QS source nodes + QS x NCR source coefficients; then the reduction area
  SrcNode<T> *src = reinterpret_cast<SrcNode<T> *>(smraw) + warp * QS;
  C2<T> *xs = reinterpret_cast<C2<T> *>(reinterpret_cast<SrcNode<T> *>(smraw) + M2L_WARPS * QS) + warp * QS * NCR;
  double2 *red = reinterpret_cast<double2 *>(smraw);
  const T kappa = (T)A.kappa, eta = (T)A.eta;
  const T inv4pi = (T)(0.25 / IGA_PI);
  for (int a0 = 0; a0 < Q; a0 += 64) {
    // target rows of this lane in the chunk
    T tx[2][3], tn[2][3], ta[2];
    bool valid[2];
    for (int k = 0; k < 2; ++k) {
      int a = a0 + lane + 32 * k;
      valid[k] = a < Q;
      long ia = (long)t * Q + (valid[k] ? a : 0);
      for (int c = 0; c < 3; ++c) {
        tx[k][c] = F32 ? (T)L.nodes32[c * NQ + ia] : (T)L.nodes[c * NQ + ia];
        tn[k][c] = F32 ? (T)L.nodes32[(3 + c) * NQ + ia] : (T)L.nodes[(3 + c) * NQ + ia];
      }
      ta[k] = F32 ? (T)L.nodes32[6 * NQ + ia] : (T)L.nodes[6 * NQ + ia];
    }
    C2<T> tot[2][NCR];
    for (int k = 0; k < 2; ++k)
      for (int c = 0; c < NCR; ++c) tot[k][c] = c2((T)0, (T)0);
    for (int kk = L.far_ptr[t] + warp; kk < L.far_ptr[t + 1]; kk += M2L_WARPS) {
      const int s = L.far_src[kk];
      // pair constants (FP32 path): D = c_t - c_s, |D|, |D|^2 and exp(i kappa |D|), from the set-up
      T D[3] = {0, 0, 0}, Dn = 0, D2 = 0;
      C2<T> e0 = c2((T)1, (T)0);
      if constexpr (F32) {
        const float4 p0 = reinterpret_cast<const float4 *>(L.pc)[2 * kk];
        const float4 p1 = reinterpret_cast<const float4 *>(L.pc)[2 * kk + 1];
        D[0] = p0.x; D[1] = p0.y; D[2] = p0.z; Dn = p0.w;
        D2 = p1.x;
        e0 = c2(p1.y, p1.z);
      }
      // stage the source nodes and coefficients of this pair
      __syncwarp();
      for (int b = lane; b < Q; b += 32) {
        long ib = (long)s * Q + b;
        SrcNode<T> sn;
        for (int c = 0; c < 3; ++c) {
          sn.dy[c] = F32 ? (T)L.nodes32[c * NQ + ib] : (T)L.nodes[c * NQ + ib];
          sn.ny[c] = F32 ? (T)L.nodes32[(3 + c) * NQ + ib] : (T)L.nodes[(3 + c) * NQ + ib];
        }
        sn.ay = F32 ? (T)L.nodes32[6 * NQ + ib] : (T)L.nodes[6 * NQ + ib];
        sn.Ddy = D[0] * sn.dy[0] + D[1] * sn.dy[1] + D[2] * sn.dy[2];
        sn.Dny = D[0] * sn.ny[0] + D[1] * sn.ny[1] + D[2] * sn.ny[2];
        src[b] = sn;
        for (int c = 0; c < ncr; ++c) {
          if constexpr (F32) {
            const float2 v = L.xhat32[ib * A.CR + cr0 + c];
            xs[b * NCR + c] = c2((T)v.x, (T)v.y);
          } else {
            const double2 v = L.xhat[ib * A.CR + cr0 + c];
            xs[b * NCR + c] = c2((T)v.x, (T)v.y);
          }
        }
      }
      __syncwarp();
      for (int k = 0; k < 2; ++k) {
        if (!valid[k]) continue;
        const T Ddx = D[0] * tx[k][0] + D[1] * tx[k][1] + D[2] * tx[k][2];
        const T Dnx = D[0] * tn[k][0] + D[1] * tn[k][1] + D[2] * tn[k][2];
        C2<T> acc[NCR];
        for (int c = 0; c < NCR; ++c) acc[c] = c2((T)0, (T)0);
        for (int b1 = 0; b1 < q; ++b1) {
          C2<T> part[NCR];
          for (int c = 0; c < NCR; ++c) part[c] = c2((T)0, (T)0);
          for (int b2 = 0; b2 < q; ++b2) {
            const int b = b1 * q + b2;
            const SrcNode<T> &y = src[b];
            T d0 = tx[k][0] - y.dy[0], d1 = tx[k][1] - y.dy[1], d2 = tx[k][2] - y.dy[2];
            T r2, ir, r, cph, sph;
            T dn_x, dn_y;  // (x-y).n~x and (x-y).n~y
            if constexpr (F32) {
              // delta = d; x - y = D + delta
              T Dd = Ddx - y.Ddy;
              T dd = d0 * d0 + d1 * d1 + d2 * d2;
              T num = (T)2 * Dd + dd;
              r2 = D2 + num;
              ir = rsqrtf((float)r2);
              r = r2 * ir;
              T del = __fdividef((float)num, (float)(r + Dn));
              T ph = kappa * del;
              T kq = rintf((float)(ph * (T)0.15915494309189535));
              ph = fmaf(-(float)kq, 6.28318548202514648f, (float)ph);
              ph = fmaf(-(float)kq, -1.7484556e-07f, (float)ph);
              float sf, cf;
              __sincosf((float)ph, &sf, &cf);
              cph = cf;
              sph = sf;
              dn_x = Dnx + d0 * tn[k][0] + d1 * tn[k][1] + d2 * tn[k][2];
              dn_y = y.Dny + d0 * y.ny[0] + d1 * y.ny[1] + d2 * y.ny[2];
            } else {
              r2 = d0 * d0 + d1 * d1 + d2 * d2;
              ir = rsqrt((double)r2);
              r = r2 * ir;
              double sd, cd;
              sincos(A.kappa * (double)r, &sd, &cd);
              cph = cd;
              sph = sd;
              dn_x = d0 * tn[k][0] + d1 * tn[k][1] + d2 * tn[k][2];
              dn_y = d0 * y.ny[0] + d1 * y.ny[1] + d2 * y.ny[2];
            }
            const T f = ir * inv4pi;
            const T kr = kappa * r;
            const T g2 = f * ir * ir;
            // G = e f;  G'(r)/r = e (-1 + i kappa r) f / r^2
            const C2<T> G = c2(cph * f, sph * f);
            const C2<T> dG = c2((-cph - sph * kr) * g2, (-sph + cph * kr) * g2);
            if (!HARD) {
              const T w1 = y.ay * dn_x, w2 = ta[k] * y.ay * eta;
              // ks = dG w1 - i eta a_x a_y G
              const C2<T> ks = c2(dG.x * w1 + G.y * w2, dG.y * w1 - G.x * w2);
              for (int c = 0; c < NCR; ++c) part[c] = fma2(ks, xs[b * NCR + c], part[c]);
            } else {
              const T w1 = -ta[k] * dn_y;  // a_x (y-x).n~y
              const C2<T> kk2 = c2(dG.x * w1, dG.y * w1);
              for (int c = 0; c < NCR; ++c) {
                const int ch = (cr0 + c) / A.R;
                part[c] = fma2(ch == 0 ? kk2 : G, xs[b * NCR + c], part[c]);
              }
            }
          }
          for (int c = 0; c < NCR; ++c) acc[c] = add(acc[c], part[c]);
        }
        for (int c = 0; c < NCR; ++c) tot[k][c] = fma2(e0, acc[c], tot[k][c]);
      }
    }
    // reduce over the warps (the staging area is reused)
    __syncthreads();
    for (int k = 0; k < 2; ++k)
      for (int c = 0; c < NCR; ++c) {
        int a = lane + 32 * k;
        red[(warp * 64 + a) * NCR + c] = make_double2((double)tot[k][c].x, (double)tot[k][c].y);
      }
    __syncthreads();
    const int na = min(64, Q - a0);
    for (int o = threadIdx.x; o < na * ncr; o += blockDim.x) {
      int a = o / ncr, c = o % ncr;
      double2 sum = make_double2(0, 0);
      for (int w = 0; w < M2L_WARPS; ++w) {
        double2 v = red[(w * 64 + a) * NCR + c];
        sum.x += v.x;
        sum.y += v.y;
      }
      L.yhat[((long)t * Q + a0 + a) * A.CR + cr0 + c] = sum;
    }
    __syncthreads();  // the reduction area is the staging area of the next chunk
  }
}

// ---- stored coupling blocks (m2l_stored): the same kernel samples (node_sample, the samples of the
// multi-column M2L) generated once per problem, then streamed by every product ----

// one thread block per admissible pair k of a level: every entry S_k[type][b][a] (column-major: the
// target node a runs fastest) with the pair factor exp(i kappa |D|) folded in (FP32 path)
template <class T>
__global__ void __launch_bounds__(256) k_m2l_fill(M2LLevel L, bool hard, double kappa, double eta,
                                                  C2<T> *__restrict__ out) {
  constexpr bool F32 = std::is_same<T, float>::value;
  const long kk = blockIdx.x;
  const int Q = L.Q, ntype = hard ? 2 : 1;
  const long NQ = (long)L.n * Q;
  int lo = 0, hi = L.n;  // target t with far_ptr[t] <= kk < far_ptr[t + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (L.far_ptr[mid] <= kk) lo = mid;
    else hi = mid;
  }
  const int t = lo, s = L.far_src[kk];
  T D[3] = {0, 0, 0}, Dn = 0, D2 = 0;
  C2<T> e0 = c2((T)1, (T)0);
  if constexpr (F32) {
    const float *pc = L.pc + 8 * kk;
    D[0] = pc[0]; D[1] = pc[1]; D[2] = pc[2]; Dn = pc[3]; D2 = pc[4];
    e0 = c2(pc[5], pc[6]);
  }
  C2<T> *S = out + kk * (long)ntype * Q * Q;
  for (int o = threadIdx.x; o < ntype * Q * Q; o += blockDim.x) {
    const int ty = o / (Q * Q), b = (o / Q) % Q, a = o % Q;
    T X[7], Y[7];
    for (int c = 0; c < 7; ++c) {
      X[c] = F32 ? (T)L.nodes32[c * NQ + (long)t * Q + a] : (T)L.nodes[c * NQ + (long)t * Q + a];
      Y[c] = F32 ? (T)L.nodes32[c * NQ + (long)s * Q + b] : (T)L.nodes[c * NQ + (long)s * Q + b];
    }
    const int type = hard ? (ty == 0 ? 1 : 2) : 0;
    const C2<T> v = node_sample<T>(type, X, X + 3, X[6], Y, Y + 3, Y[6], D, Dn, D2, (T)kappa, (T)eta);
    S[o] = F32 ? mul(e0, v) : v;
  }
}

// cp.async of one coupling-block entry (8 or 16 bytes) into shared memory; src_bytes = 0 fills zeros
template <int BYTES>
__device__ inline void cp_async_zfill(void *dst, const void *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES), "r"(src_bytes)
               : "memory");
}
__device__ inline void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// M2L from the stored blocks: one block per target cluster, warps over the interaction list, lane rows
// a0 + lane and a0 + lane + 32.  The stored rows stream through a per-warp ring of D shared-memory
// slots filled by asynchronous copies (row b + D - 1 is requested while row b is used), so that each
// warp keeps D rows of the block in flight instead of one load per lane.
template <class T, int NCR, bool HARD, int D>
__global__ void __launch_bounds__(32 * M2L_WARPS) k_m2l_stored(M2LArgs A, int cr0) {
  extern __shared__ __align__(16) unsigned char smst[];
  constexpr bool F32 = std::is_same<T, float>::value;
  constexpr int ntype = HARD ? 2 : 1, ES = sizeof(C2<T>);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int li = 0;
  while (li + 1 < A.nlev && (int)blockIdx.x >= A.lev[li + 1].first) ++li;
  const M2LLevel &L = A.lev[li];
  const int t = blockIdx.x - L.first;
  const int Q = L.Q, q = L.q, QS = A.QS;
  const int ncr = min(NCR, A.CR - cr0);
  C2<T> *xs = reinterpret_cast<C2<T> *>(smst) + warp * QS * NCR;
  C2<T> *ring = reinterpret_cast<C2<T> *>(smst) + M2L_WARPS * QS * NCR + warp * D * ntype * 64;
  double2 *red = reinterpret_cast<double2 *>(smst);
  const C2<T> *Sall = reinterpret_cast<const C2<T> *>(L.stored);
  const C2<T> zero = c2((T)0, (T)0);
  for (int a0 = 0; a0 < Q; a0 += 64) {
    C2<T> tot0[NCR], tot1[NCR];
    for (int c = 0; c < NCR; ++c) tot0[c] = tot1[c] = zero;
    for (int kk = L.far_ptr[t] + warp; kk < L.far_ptr[t + 1]; kk += M2L_WARPS) {
      const int s = L.far_src[kk];
      const C2<T> *Sk = Sall + (long)kk * ntype * Q * Q;
      // rows 0 .. D - 2 of the block requested before x_s is staged
      auto issue = [&](int b) {
        C2<T> *slot = ring + (b % D) * ntype * 64;
#pragma unroll
        for (int ty = 0; ty < ntype; ++ty) {
          const C2<T> *src = Sk + ((long)ty * Q + b) * Q;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int col = a0 + lane + 32 * h;
            const bool ok = col < Q;
            cp_async_zfill<ES>(slot + ty * 64 + lane + 32 * h, ok ? src + col : src, ok ? ES : 0);
          }
        }
      };
      __syncwarp();  // the previous pair's reads of the ring and of x_s are done
#pragma unroll
      for (int i = 0; i < D - 1; ++i) {
        if (i < Q) issue(i);
        cp_async_commit_group();
      }
      for (int b = lane; b < Q; b += 32) {
        const long ib = (long)s * Q + b;
        for (int c = 0; c < ncr; ++c) {
          if constexpr (F32) {
            const float2 v = L.xhat32[ib * A.CR + cr0 + c];
            xs[b * NCR + c] = c2((T)v.x, (T)v.y);
          } else {
            const double2 v = L.xhat[ib * A.CR + cr0 + c];
            xs[b * NCR + c] = c2((T)v.x, (T)v.y);
          }
        }
      }
      for (int b1 = 0; b1 < q; ++b1) {
        C2<T> p0[NCR], p1[NCR];
        for (int c = 0; c < NCR; ++c) p0[c] = p1[c] = zero;
        for (int b2 = 0; b2 < q; ++b2) {
          const int b = b1 * q + b2;
          cp_async_wait_group<D - 2>();  // row b has landed (this lane's copies)
          __syncwarp();                  // ... and every lane's
          const C2<T> *slot = ring + (b % D) * ntype * 64;
          const C2<T> s0a = slot[lane], s0b = slot[lane + 32];
          // the staged x_s values of row b (broadcast to the warp), two columns per 16-byte load in FP32
          C2<T> xv[NCR];
          if constexpr (F32 && NCR % 2 == 0) {
            const float4 *xp = reinterpret_cast<const float4 *>(xs + b * NCR);
#pragma unroll
            for (int c = 0; c < NCR / 2; ++c) {
              const float4 v = xp[c];
              xv[2 * c] = c2((T)v.x, (T)v.y);
              xv[2 * c + 1] = c2((T)v.z, (T)v.w);
            }
          } else {
#pragma unroll
            for (int c = 0; c < NCR; ++c) xv[c] = xs[b * NCR + c];
          }
          if (!HARD) {
#pragma unroll
            for (int c = 0; c < NCR; ++c) {
              p0[c] = fma2(s0a, xv[c], p0[c]);
              p1[c] = fma2(s0b, xv[c], p1[c]);
            }
          } else {
            const C2<T> s1a = slot[64 + lane], s1b = slot[64 + lane + 32];
#pragma unroll
            for (int c = 0; c < NCR; ++c) {
              const bool k0 = (cr0 + c) / A.R == 0;
              p0[c] = fma2(k0 ? s0a : s1a, xv[c], p0[c]);
              p1[c] = fma2(k0 ? s0b : s1b, xv[c], p1[c]);
            }
          }
          // the slot of row b - 1 is free (every lane passed this iteration's __syncwarp)
          if (b + D - 1 < Q) issue(b + D - 1);
          cp_async_commit_group();
        }
        for (int c = 0; c < NCR; ++c) {
          tot0[c] = add(tot0[c], p0[c]);
          tot1[c] = add(tot1[c], p1[c]);
        }
      }
      cp_async_wait_group<0>();
    }
    __syncthreads();
    for (int c = 0; c < NCR; ++c) {
      red[(warp * 64 + lane) * NCR + c] = make_double2((double)tot0[c].x, (double)tot0[c].y);
      red[(warp * 64 + lane + 32) * NCR + c] = make_double2((double)tot1[c].x, (double)tot1[c].y);
    }
    __syncthreads();
    const int na = min(64, Q - a0);
    for (int o = threadIdx.x; o < na * ncr; o += blockDim.x) {
      const int a = o / ncr, c = o % ncr;
      double2 sum = make_double2(0, 0);
      for (int w = 0; w < M2L_WARPS; ++w) {
        const double2 v = red[(w * 64 + a) * NCR + c];
        sum.x += v.x;
        sum.y += v.y;
      }
      L.yhat[((long)t * Q + a0 + a) * A.CR + cr0 + c] = sum;
    }
    __syncthreads();
  }
}

// Multi-column M2L: per target cluster and column chunk, every coupling block S_ts (q^2 x q^2) is
// generated once into shared memory and applied to the chunk's columns of xhat_s with a register
// tiled product (4 x 4 complex outputs per thread).  A chunk lies within one channel, so one kernel
// type per block.
constexpr int GEMM_T = 16;  // thread tile grid 16 x 16

template <class T>
__global__ void __launch_bounds__(256) k_m2l_gemm(M2LArgs A, int Wc) {
  extern __shared__ __align__(16) unsigned char smg[];
  constexpr bool F32 = std::is_same<T, float>::value;
  int li = 0;
  while (li + 1 < A.nlev && (int)blockIdx.x >= A.lev[li + 1].first) ++li;
  const M2LLevel &L = A.lev[li];
  const int t = blockIdx.x - L.first;
  const int Q = L.Q;  // <= 64 (4 x 16 thread rows)
  const long NQ = (long)L.n * Q;
  const int cr0 = blockIdx.y * Wc, ch = cr0 / A.R;
  const int type = A.hard ? (ch == 0 ? 1 : 2) : 0;
  C2<T> *S = reinterpret_cast<C2<T> *>(smg);            // [Q][Q]
  C2<T> *Xs = S + Q * Q;                                 // [Q][Wc]
  T *tn = reinterpret_cast<T *>(Xs + Q * Wc);            // target nodes [Q][8]
  T *sn = tn + Q * 8;                                    // source nodes [Q][8]
  const T kappa = (T)A.kappa, eta = (T)A.eta;
  for (int a = threadIdx.x; a < Q; a += blockDim.x) {
    long ia = (long)t * Q + a;
    for (int c = 0; c < 7; ++c) tn[a * 8 + c] = F32 ? (T)L.nodes32[c * NQ + ia] : (T)L.nodes[c * NQ + ia];
  }
  const int ty = threadIdx.x / GEMM_T, tx = threadIdx.x % GEMM_T;
  C2<T> acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = c2((T)0, (T)0);
  for (int kk = L.far_ptr[t]; kk < L.far_ptr[t + 1]; ++kk) {
    const int s = L.far_src[kk];
    T D[3] = {0, 0, 0}, Dn = 0, D2 = 0;
    C2<T> e0 = c2((T)1, (T)0);
    if constexpr (F32) {
      const float4 p0 = reinterpret_cast<const float4 *>(L.pc)[2 * kk];
      const float4 p1 = reinterpret_cast<const float4 *>(L.pc)[2 * kk + 1];
      D[0] = p0.x; D[1] = p0.y; D[2] = p0.z; Dn = p0.w;
      D2 = p1.x;
      e0 = c2(p1.y, p1.z);
    }
    __syncthreads();  // previous contraction done with S, Xs, sn
    for (int b = threadIdx.x; b < Q; b += blockDim.x) {
      long ib = (long)s * Q + b;
      for (int c = 0; c < 7; ++c) sn[b * 8 + c] = F32 ? (T)L.nodes32[c * NQ + ib] : (T)L.nodes[c * NQ + ib];
    }
    for (int i = threadIdx.x; i < Q * Wc; i += blockDim.x) {
      int b = i / Wc, c = i % Wc;
      C2<T> xv;
      if constexpr (F32) {
        const float2 v = L.xhat32[((long)s * Q + b) * A.CR + cr0 + c];
        xv = c2((T)v.x, (T)v.y);
      } else {
        const double2 v = L.xhat[((long)s * Q + b) * A.CR + cr0 + c];
        xv = c2((T)v.x, (T)v.y);
      }
      // the pair factor exp(i kappa |D|) is folded into the source coefficients
      Xs[i] = F32 ? mul(e0, xv) : xv;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
      int a = i / Q, b = i % Q;
      const T *X = tn + a * 8, *Y = sn + b * 8;
      S[i] = node_sample<T>(type, X, X + 3, X[6], Y, Y + 3, Y[6], D, Dn, D2, kappa, eta);
    }
    __syncthreads();
    C2<T> part[4][4];  // this pair's sums (blocked accumulation)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) part[i][j] = c2((T)0, (T)0);
    for (int b = 0; b < Q; ++b) {
      C2<T> sv[4], xv[4];
      for (int i = 0; i < 4; ++i) {
        int a = ty + GEMM_T * i;
        sv[i] = a < Q ? S[a * Q + b] : c2((T)0, (T)0);
      }
      for (int j = 0; j < 4; ++j) {
        int c = tx + GEMM_T * j;
        xv[j] = c < Wc ? Xs[b * Wc + c] : c2((T)0, (T)0);
      }
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) part[i][j] = fma2(sv[i], xv[j], part[i][j]);
    }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] = add(acc[i][j], part[i][j]);
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int a = ty + GEMM_T * i, c = tx + GEMM_T * j;
      if (a < Q && c < Wc)
        L.yhat[((long)t * Q + a) * A.CR + cr0 + c] = make_double2((double)acc[i][j].x, (double)acc[i][j].y);
    }
}

// pair constants, per admissible pair k of a level (CSR order):
// [D (3), |D|, |D|^2, cos(kappa |D|), sin(kappa |D|), sigma] with D = c_t - c_s in FP64 and sigma a power
// of two that scales the pair's coupling block to at most 2^12 in magnitude (used by the FP16 operands
// of the tensor-core M2L).  sigma comes from a bound on the kernel samples over the two clusters' nodes:
// with rho the largest node distance from the cluster centre and a_max the largest Jacobian,
// |x - y| lies in [|D| - rho_t - rho_s, |D| + rho_t + rho_s] and every kernel type is at most
// (1 + kappa r_hi)(1 + a_t)(1 + a_s)(1 + |eta|) / (4 pi r_lo).
// per cluster: rho = the largest node distance from the centre, a_max = the largest node Jacobian
__global__ void k_cluster_extent(const double *__restrict__ nodes, const double *__restrict__ center, int n, int Q,
                                 double2 *__restrict__ ext) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const long NQ = (long)n * Q;
  double rho = 0.0, amax = 0.0;
  for (int a = 0; a < Q; ++a) {
    const long i = (long)c * Q + a;
    const double dx = nodes[i] - center[3 * c], dy = nodes[NQ + i] - center[3 * c + 1],
                 dz = nodes[2 * NQ + i] - center[3 * c + 2];
    rho = fmax(rho, sqrt(dx * dx + dy * dy + dz * dz));
    amax = fmax(amax, nodes[6 * NQ + i]);
  }
  ext[c] = make_double2(rho, amax);
}

// one thread per admissible pair k (CSR order), its target t from the row pointers
__global__ void k_pair_consts(const int *__restrict__ far_ptr, const int *__restrict__ far_src,
                              const double *__restrict__ center, const double2 *__restrict__ ext, int n, long nfar,
                              double kappa, double eta, float *__restrict__ pc) {
  const long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k >= nfar) return;
  int lo = 0, hi = n;  // t with far_ptr[t] <= k < far_ptr[t + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (far_ptr[mid] <= k) lo = mid;
    else hi = mid;
  }
  const int t = lo, s = far_src[k];
  double D[3] = {center[3 * t] - center[3 * s], center[3 * t + 1] - center[3 * s + 1],
                 center[3 * t + 2] - center[3 * s + 2]};
  double nD = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
  double sn, cs;
  sincos(fmod(kappa * nD, TWO_PI), &sn, &cs);
  const double2 et = ext[t], es = ext[s];
  const double r_lo = fmax(nD - et.x - es.x, 1e-3 * nD), r_hi = nD + et.x + es.x;
  const double bound = (1.0 + kappa * r_hi) * (1.0 + et.y) * (1.0 + es.y) * (1.0 + fabs(eta)) / (4.0 * IGA_PI * r_lo);
  float *o = pc + 8L * k;
  o[0] = (float)D[0]; o[1] = (float)D[1]; o[2] = (float)D[2]; o[3] = (float)nD;
  o[4] = (float)(nD * nD); o[5] = (float)cs; o[6] = (float)sn;
  o[7] = (float)exp2(12.0 - ceil(log2(bound)));
}

// shared memory of the row kernel: per warp QS source nodes and their NCR coefficients (or the
// reduction area)
size_t rows_smem(int QS, int ncr, bool fp32) {
  const size_t node = fp32 ? sizeof(SrcNode<float>) : sizeof(SrcNode<double>);
  const size_t coef = fp32 ? sizeof(C2<float>) : sizeof(C2<double>);
  return std::max((size_t)M2L_WARPS * QS * node + (size_t)M2L_WARPS * QS * ncr * coef,
                  (size_t)M2L_WARPS * 64 * ncr * sizeof(double2));
}

template <class T, int NCR, bool HARD>
void launch_rows(const M2LArgs &A, int nblocks, cudaStream_t st) {
  const size_t smem = rows_smem(A.QS, NCR, std::is_same<T, float>::value);
  auto kfn = k_m2l_rows<T, NCR, HARD>;
  IGA_CUDA(set_max_dynamic_smem(kfn, smem));
  for (int cr0 = 0; cr0 < A.CR; cr0 += NCR) {
    kfn<<<nblocks, 32 * M2L_WARPS, smem, st>>>(A, cr0);
    note_launch();
  }
}

template <class T, int NCR, bool HARD, int D>
size_t stored_smem(const M2LArgs &A) {
  const size_t pts = (size_t)M2L_WARPS * (A.QS * NCR + D * (HARD ? 2 : 1) * 64) * sizeof(C2<T>);
  return std::max(pts, (size_t)M2L_WARPS * 64 * NCR * sizeof(double2));
}

template <class T, int NCR, bool HARD>
void launch_stored(const M2LArgs &A, int nblocks, cudaStream_t st) {
  // eight rows in flight per warp where the shared memory allows, else three
  const bool deep = stored_smem<T, NCR, HARD, 8>(A) <= 200 * 1024;
  const size_t smem = deep ? stored_smem<T, NCR, HARD, 8>(A) : stored_smem<T, NCR, HARD, 3>(A);
  auto kfn = deep ? k_m2l_stored<T, NCR, HARD, 8> : k_m2l_stored<T, NCR, HARD, 3>;
  IGA_CUDA(set_max_dynamic_smem(kfn, smem));
  for (int cr0 = 0; cr0 < A.CR; cr0 += NCR) {
    kfn<<<nblocks, 32 * M2L_WARPS, smem, st>>>(A, cr0);
    note_launch();
  }
}

template <class T>
void launch_stored_typed(const M2LArgs &A, int nblocks, cudaStream_t st) {
  if (A.hard) launch_stored<T, 7, true>(A, nblocks, st);
  else if (A.CR == 1) launch_stored<T, 1, false>(A, nblocks, st);
  else if (A.CR == 2) launch_stored<T, 2, false>(A, nblocks, st);
  else if (A.CR < 8) launch_stored<T, 4, false>(A, nblocks, st);
  else launch_stored<T, 8, false>(A, nblocks, st);
}

template <class T>
void launch_typed(const M2LArgs &A, int nblocks, cudaStream_t st) {
  if (A.hard) {
    launch_rows<T, 7, true>(A, nblocks, st);
  } else if (A.CR == 1) {
    launch_rows<T, 1, false>(A, nblocks, st);
  } else if (A.CR == 2) {
    launch_rows<T, 2, false>(A, nblocks, st);
  } else if (A.CR < 8 || !std::is_same<T, float>::value) {
    launch_rows<T, 4, false>(A, nblocks, st);
  } else {
    launch_rows<T, 8, false>(A, nblocks, st);
  }
}

}  // namespace

void launch_pair_consts(const DeviceProblem &d, const HostSetup &S, double kappa, double eta, cudaStream_t st) {
  for (int l = S.lmin; l <= S.L; ++l) {
    int n = S.lev[l].n;
    const long nfar = (long)S.lev[l].far_src.size();
    k_cluster_extent<<<(n + 127) / 128, 128, 0, st>>>(d.nodes[l], d.centers[l], n, S.lev[l].q * S.lev[l].q,
                                                      reinterpret_cast<double2 *>(d.cext[l]));
    note_launch();
    if (nfar == 0) continue;
    k_pair_consts<<<(int)((nfar + 255) / 256), 256, 0, st>>>(d.far_ptr[l], d.far_src[l], d.centers[l],
                                                             reinterpret_cast<const double2 *>(d.cext[l]), n, nfar,
                                                             kappa, eta, d.pairc[l]);
    note_launch();
  }
  IGA_CUDA(cudaGetLastError());
}

size_t m2l_stored_entries(const HostSetup &S, int l) {
  const size_t Q = (size_t)S.lev[l].q * S.lev[l].q;
  return S.lev[l].far_src.size() * Q * Q * (S.hard ? 2 : 1);
}

void launch_m2l_fill(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, cudaStream_t st) {
  const bool fp32 = o.precision != IGABEM_FP64;
  for (int l = S.lmin; l <= S.L; ++l) {
    const long nfar = (long)S.lev[l].far_src.size();
    if (nfar == 0) continue;
    M2LLevel L{};
    L.far_ptr = d.far_ptr[l];
    L.far_src = d.far_src[l];
    L.nodes = d.nodes[l];
    L.nodes32 = d.nodes32[l];
    L.pc = d.pairc[l];
    L.n = S.lev[l].n;
    L.q = S.lev[l].q;
    L.Q = L.q * L.q;
    if (fp32)
      k_m2l_fill<float><<<(unsigned)nfar, 256, 0, st>>>(L, S.hard, o.kappa, o.eta_cfie,
                                                        reinterpret_cast<C2<float> *>(d.m2ls[l]));
    else
      k_m2l_fill<double><<<(unsigned)nfar, 256, 0, st>>>(L, S.hard, o.kappa, o.eta_cfie,
                                                         reinterpret_cast<C2<double> *>(d.m2ls[l]));
    note_launch();
  }
  IGA_CUDA(cudaGetLastError());
}

bool m2l_rows_supported(const HostSetup &S, const igabem_options &o, int R) {
  if (S.L - S.lmin + 1 > 16) return false;
  int QS = 0;
  for (int l = S.lmin; l <= S.L; ++l) QS = std::max(QS, S.lev[l].q * S.lev[l].q);
  if (R > 1 && QS <= 64) return true;  // the multi-column kernel
  const bool fp32 = o.precision != IGABEM_FP64;
  const int CR = (S.hard ? 7 : 1) * R;
  const int ncr = S.hard ? 7 : (CR == 1 ? 1 : CR == 2 ? 2 : (CR < 8 || !fp32) ? 4 : 8);
  return rows_smem(QS, ncr, fp32) <= (size_t)max_optin_smem();
}

void launch_m2l_rows(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                     bool fp32, cudaStream_t st) {
  M2LArgs A;
  A.QS = 0;
  A.R = R;
  A.CR = (S.hard ? 7 : 1) * R;
  A.kappa = o.kappa;
  A.eta = o.eta_cfie;
  A.hard = S.hard;
  A.nlev = 0;
  int nblocks = 0;
  for (int l = S.lmin; l <= S.L; ++l) {
    M2LLevel &L = A.lev[A.nlev++];
    L.far_ptr = d.far_ptr[l];
    L.far_src = d.far_src[l];
    L.nodes = d.nodes[l];
    L.nodes32 = d.nodes32[l];
    L.pc = d.pairc[l];
    L.xhat = reinterpret_cast<const double2 *>(d.xhat[l]);
    L.xhat32 = d.xhat32.empty() ? nullptr : d.xhat32[l];
    L.stored = d.m2ls.empty() ? nullptr : d.m2ls[l];
    L.yhat = reinterpret_cast<double2 *>(d.yhat[l]);
    L.n = S.lev[l].n;
    L.first = nblocks;
    L.q = S.lev[l].q;
    L.Q = L.q * L.q;
    A.QS = std::max(A.QS, L.Q);
    nblocks += S.lev[l].n;
  }
  if (A.nlev > 0 && A.lev[0].stored) {  // stored coupling blocks: stream them
    if (fp32) launch_stored_typed<float>(A, nblocks, st);
    else launch_stored_typed<double>(A, nblocks, st);
  } else if (R > 1 && A.QS <= 64) {
    // column chunk: the largest divisor of R not above 64 (chunks never straddle two channels)
    int Wc = 1;
    for (int w = std::min(R, 64); w >= 1; --w)
      if (R % w == 0) {
        Wc = w;
        break;
      }
    const size_t tsz = fp32 ? sizeof(float) : sizeof(double);
    size_t smem = (size_t)A.QS * A.QS * 2 * tsz + (size_t)A.QS * Wc * 2 * tsz + (size_t)A.QS * 16 * tsz;
    dim3 grid(nblocks, A.CR / Wc);
    if (fp32) {
      IGA_CUDA(set_max_dynamic_smem(k_m2l_gemm<float>, smem));
      k_m2l_gemm<float><<<grid, 256, smem, st>>>(A, Wc);
    } else {
      IGA_CUDA(set_max_dynamic_smem(k_m2l_gemm<double>, smem));
      k_m2l_gemm<double><<<grid, 256, smem, st>>>(A, Wc);
    }
    note_launch();
  } else if (fp32) {
    launch_typed<float>(A, nblocks, st);
  } else {
    launch_typed<double>(A, nblocks, st);
  }
  IGA_CUDA(cudaGetLastError());
}

}  // namespace igabem
