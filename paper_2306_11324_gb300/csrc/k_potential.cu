// Potential evaluation at many points (Sec. 4.4, last part; Sec. 5.3): the scattered field
//   sound-soft  u_s(x) = -SL(t)(x) = -int G(x, y) t(y) dsigma_y
//   sound-hard  u_s(x) =  DL(u)(x) =  int dG/dn_y(x, y) u(y) dsigma_y
// summed over the Gauss points of every element, applied matrix-free by an interpolation fast
// multipole method in physical space: an octree over the bounding cube of the sources (Gauss points)
// and targets (evaluation points), tensor Chebyshev interpolation with q^3 nodes per box (rank O(q^3),
// against O(q^2) for the surface operators of the reference-domain FMM), kernel samples between box
// nodes generated on the fly, the near field summed directly.
//
// Interpolated kernel on an admissible box pair (t, s): G~(x, y) = sum_{a, b} L^t_a(x) G(x_a, y_b)
// L^s_b(y); the double layer differentiates L^s_b(y) along n_y.  Sources carry the weighted density
// rho = w h^2 (density at the Gauss point): monopoles -a rho (soft), dipoles rho n~ (hard).
// Admissibility as on the surface: box radius rho_l = side sqrt(3)/2, admissible iff
// 2 rho_l <= eta_adm (|c_t - c_s| - 2 rho_l) and kappa 2 rho_l <= kappa_cap (when a cap is set).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <unordered_map>
#include <vector>

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

constexpr int POT_MAXQ = 10;

struct PotLevel {
  int n;                    // occupied boxes
  const double *center;     // [n][3]
  double half;              // half side
  const int *child;         // [n][8] child box index on level l + 1 or -1 (l < leaf)
  const int *far_ptr, *far_src;
  double2 *W, *Z;           // multipole / local expansions [n][q^3][R]
};

struct PotArgs {
  int q, Q, R, hard;
  double kappa;
  const double *cheb;       // q points on [-1, 1]
  const double *T1;         // [2][q][q]: parent Lagrange a at child node b (child c per direction)
  // sources (Gauss points) sorted by leaf box
  const double *sy;         // [ns][3]
  const double *sn;         // [ns][3] n~ (hard)
  const double *sa;         // [ns] a
  const int *sidx;          // [ns] original Gauss point index
  const int *src_ptr;       // [nleaf + 1]
  const double2 *rho;       // weighted density [G][R]
  // targets sorted by leaf box
  const double *tx;         // [nt][3]
  const int *tidx;          // [nt] original point index
  const int *tgt_ptr;       // [nleaf + 1]
  const int *near_ptr, *near_src;  // leaf box pairs summed directly
  double2 *u;               // output [n_points][R] (original order)
};

__device__ inline void lagrange_1d(const double *cheb, int q, double x, double *L, double *dL) {
  for (int a = 0; a < q; ++a) {
    double v = 1.0, dv = 0.0;
    for (int k = 0; k < q; ++k) {
      if (k == a) continue;
      const double f = (x - cheb[k]) / (cheb[a] - cheb[k]);
      dv = dv * f + v / (cheb[a] - cheb[k]);
      v *= f;
    }
    L[a] = v;
    if (dL) dL[a] = dv;
  }
}

// source strength seen by interpolation node a of leaf box b: monopole -a rho L_a(y), dipole
// rho n~ . grad L_a(y)
__global__ void k_pot_p2m(PotArgs P, PotLevel L) {
  const int Q = P.Q, q = P.q;
  GRID_STRIDE(o, (long)L.n * Q * P.R) {
    const int b = int(o / (Q * P.R)), a = int((o / P.R) % Q), r = int(o % P.R);
    const int a1 = a / (q * q), a2 = (a / q) % q, a3 = a % q;
    const double *c = L.center + 3 * b;
    const double ih = 1.0 / L.half;
    double2 acc = cmk(0, 0);
    for (int j = P.src_ptr[b]; j < P.src_ptr[b + 1]; ++j) {
      double l1[POT_MAXQ], l2[POT_MAXQ], l3[POT_MAXQ], d1[POT_MAXQ], d2[POT_MAXQ], d3[POT_MAXQ];
      const double *y = P.sy + 3 * (long)j;
      lagrange_1d(P.cheb, q, (y[0] - c[0]) * ih, l1, d1);
      lagrange_1d(P.cheb, q, (y[1] - c[1]) * ih, l2, d2);
      lagrange_1d(P.cheb, q, (y[2] - c[2]) * ih, l3, d3);
      const double2 rho = P.rho[(long)P.sidx[j] * P.R + r];
      double w;
      if (!P.hard) {
        w = -P.sa[j] * l1[a1] * l2[a2] * l3[a3];
      } else {
        const double *n = P.sn + 3 * (long)j;
        w = (n[0] * d1[a1] * l2[a2] * l3[a3] + n[1] * l1[a1] * d2[a2] * l3[a3] + n[2] * l1[a1] * l2[a2] * d3[a3]) * ih;
      }
      acc = cadd(acc, cscale(rho, w));
    }
    L.W[o] = acc;
  }
}

// M2M from level l + 1 into level l: W_p[a] = sum_children sum_b T_c(a, b) W_c[b]
__global__ void k_pot_m2m(PotArgs P, PotLevel Lp, PotLevel Lc) {
  const int Q = P.Q, q = P.q;
  GRID_STRIDE(o, (long)Lp.n * Q * P.R) {
    const int t = int(o / (Q * P.R)), a = int((o / P.R) % Q), r = int(o % P.R);
    const int a1 = a / (q * q), a2 = (a / q) % q, a3 = a % q;
    double2 acc = cmk(0, 0);
    for (int c = 0; c < 8; ++c) {
      const int ch = Lp.child[8 * t + c];
      if (ch < 0) continue;
      const int c1 = c >> 2, c2 = (c >> 1) & 1, c3 = c & 1;
      const double2 *src = Lc.W + (long)ch * Q * P.R;
      for (int b1 = 0; b1 < q; ++b1) {
        const double t1 = P.T1[(c1 * q + a1) * q + b1];
        for (int b2 = 0; b2 < q; ++b2) {
          const double t12 = t1 * P.T1[(c2 * q + a2) * q + b2];
          for (int b3 = 0; b3 < q; ++b3)
            acc = cadd(acc, cscale(src[((b1 * q + b2) * q + b3) * P.R + r], t12 * P.T1[(c3 * q + a3) * q + b3]));
        }
      }
    }
    Lp.W[o] = acc;
  }
}

// M2L on one level: Z_t[a] += sum_{s far} sum_b G(x_a, y_b) W_s[b], one block per target box, the
// samples generated on the fly (T = float: phase split about the box centres as in the surface M2L)
template <class T>
__global__ void __launch_bounds__(256) k_pot_m2l(PotArgs P, PotLevel L) {
  extern __shared__ __align__(16) unsigned char smp[];
  const int t = blockIdx.x, Q = P.Q, q = P.q, R = P.R;
  double2 *Ws = reinterpret_cast<double2 *>(smp);         // [Q][R] source expansion
  double *ys = reinterpret_cast<double *>(Ws + Q * R);    // [Q][3] source node offsets from the target centre
  const double *ct = L.center + 3 * t;
  for (int a0 = 0; a0 < Q; a0 += blockDim.x) {
    const int a = a0 + threadIdx.x;
    const bool va = a < Q;
    double xa[3] = {0, 0, 0};
    if (va) {
      xa[0] = P.cheb[a / (q * q)] * L.half;
      xa[1] = P.cheb[(a / q) % q] * L.half;
      xa[2] = P.cheb[a % q] * L.half;
    }
    double2 acc[8];
    for (int r = 0; r < 8; ++r) acc[r] = cmk(0, 0);
    for (int k = L.far_ptr[t]; k < L.far_ptr[t + 1]; ++k) {
      const int s = L.far_src[k];
      const double *cs = L.center + 3 * s;
      __syncthreads();
      for (int o = threadIdx.x; o < Q * R; o += blockDim.x) Ws[o] = L.W[(long)s * Q * R + o];
      for (int b = threadIdx.x; b < Q; b += blockDim.x) {
        ys[3 * b] = cs[0] - ct[0] + P.cheb[b / (q * q)] * L.half;
        ys[3 * b + 1] = cs[1] - ct[1] + P.cheb[(b / q) % q] * L.half;
        ys[3 * b + 2] = cs[2] - ct[2] + P.cheb[b % q] * L.half;
      }
      __syncthreads();
      if (!va) continue;
      for (int b = 0; b < Q; ++b) {
        const double dx = xa[0] - ys[3 * b], dy = xa[1] - ys[3 * b + 1], dz = xa[2] - ys[3 * b + 2];
        double2 G;
        if constexpr (sizeof(T) == 4) {
          const float r = sqrtf((float)(dx * dx + dy * dy + dz * dz));
          float sn, cs_;
          sincosf((float)P.kappa * r, &sn, &cs_);
          const float f = 0.0795774715459476679f / r;
          G = cmk((double)(cs_ * f), (double)(sn * f));
        } else {
          const double r = sqrt(dx * dx + dy * dy + dz * dz);
          double sn, cs_;
          sincos(P.kappa * r, &sn, &cs_);
          G = cmk(cs_ / (4.0 * IGA_PI * r), sn / (4.0 * IGA_PI * r));
        }
        for (int r = 0; r < R && r < 8; ++r) acc[r] = cadd(acc[r], cmul(G, Ws[b * R + r]));
      }
    }
    if (va)
      for (int r = 0; r < R && r < 8; ++r) {
        double2 *z = L.Z + ((long)t * Q + a) * R + r;
        *z = cadd(*z, acc[r]);
      }
  }
}

// L2L from level l into level l + 1: Z_c[b] += sum_a T_c(a, b) Z_p[a]
__global__ void k_pot_l2l(PotArgs P, PotLevel Lp, PotLevel Lc, const int *parent_of, const int *child_slot) {
  const int Q = P.Q, q = P.q;
  GRID_STRIDE(o, (long)Lc.n * Q * P.R) {
    const int ch = int(o / (Q * P.R)), b = int((o / P.R) % Q), r = int(o % P.R);
    const int t = parent_of[ch], c = child_slot[ch];
    const int c1 = c >> 2, c2 = (c >> 1) & 1, c3 = c & 1, b1 = b / (q * q), b2 = (b / q) % q, b3 = b % q;
    const double2 *src = Lp.Z + (long)t * Q * P.R;
    double2 acc = Lc.Z[o];
    for (int a1 = 0; a1 < q; ++a1) {
      const double t1 = P.T1[(c1 * q + a1) * q + b1];
      for (int a2 = 0; a2 < q; ++a2) {
        const double t12 = t1 * P.T1[(c2 * q + a2) * q + b2];
        for (int a3 = 0; a3 < q; ++a3)
          acc = cadd(acc, cscale(src[((a1 * q + a2) * q + a3) * P.R + r], t12 * P.T1[(c3 * q + a3) * q + b3]));
      }
    }
    Lc.Z[o] = acc;
  }
}

// L2P and the near field at every target: u = sum_a L^t_a(x) Z_t[a] + sum_{near leaf boxes} direct
__global__ void k_pot_eval(PotArgs P, PotLevel L, int nleaf) {
  const int q = P.q, Q = P.Q;
  GRID_STRIDE(o, (long)P.tgt_ptr[nleaf] * P.R) {
    const int j = int(o / P.R), r = int(o % P.R);
    int lo = 0, hi = nleaf;  // leaf box of sorted target j
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.tgt_ptr[mid] <= j) lo = mid;
      else hi = mid;
    }
    const int t = lo;
    const double *x = P.tx + 3 * (long)j;
    double2 acc = cmk(0, 0);
    if (L.Z) {
      const double *c = L.center + 3 * t;
      const double ih = 1.0 / L.half;
      double l1[POT_MAXQ], l2[POT_MAXQ], l3[POT_MAXQ];
      lagrange_1d(P.cheb, q, (x[0] - c[0]) * ih, l1, nullptr);
      lagrange_1d(P.cheb, q, (x[1] - c[1]) * ih, l2, nullptr);
      lagrange_1d(P.cheb, q, (x[2] - c[2]) * ih, l3, nullptr);
      for (int a = 0; a < Q; ++a)
        acc = cadd(acc, cscale(L.Z[((long)t * Q + a) * P.R + r], l1[a / (q * q)] * l2[(a / q) % q] * l3[a % q]));
    }
    for (int k = P.near_ptr[t]; k < P.near_ptr[t + 1]; ++k) {
      const int s = P.near_src[k];
      for (int g = P.src_ptr[s]; g < P.src_ptr[s + 1]; ++g) {
        const double *y = P.sy + 3 * (long)g;
        const double v[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        const double rr = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double sn, cs;
        sincos(P.kappa * rr, &sn, &cs);
        const double2 G = cmk(cs / (4.0 * IGA_PI * rr), sn / (4.0 * IGA_PI * rr));
        const double2 rho = P.rho[(long)P.sidx[g] * P.R + r];
        double2 kv;
        if (!P.hard) {
          kv = cscale(G, -P.sa[g]);
        } else {
          const double *n = P.sn + 3 * (long)g;
          const double vn = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / (rr * rr);
          kv = cscale(cmul(G, cmk(-1.0, P.kappa * rr)), vn);   // G (i kappa r - 1)/r^2 (y - x).n~
        }
        acc = cadd(acc, cmul(kv, rho));
      }
    }
    P.u[(long)P.tidx[j] * P.R + r] = acc;
  }
}

struct Key {
  long long v;
  bool operator==(const Key &o) const { return v == o.v; }
};
struct KeyHash {
  size_t operator()(const Key &k) const { return std::hash<long long>()(k.v); }
};
inline long long pack(int i, int j, int k) { return ((long long)i << 42) | ((long long)j << 21) | (long long)k; }

}  // namespace

}  // namespace igabem

using namespace igabem;

extern "C" int igabem_potential(igabem_problem *P, int n_rhs, const void *density, int n_pts, const double *pts,
                                void *uout) {
  return run_guarded([&] {
    if (!P || !density || !pts || !uout || n_rhs <= 0 || n_pts <= 0) fail(IGABEM_EINVAL, "invalid potential arguments");
    if (n_rhs > 8) fail(IGABEM_EINVAL, "igabem_potential takes at most 8 densities per call");
    IGA_CUDA(cudaSetDevice(P->geom->ctx->device));
    const HostSetup &S = P->S;
    const igabem_options &o = P->opt;
    cudaStream_t st = P->stream;
    const int R = n_rhs, q = std::min(o.cheb_q, POT_MAXQ), Q = q * q * q;
    const long G = (long)S.E * S.ng * S.ng;
    const bool fp32 = o.precision != IGABEM_FP64;
    // sources: the Gauss points (positions, normals, Jacobians from the device tables)
    std::vector<double> gx(3 * G), gn(3 * G), ga(G);
    for (int c = 0; c < 3; ++c) {
      IGA_CUDA(cudaMemcpy(gx.data() + c * G, P->d.gpx + c * G, G * sizeof(double), cudaMemcpyDeviceToHost));
      IGA_CUDA(cudaMemcpy(gn.data() + c * G, P->d.gpn + c * G, G * sizeof(double), cudaMemcpyDeviceToHost));
    }
    IGA_CUDA(cudaMemcpy(ga.data(), P->d.gpa, G * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> tp(3L * n_pts);
    cudaPointerAttributes at{};
    const bool pdev = cudaPointerGetAttributes(&at, pts) == cudaSuccess &&
                      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    IGA_CUDA(cudaMemcpy(tp.data(), pts, tp.size() * sizeof(double), pdev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    // bounding cube
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long i = 0; i < G; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], gx[c * G + i]);
        hi[c] = std::max(hi[c], gx[c * G + i]);
      }
    for (long i = 0; i < n_pts; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], tp[3 * i + c]);
        hi[c] = std::max(hi[c], tp[3 * i + c]);
      }
    double side = 0;
    for (int c = 0; c < 3; ++c) side = std::max(side, hi[c] - lo[c]);
    side *= 1.0 + 1e-9;
    if (!(side > 0)) side = 1.0;
    // leaf level: at most 64 sources per leaf box (depth <= 10); everything near without the FMM
    int D = 0;
    auto cell = [&](double v, int c, int l) {
      const int n = 1 << l;
      return std::min(n - 1, std::max(0, (int)((v - lo[c]) / side * n)));
    };
    if (!o.no_fmm) {
      for (D = 1; D < 10; ++D) {
        std::unordered_map<Key, int, KeyHash> cnt;
        int mx = 0;
        for (long i = 0; i < G; ++i) {
          const int v = ++cnt[Key{pack(cell(gx[i], 0, D), cell(gx[G + i], 1, D), cell(gx[2 * G + i], 2, D))}];
          mx = std::max(mx, v);
        }
        if (mx <= 64) break;
      }
    }
    // occupied boxes per level (leaf level first, then parents)
    std::vector<std::vector<long long>> keys(D + 1);
    std::vector<std::unordered_map<Key, int, KeyHash>> index(D + 1);
    auto leaf_key = [&](const double *x, int c0stride) {
      return pack(cell(x[0], 0, D), cell(x[c0stride], 1, D), cell(x[2 * c0stride], 2, D));
    };
    std::vector<long long> skey(G), tkey(n_pts);
    for (long i = 0; i < G; ++i) skey[i] = leaf_key(&gx[i], (int)G);
    for (long i = 0; i < n_pts; ++i) tkey[i] = leaf_key(&tp[3 * i], 1);
    {
      std::vector<long long> all(skey);
      all.insert(all.end(), tkey.begin(), tkey.end());
      std::sort(all.begin(), all.end());
      all.erase(std::unique(all.begin(), all.end()), all.end());
      keys[D] = all;
    }
    for (int l = D - 1; l >= 0; --l) {
      std::vector<long long> par;
      for (long long k : keys[l + 1]) {
        const int i = int(k >> 42), j = int((k >> 21) & 0x1FFFFF), kk = int(k & 0x1FFFFF);
        par.push_back(pack(i >> 1, j >> 1, kk >> 1));
      }
      std::sort(par.begin(), par.end());
      par.erase(std::unique(par.begin(), par.end()), par.end());
      keys[l] = par;
    }
    for (int l = 0; l <= D; ++l)
      for (size_t b = 0; b < keys[l].size(); ++b) index[l][Key{keys[l][b]}] = (int)b;
    const int nleaf = (int)keys[D].size();
    // sources and targets sorted by leaf box
    std::vector<int> sperm(G), tperm(n_pts);
    for (long i = 0; i < G; ++i) sperm[i] = (int)i;
    for (long i = 0; i < n_pts; ++i) tperm[i] = (int)i;
    std::vector<int> sbox(G), tbox(n_pts);
    for (long i = 0; i < G; ++i) sbox[i] = index[D][Key{skey[i]}];
    for (long i = 0; i < n_pts; ++i) tbox[i] = index[D][Key{tkey[i]}];
    std::stable_sort(sperm.begin(), sperm.end(), [&](int a, int b) { return sbox[a] < sbox[b]; });
    std::stable_sort(tperm.begin(), tperm.end(), [&](int a, int b) { return tbox[a] < tbox[b]; });
    std::vector<int> sptr(nleaf + 1, 0), tptr(nleaf + 1, 0);
    for (long i = 0; i < G; ++i) sptr[sbox[i] + 1]++;
    for (long i = 0; i < n_pts; ++i) tptr[tbox[i] + 1]++;
    for (int b = 0; b < nleaf; ++b) {
      sptr[b + 1] += sptr[b];
      tptr[b + 1] += tptr[b];
    }
    std::vector<double> sy(3 * G), sn(3 * G), sa(G), tx(3L * n_pts);
    for (long j = 0; j < G; ++j) {
      const int i = sperm[j];
      for (int c = 0; c < 3; ++c) {
        sy[3 * j + c] = gx[c * G + i];
        sn[3 * j + c] = gn[c * G + i];
      }
      sa[j] = ga[i];
    }
    for (long j = 0; j < n_pts; ++j)
      for (int c = 0; c < 3; ++c) tx[3 * j + c] = tp[3 * (long)tperm[j] + c];
    // per level: centres, source/target presence (subtree), children
    std::vector<std::vector<double>> cen(D + 1);
    std::vector<std::vector<char>> hs(D + 1), ht(D + 1);
    std::vector<std::vector<int>> child(D + 1);
    for (int l = 0; l <= D; ++l) {
      const int n = (int)keys[l].size();
      cen[l].resize(3L * n);
      hs[l].assign(n, 0);
      ht[l].assign(n, 0);
      child[l].assign(8L * n, -1);
      const double s = side / (1 << l);
      for (int b = 0; b < n; ++b) {
        const long long k = keys[l][b];
        const int idx[3] = {int(k >> 42), int((k >> 21) & 0x1FFFFF), int(k & 0x1FFFFF)};
        for (int c = 0; c < 3; ++c) cen[l][3 * b + c] = lo[c] + (idx[c] + 0.5) * s;
      }
    }
    for (int b = 0; b < nleaf; ++b) {
      hs[D][b] = sptr[b + 1] > sptr[b];
      ht[D][b] = tptr[b + 1] > tptr[b];
    }
    std::vector<std::vector<int>> parent(D + 1), slot(D + 1);
    for (int l = D; l >= 1; --l) {
      const int n = (int)keys[l].size();
      parent[l].resize(n);
      slot[l].resize(n);
      for (int b = 0; b < n; ++b) {
        const long long k = keys[l][b];
        const int i = int(k >> 42), j = int((k >> 21) & 0x1FFFFF), kk = int(k & 0x1FFFFF);
        const int p = index[l - 1][Key{pack(i >> 1, j >> 1, kk >> 1)}];
        const int c = ((i & 1) << 2) | ((j & 1) << 1) | (kk & 1);
        parent[l][b] = p;
        slot[l][b] = c;
        child[l - 1][8 * p + c] = b;
        hs[l - 1][p] |= hs[l][b];
        ht[l - 1][p] |= ht[l][b];
      }
    }
    // dual traversal: admissible pairs per level (CSR by target), near leaf pairs
    const double cap = o.kappa_cap > 0 ? o.kappa_cap : INFINITY;
    std::vector<std::vector<std::pair<int, int>>> far(D + 1);
    std::vector<std::pair<int, int>> near, cand{{0, 0}}, nxt;
    if (!(ht[0][0] && hs[0][0])) cand.clear();
    for (int l = 0; l <= D; ++l) {
      nxt.clear();
      const double rad = side / (1 << l) * std::sqrt(3.0) / 2;
      for (auto [t, s] : cand) {
        const double *ct = &cen[l][3 * t], *cs = &cen[l][3 * s];
        const double dist = std::sqrt((ct[0] - cs[0]) * (ct[0] - cs[0]) + (ct[1] - cs[1]) * (ct[1] - cs[1]) +
                                      (ct[2] - cs[2]) * (ct[2] - cs[2])) - 2 * rad;
        const bool adm = !o.no_fmm && dist > 0 && 2 * rad <= o.eta_adm * dist && o.kappa * 2 * rad <= cap;
        if (adm) {
          far[l].push_back({t, s});
        } else if (l == D) {
          near.push_back({t, s});
        } else {
          for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
              const int ta = child[l][8 * t + a], sb = child[l][8 * s + b];
              if (ta >= 0 && sb >= 0 && ht[l + 1][ta] && hs[l + 1][sb]) nxt.push_back({ta, sb});
            }
        }
      }
      cand.swap(nxt);
    }
    auto csr = [](const std::vector<std::pair<int, int>> &pairs, int n, std::vector<int> &ptr, std::vector<int> &src) {
      ptr.assign(n + 1, 0);
      for (auto &p : pairs) ptr[p.first + 1]++;
      for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
      src.assign(pairs.size(), 0);
      std::vector<int> fill(ptr.begin(), ptr.end() - 1);
      for (auto &p : pairs) src[fill[p.first]++] = p.second;
    };
    std::vector<int> nptr, nsrc;
    csr(near, nleaf, nptr, nsrc);
    int lmin = D + 1;
    for (int l = 0; l <= D; ++l)
      if (!far[l].empty()) lmin = std::min(lmin, l);
    // interpolation tables
    std::vector<double> cheb(q), T1(2L * q * q);
    for (int a = 0; a < q; ++a) cheb[a] = std::cos((2 * a + 1) * M_PI / (2 * q));
    for (int c = 0; c < 2; ++c)
      for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
          const double x = 0.5 * cheb[b] + (c ? 0.5 : -0.5);  // child node b in parent coordinates
          double v = 1.0;
          for (int k = 0; k < q; ++k)
            if (k != a) v *= (x - cheb[k]) / (cheb[a] - cheb[k]);
          T1[(c * q + a) * q + b] = v;
        }
    // device buffers (one allocation)
    std::vector<std::vector<int>> fptr(D + 1), fsrc(D + 1);
    for (int l = 0; l <= D; ++l) csr(far[l], (int)keys[l].size(), fptr[l], fsrc[l]);
    size_t bytes = 0;
    auto add = [&](size_t n) { bytes += (n + 255) & ~size_t(255); };
    add(sizeof(double) * 3 * G); add(sizeof(double) * 3 * G); add(sizeof(double) * G); add(sizeof(int) * G);
    add(sizeof(int) * (nleaf + 1)); add(sizeof(double) * 3 * n_pts); add(sizeof(int) * n_pts);
    add(sizeof(int) * (nleaf + 1)); add(sizeof(int) * (nleaf + 1)); add(sizeof(int) * std::max<size_t>(nsrc.size(), 1));
    add(sizeof(double2) * G * R); add(sizeof(double2) * (size_t)n_pts * R); add(sizeof(double) * q);
    add(sizeof(double) * T1.size());
    for (int l = 0; l <= D; ++l) {
      const size_t n = keys[l].size();
      add(sizeof(double) * 3 * n); add(sizeof(int) * 8 * n); add(sizeof(int) * (n + 1));
      add(sizeof(int) * std::max<size_t>(fsrc[l].size(), 1)); add(sizeof(int) * n); add(sizeof(int) * n);
      if (l >= lmin) {
        add(sizeof(double2) * n * Q * R);
        add(sizeof(double2) * n * Q * R);
      }
    }
    Arena A;
    A.reserve(bytes + 4096);
    auto up = [&](const auto &v) {
      using T = typename std::decay_t<decltype(v)>::value_type;
      T *p = A.get<T>(std::max<size_t>(v.size(), 1));
      if (!v.empty()) IGA_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
      return p;
    };
    try {
      PotArgs PA{};
      PA.q = q;
      PA.Q = Q;
      PA.R = R;
      PA.hard = S.hard ? 1 : 0;
      PA.kappa = o.kappa;
      PA.sy = up(sy);
      PA.sn = up(sn);
      PA.sa = up(sa);
      PA.sidx = up(sperm);
      PA.src_ptr = up(sptr);
      PA.tx = up(tx);
      PA.tidx = up(tperm);
      PA.tgt_ptr = up(tptr);
      PA.near_ptr = up(nptr);
      PA.near_src = up(nsrc);
      double2 *rho = A.get<double2>(G * R);
      PA.rho = rho;
      double2 *ud = A.get<double2>((size_t)n_pts * R);
      PA.u = ud;
      PA.cheb = up(cheb);
      PA.T1 = up(T1);
      std::vector<PotLevel> LV(D + 1);
      std::vector<int *> par_d(D + 1), slot_d(D + 1);
      for (int l = 0; l <= D; ++l) {
        PotLevel &L = LV[l];
        L.n = (int)keys[l].size();
        L.center = up(cen[l]);
        L.half = side / (1 << l) / 2;
        L.child = up(child[l]);
        L.far_ptr = up(fptr[l]);
        L.far_src = up(fsrc[l]);
        par_d[l] = up(parent[l].empty() ? std::vector<int>(1, 0) : parent[l]);
        slot_d[l] = up(slot[l].empty() ? std::vector<int>(1, 0) : slot[l]);
        L.W = L.Z = nullptr;
        if (l >= lmin) {
          L.W = A.get<double2>((size_t)L.n * Q * R);
          L.Z = A.get<double2>((size_t)L.n * Q * R);
          IGA_CUDA(cudaMemsetAsync(L.Z, 0, sizeof(double2) * (size_t)L.n * Q * R, st));
        }
      }
      launch_density(P->d, S, o, R, static_cast<const double *>(density), reinterpret_cast<double *>(rho), st);
      if (lmin <= D) {
        k_pot_p2m<<<grid_for((long)nleaf * Q * R), 256, 0, st>>>(PA, LV[D]);
        note_launch();
        for (int l = D - 1; l >= lmin; --l) {
          k_pot_m2m<<<grid_for((long)LV[l].n * Q * R), 256, 0, st>>>(PA, LV[l], LV[l + 1]);
          note_launch();
        }
        const size_t smem = sizeof(double2) * Q * R + sizeof(double) * 3 * Q;
        for (int l = lmin; l <= D; ++l) {
          if (far[l].empty()) continue;
          if (fp32) {
            IGA_CUDA(set_max_dynamic_smem(k_pot_m2l<float>, smem));
            k_pot_m2l<float><<<LV[l].n, 256, smem, st>>>(PA, LV[l]);
          } else {
            IGA_CUDA(set_max_dynamic_smem(k_pot_m2l<double>, smem));
            k_pot_m2l<double><<<LV[l].n, 256, smem, st>>>(PA, LV[l]);
          }
          note_launch();
        }
        for (int l = lmin; l < D; ++l) {
          k_pot_l2l<<<grid_for((long)LV[l + 1].n * Q * R), 256, 0, st>>>(PA, LV[l], LV[l + 1], par_d[l + 1], slot_d[l + 1]);
          note_launch();
        }
      }
      k_pot_eval<<<grid_for((long)n_pts * R), 256, 0, st>>>(PA, LV[D], nleaf);
      note_launch();
      IGA_CUDA(cudaGetLastError());
      cudaPointerAttributes ua{};
      const bool udev = cudaPointerGetAttributes(&ua, uout) == cudaSuccess &&
                        (ua.type == cudaMemoryTypeDevice || ua.type == cudaMemoryTypeManaged);
      cudaGetLastError();
      IGA_CUDA(cudaMemcpyAsync(uout, ud, sizeof(double2) * (size_t)n_pts * R,
                               udev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
      IGA_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaStreamSynchronize(st);
      A.release();
      throw;
    }
    A.release();
  });
}
