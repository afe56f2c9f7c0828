// Host set-up of a discretised CFIE problem: geometry extraction, quadrature rules, spaces,
// touching element pairs, cluster tree and block partition (Sec. 3 and 4 of Doelz, Harbrecht and
// Multerer).  Plain C++; everything here runs once per problem.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <numeric>
#include <thread>
#include <string>
#include <unordered_map>

#include "internal.h"

namespace igabem {

// ----------------------------------------------------------------------------------------------
// Gauss-Legendre rule: roots of P_n by Newton's method from cos(pi (i + 3/4) / (n + 1/2)),
// weights 2 / ((1 - x^2) P_n'(x)^2), mapped to [0, 1].

void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
    }
    x[i] = 0.5 * (1.0 - z);  // ascending on [0, 1]
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ----------------------------------------------------------------------------------------------
// B-splines (Sec. 3.1): the p+1 functions that do not vanish on knot span mu, by the triangular
// Cox-de Boor scheme, and their first derivatives.

static int find_span(const std::vector<double> &kn, int p, double x) {
  int k = (int)kn.size() - p - 1;
  if (x >= kn[k]) return k - 1;
  int lo = p, hi = k;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < kn[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

constexpr int MAX_DEG = 15;  // largest B-spline degree the host tables handle

static void span_basis(const std::vector<double> &kn, int p, int mu, double x, double *N,
                       double *dN) {
  double left[MAX_DEG + 2], right[MAX_DEG + 2], prev[MAX_DEG + 2];
  N[0] = 1.0;
  for (int d = 1; d <= p; ++d) {
    left[d] = x - kn[mu + 1 - d];
    right[d] = kn[mu + d] - x;
    if (d == p && dN) std::copy(N, N + p, prev);
    double saved = 0.0;
    for (int r = 0; r < d; ++r) {
      double den = right[r + 1] + left[d - r];
      double t = den != 0.0 ? N[r] / den : 0.0;
      N[r] = saved + right[r + 1] * t;
      saved = left[d - r] * t;
    }
    N[d] = saved;
  }
  if (!dN) return;
  if (p == 0) {
    dN[0] = 0.0;
    return;
  }
  // d/dx b_j^p = p/(xi_{j+p}-xi_j) b_j^{p-1} - p/(xi_{j+p+1}-xi_{j+1}) b_{j+1}^{p-1},
  // j = mu-p+i; prev[i'] = b_{mu-p+1+i'}^{p-1}
  for (int i = 0; i <= p; ++i) {
    int j = mu - p + i;
    double v = 0.0;
    if (i >= 1) {
      double den = kn[j + p] - kn[j];
      if (den > 0) v += p / den * prev[i - 1];
    }
    if (i <= p - 1) {
      double den = kn[j + p + 1] - kn[j + 1];
      if (den > 0) v -= p / den * prev[i];
    }
    dN[i] = v;
  }
}

// Homogeneous point (and derivatives) of a patch at (s, t), evaluated with the polynomial piece of
// spans (m1, m2).
static void patch_h(const Patch &P, int m1, int m2, double s, double t, double H[4], double Hs[4],
                    double Ht[4]) {
  double b1[8], d1[8], b2[8], d2[8];
  span_basis(P.kn1, P.p1, m1, s, b1, d1);
  span_basis(P.kn2, P.p2, m2, t, b2, d2);
  for (int c = 0; c < 4; ++c) H[c] = Hs[c] = Ht[c] = 0.0;
  for (int i = 0; i <= P.p1; ++i)
    for (int j = 0; j <= P.p2; ++j) {
      const double *h = &P.hw[((m1 - P.p1 + i) * P.k2 + (m2 - P.p2 + j)) * 4];
      for (int c = 0; c < 4; ++c) {
        H[c] += b1[i] * b2[j] * h[c];
        Hs[c] += d1[i] * b2[j] * h[c];
        Ht[c] += b1[i] * d2[j] * h[c];
      }
    }
}

// Point of a patch at (s, t) (no derivatives): the same polynomial-piece sums as patch_h.
static void patch_point(const Patch &P, double s, double t, double F[3]) {
  const int m1 = find_span(P.kn1, P.p1, s), m2 = find_span(P.kn2, P.p2, t);
  double b1[MAX_DEG + 1], b2[MAX_DEG + 1];
  span_basis(P.kn1, P.p1, m1, s, b1, nullptr);
  span_basis(P.kn2, P.p2, m2, t, b2, nullptr);
  double H[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i <= P.p1; ++i)
    for (int j = 0; j <= P.p2; ++j) {
      const double *h = &P.hw[((m1 - P.p1 + i) * P.k2 + (m2 - P.p2 + j)) * 4];
      for (int c = 0; c < 4; ++c) H[c] += b1[i] * b2[j] * h[c];
    }
  for (int c = 0; c < 3; ++c) F[c] = H[c] / H[3];
}

static void patch_eval(const Patch &P, double s, double t, double F[3], double Fs[3] = nullptr,
                       double Ft[3] = nullptr) {
  double H[4], Hs[4], Ht[4];
  patch_h(P, find_span(P.kn1, P.p1, s), find_span(P.kn2, P.p2, t), s, t, H, Hs, Ht);
  for (int c = 0; c < 3; ++c) {
    F[c] = H[c] / H[3];
    if (Fs) Fs[c] = (Hs[c] - F[c] * Hs[3]) / H[3];
    if (Ft) Ft[c] = (Ht[c] - F[c] * Ht[3]) / H[3];
  }
}

static double bernstein(int n, int k, double u) {
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
  return c * std::pow(u, k) * std::pow(1.0 - u, n - k);
}

// Inverse of the Bernstein collocation matrix V[i][k] = B_k^n(i/n) (Gauss-Jordan).
static std::vector<double> bernstein_collocation_inverse(int n) {
  int s = n + 1;
  std::vector<double> A(s * s), I(s * s, 0.0);
  for (int i = 0; i < s; ++i) {
    for (int k = 0; k < s; ++k) A[i * s + k] = n == 0 ? 1.0 : bernstein(n, k, double(i) / n);
    I[i * s + i] = 1.0;
  }
  for (int c = 0; c < s; ++c) {
    int piv = c;
    for (int r = c + 1; r < s; ++r)
      if (std::fabs(A[r * s + c]) > std::fabs(A[piv * s + c])) piv = r;
    for (int k = 0; k < s; ++k) {
      std::swap(A[c * s + k], A[piv * s + k]);
      std::swap(I[c * s + k], I[piv * s + k]);
    }
    double d = A[c * s + c];
    for (int k = 0; k < s; ++k) {
      A[c * s + k] /= d;
      I[c * s + k] /= d;
    }
    for (int r = 0; r < s; ++r)
      if (r != c) {
        double f = A[r * s + c];
        for (int k = 0; k < s; ++k) {
          A[r * s + k] -= f * A[c * s + k];
          I[r * s + k] -= f * I[c * s + k];
        }
      }
  }
  return I;
}

// ----------------------------------------------------------------------------------------------
// Regularising transforms for touching element pairs (same derivation as documented with the
// device quadrature): identical 8 regions, common edge 6, common vertex 4; ns points per variable.

// The regions are ordered with the sign s1 outermost: region (s1 = 1, 1 - s2, tri) is region (0, s2, tri)
// with x and y exchanged, so the first half of the points (s1 = 0) and both orientations of each give
// the whole rule (the singular kernel uses that).
static void rule_identical(const std::vector<double> &gx, const std::vector<double> &gw, Rule4 &R) {
  int n = (int)gx.size();
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < 2; ++s2)
      for (int tri = 0; tri < 2; ++tri)
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c)
              for (int d = 0; d < n; ++d) {
                double xi = gx[a], eta = gx[b], t1 = gx[c], t2 = gx[d];
                double z1 = tri == 0 ? xi : xi * eta, z2 = tri == 0 ? xi * eta : xi;
                double b1 = (1 - z1) * t1, b2 = (1 - z2) * t2;
                double jac = xi * (1 - z1) * (1 - z2);
                double x1 = s1 == 0 ? b1 : b1 + z1, y1 = s1 == 0 ? b1 + z1 : b1;
                double x2 = s2 == 0 ? b2 : b2 + z2, y2 = s2 == 0 ? b2 + z2 : b2;
                R.x1.push_back(x1); R.x2.push_back(x2); R.y1.push_back(y1); R.y2.push_back(y2);
                R.w.push_back(gw[a] * gw[b] * gw[c] * gw[d] * jac);
              }
}

static void rule_edge(const std::vector<double> &gx, const std::vector<double> &gw, Rule4 &R) {
  int n = (int)gx.size();
  for (int sz = 0; sz < 2; ++sz)
    for (int pyr = 0; pyr < 3; ++pyr)
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
          for (int c = 0; c < n; ++c)
            for (int d = 0; d < n; ++d) {
              double xi = gx[a], e1 = gx[b], e2 = gx[c], t = gx[d];
              double x1, y1, z;
              if (pyr == 0) { x1 = xi; y1 = xi * e1; z = xi * e2; }
              else if (pyr == 1) { y1 = xi; x1 = xi * e1; z = xi * e2; }
              else { z = xi; x1 = xi * e1; y1 = xi * e2; }
              double bb = (1 - z) * t, jac = xi * xi * (1 - z);
              double x2 = sz == 0 ? bb : bb + z, y2 = sz == 0 ? bb + z : bb;
              R.x1.push_back(x1); R.x2.push_back(x2); R.y1.push_back(y1); R.y2.push_back(y2);
              R.w.push_back(gw[a] * gw[b] * gw[c] * gw[d] * jac);
            }
}

static void rule_vertex(const std::vector<double> &gx, const std::vector<double> &gw, Rule4 &R) {
  int n = (int)gx.size();
  for (int big = 0; big < 4; ++big)
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c)
          for (int d = 0; d < n; ++d) {
            double xi = gx[a], e[3] = {gx[b], gx[c], gx[d]}, co[4];
            co[big] = xi;
            for (int i = 0, k = 0; i < 4; ++i)
              if (i != big) co[i] = xi * e[k++];
            R.x1.push_back(co[0]); R.x2.push_back(co[1]); R.y1.push_back(co[2]); R.y2.push_back(co[3]);
            R.w.push_back(gw[a] * gw[b] * gw[c] * gw[d] * xi * xi * xi);
          }
}

// Sharing tables of a rule (Rule4::share).  In the tensor rules above each coordinate of a point
// depends on three of the four Gauss indices at most, so inside a chunk of consecutive points (whole
// groups of ns^2 points with the first two indices fixed) a coordinate takes few distinct values and
// many points repeat one element's point: the singular kernel evaluates the geometry once per distinct
// value / point of a chunk.
static void share_tables(Rule4 &R, int ch, int &nv_max, int &nd_max) {
  const int n = (int)R.w.size(), nch = (n + ch - 1) / ch, hdr = sing_share_header(ch);
  R.share.assign((size_t)nch * hdr + (size_t)n * 6, 0);
  unsigned char *PI = R.share.data() + (size_t)nch * hdr;
  for (int c = 0; c < nch; ++c) {
    unsigned char *H = R.share.data() + (size_t)c * hdr;
    const int p0 = c * ch, cn = std::min(ch, n - p0);
    for (int side = 0; side < 2; ++side) {
      const std::vector<double> &a = side ? R.y1 : R.x1, &b = side ? R.y2 : R.x2;
      std::map<double, int> m1, m2;
      std::map<std::pair<double, double>, int> md;
      auto put = [&](auto &m, const auto &key, int list, int t) {
        auto it = m.find(key);
        int id;
        if (it == m.end()) {
          id = (int)m.size();
          m.emplace(key, id);
          H[6 + list * ch + id] = (unsigned char)t;
        } else {
          id = it->second;
        }
        PI[(size_t)(p0 + t) * 6 + list] = (unsigned char)id;
        return id;
      };
      std::vector<int> grp(cn);
      for (int t = 0; t < cn; ++t) {
        const int p = p0 + t;
        put(m1, a[p], 3 * side, t);
        put(m2, b[p], 3 * side + 1, t);
        grp[t] = put(md, std::make_pair(a[p], b[p]), 3 * side + 2, t);
      }
      const int nd = (int)md.size();
      H[3 * side] = (unsigned char)m1.size();
      H[3 * side + 1] = (unsigned char)m2.size();
      H[3 * side + 2] = (unsigned char)nd;
      // the chunk's points grouped by distinct point, ascending within a group
      unsigned char *goff = H + 6 + 6 * ch + side * (ch + 1), *gmem = H + 6 + 6 * ch + 2 * (ch + 1) + side * ch;
      std::vector<int> cnt(nd + 1, 0);
      for (int t = 0; t < cn; ++t) cnt[grp[t] + 1]++;
      for (int g = 0; g < nd; ++g) cnt[g + 1] += cnt[g];
      for (int g = 0; g <= nd; ++g) goff[g] = (unsigned char)cnt[g];
      for (int t = 0; t < cn; ++t) gmem[cnt[grp[t]]++] = (unsigned char)t;
      nv_max = std::max(nv_max, (int)std::max(m1.size(), m2.size()));
      nd_max = std::max(nd_max, nd);
    }
  }
}

// The eight symmetries of the unit square, in the order identity, rotations by 90/180/270
// degrees, then these composed with the diagonal reflection; applied to corner coordinates.
static void d4(int k, int u, int v, int &ou, int &ov) {
  int a = u, b = v;
  if (k >= 4) std::swap(a, b);  // S(u,v) = (v,u), applied first
  for (int r = 0; r < (k & 3); ++r) {  // R(u,v) = (1-v, u)
    int na = 1 - b, nb = a;
    a = na;
    b = nb;
  }
  ou = a;
  ov = b;
}

// ----------------------------------------------------------------------------------------------
// spatial hash of points (coincidence within tol)

struct PointHash {
  double cell;
  std::unordered_map<long long, std::vector<int>> map;
  static long long key(long long a, long long b, long long c) {
    return (a * 73856093LL) ^ (b * 19349663LL) ^ (c * 83492791LL);
  }
  long long ci(double v) const { return (long long)std::floor(v / cell); }
  void insert(const double *x, int id) { map[key(ci(x[0]), ci(x[1]), ci(x[2]))].push_back(id); }
  template <class F> void near(const double *x, F f) const {
    long long a = ci(x[0]), b = ci(x[1]), c = ci(x[2]);
    for (long long i = a - 1; i <= a + 1; ++i)
      for (long long j = b - 1; j <= b + 1; ++j)
        for (long long k = c - 1; k <= c + 1; ++k) {
          auto it = map.find(key(i, j, k));
          if (it != map.end())
            for (int id : it->second) f(id);
        }
  }
};

// CSR lists (row pointers, columns ascending within a row) of distinct pairs (row, column) with rows and
// columns in 0..n-1: two stable counting passes, by column and then by row.
static void csr_of_pairs(const std::vector<std::pair<int, int>> &pairs, int n, std::vector<int> &ptr,
                         std::vector<int> &col) {
  std::vector<int> cnt(n + 1, 0);
  for (const auto &pr : pairs) cnt[pr.second + 1]++;
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> by_col(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) by_col[cnt[pairs[i].second]++] = (int)i;
  ptr.assign(n + 1, 0);
  for (const auto &pr : pairs) ptr[pr.first + 1]++;
  for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  col.resize(pairs.size());
  for (int i : by_col) col[fill[pairs[i].first]++] = pairs[i].second;
}

// body(i) for i in [0, n) on up to 16 host threads (independent iterations writing disjoint data)
template <class F>
static void parallel_for(long n, const F &body) {
  const long nt = std::min<long>(std::min<long>(16, std::max(1u, std::thread::hardware_concurrency())), n);
  if (nt <= 1) {
    for (long i = 0; i < n; ++i) body(i);
    return;
  }
  std::vector<std::thread> th;
  for (long k = 0; k < nt; ++k)
    th.emplace_back([&, k] {
      for (long i = k; i < n; i += nt) body(i);
    });
  for (auto &t : th) t.join();
}

static double dist3(const double *a, const double *b) {
  return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                   (a[2] - b[2]) * (a[2] - b[2]));
}

// ----------------------------------------------------------------------------------------------

void build_setup(const std::vector<Patch> &patches, const igabem_options &opt, HostSetup &S, const GeoCache *hit,
                 GeoCache *fill) {
  const int np = (int)patches.size();
  const int m = opt.level_m, p = opt.degree_p;
  if (m < 0 || m > 12) fail(IGABEM_EINVAL, "level_m must lie in 0..12");
  if (p < 0 || p > 6) fail(IGABEM_EINVAL, "degree_p must lie in 0..6");
  S.hard = opt.bc == IGABEM_SOUND_HARD;
  if (S.hard && p < 1) fail(IGABEM_EINVAL, "sound-hard problems need degree_p >= 1");
  S.np = np; S.m = m; S.p = p; S.n1 = 1 << m; S.h = 1.0 / S.n1;
  S.E = np * S.n1 * S.n1; S.nb = S.n1 + p; S.nloc = (p + 1) * (p + 1);
  S.NX = (long)np * S.nb * S.nb;
  S.ng = opt.gauss_regular; S.ns = opt.gauss_singular;
  if (S.ng < 1 || S.ng > 8 || S.ns < 1 || S.ns > 10) fail(IGABEM_EINVAL, "quadrature orders out of range");

  // --- per-element rational Bezier nets ---
  if (hit) {
    S.edeg = hit->edeg;
    S.eoff = hit->eoff;
    S.ebez = hit->ebez;
    S.corners = hit->corners;
    S.scale = hit->scale;
  } else {
    S.edeg.resize(2 * S.E);
    S.eoff.resize(S.E);
    long off = 0;
    for (int j = 0; j < np; ++j) {
      const Patch &P = patches[j];
      for (const std::vector<double> *kn : {&P.kn1, &P.kn2})
        for (double x : *kn) {
          double y = x * S.n1;
          if (std::fabs(y - std::round(y)) > 1e-9)
            fail(IGABEM_EINVAL, "patch " + std::to_string(j) +
                                    ": a knot is not an element boundary at this level m");
        }
      for (int e = 0; e < S.n1 * S.n1; ++e) {
        int id = j * S.n1 * S.n1 + e;
        S.edeg[2 * id] = P.p1; S.edeg[2 * id + 1] = P.p2;
        S.eoff[id] = off;
        off += 4L * (P.p1 + 1) * (P.p2 + 1);
      }
    }
    S.ebez.assign(off, 0.0);
    S.corners.assign(12L * S.E, 0.0);
    for (int j = 0; j < np; ++j) {
      const Patch &P = patches[j];
      if (P.p1 > MAX_DEG || P.p2 > MAX_DEG) fail(IGABEM_EINVAL, "patch degree above " + std::to_string(MAX_DEG));
      const int s1 = P.p1 + 1, s2 = P.p2 + 1;
      // The element's Bezier net is linear in the control points of its polynomial piece:
      // net = E1[ix] CP E2[iy]^T per homogeneous component, with E = (Bezier collocation inverse) x
      // (B-spline values at the element's collocation points u_a = a / p) per direction.
      auto factors = [&](const std::vector<double> &kn, int pd, std::vector<int> &span, std::vector<double> &E) {
        const int sd = pd + 1;
        const std::vector<double> Vi = bernstein_collocation_inverse(pd);
        span.assign(S.n1, 0);
        E.assign((size_t)S.n1 * sd * sd, 0.0);
        std::vector<double> B((size_t)sd * sd);
        for (int ix = 0; ix < S.n1; ++ix) {
          span[ix] = find_span(kn, pd, (ix + 0.5) * S.h);
          for (int a = 0; a < sd; ++a) {
            const double u = pd ? double(a) / pd : 0.0;
            span_basis(kn, pd, span[ix], (ix + u) * S.h, &B[(size_t)a * sd], nullptr);
          }
          for (int a = 0; a < sd; ++a)
            for (int i = 0; i < sd; ++i) {
              double acc = 0;
              for (int k = 0; k < sd; ++k) acc += Vi[a * sd + k] * B[(size_t)k * sd + i];
              E[((size_t)ix * sd + a) * sd + i] = acc;
            }
        }
      };
      std::vector<int> span1, span2;
      std::vector<double> E1, E2;
      factors(P.kn1, P.p1, span1, E1);
      factors(P.kn2, P.p2, span2, E2);
      parallel_for(S.n1, [&](long ixl) {
        const int ix = (int)ixl;
        std::vector<double> T((size_t)s1 * s2 * 4);
        for (int iy = 0; iy < S.n1; ++iy) {
          const int id = (j * S.n1 + ix) * S.n1 + iy;
          const int i0 = span1[ix] - P.p1, j0 = span2[iy] - P.p2;
          const double *e1 = &E1[(size_t)ix * s1 * s1], *e2 = &E2[(size_t)iy * s2 * s2];
          // T[i][b] = sum_jj E2[b][jj] CP[i0 + i][j0 + jj]
          for (int i = 0; i < s1; ++i)
            for (int b = 0; b < s2; ++b)
              for (int c = 0; c < 4; ++c) {
                double acc = 0;
                for (int jj = 0; jj < s2; ++jj) acc += e2[b * s2 + jj] * P.hw[((i0 + i) * P.k2 + (j0 + jj)) * 4 + c];
                T[(i * s2 + b) * 4 + c] = acc;
              }
          double *out = &S.ebez[S.eoff[id]];
          for (int a = 0; a < s1; ++a)
            for (int b = 0; b < s2; ++b)
              for (int c = 0; c < 4; ++c) {
                double acc = 0;
                for (int i = 0; i < s1; ++i) acc += e1[a * s1 + i] * T[(i * s2 + b) * 4 + c];
                out[(a * s2 + b) * 4 + c] = acc;
              }
          const int ca[4] = {0, P.p1, 0, P.p1}, cb[4] = {0, 0, P.p2, P.p2};
          for (int c = 0; c < 4; ++c) {
            const double *hw = &out[(ca[c] * s2 + cb[c]) * 4];
            for (int k = 0; k < 3; ++k) S.corners[(id * 4 + c) * 3 + k] = hw[k] / hw[3];
          }
        }
      });
    }
    S.scale = 0;
    for (double v : S.corners) S.scale = std::max(S.scale, std::fabs(v));
    if (fill) {
      fill->m = m;
      fill->edeg = S.edeg;
      fill->eoff = S.eoff;
      fill->ebez = S.ebez;
      fill->corners = S.corners;
      fill->scale = S.scale;
    }
  }

  // --- quadrature ---
  gauss_legendre01(S.ng, S.gx, S.gw);
  std::vector<double> sx, sw;
  gauss_legendre01(S.ns, sx, sw);
  rule_identical(sx, sw, S.r_id);
  rule_edge(sx, sw, S.r_edge);
  rule_vertex(sx, sw, S.r_vert);
  // chunk of the singular kernel: whole groups of ns^2 points, at most 128 (one point per thread)
  {
    const int g = S.ns * S.ns <= 128 ? S.ns * S.ns : 128;
    int pg1 = 1;
    for (int v : S.edeg) pg1 = std::max(pg1, v + 1);
    // the largest chunk whose shared memory lets two blocks share an SM (larger chunks share more element
    // geometry and form fewer groups), else the smallest chunk that fits at all
    std::vector<std::pair<int, double>> cands;  // (chunk, bytes)
    for (int ch = (128 / g) * g; ch >= g; ch -= g) {
      int nv = 0, nd = 0;
      for (Rule4 *r : {&S.r_id, &S.r_edge, &S.r_vert}) share_tables(*r, ch, nv, nd);
      cands.push_back({ch, 8.0 * sing_layout(ch, S.nloc, S.hard, nv, nd, pg1).total});
    }
    int chosen = 0;
    for (double lim : {112.0 * 1024, 227.0 * 1024}) {
      for (const auto &c : cands)
        if (c.second <= lim && (lim < 200 * 1024 || c.first == g)) {
          chosen = c.first;
          break;
        }
      if (chosen) break;
    }
    if (chosen) {
      S.sing_ch = chosen;
      S.sing_nv = S.sing_nd = 0;
      for (Rule4 *r : {&S.r_id, &S.r_edge, &S.r_vert}) share_tables(*r, chosen, S.sing_nv, S.sing_nd);
    }
    if (!chosen) fail(IGABEM_EINVAL, "gauss_singular and degree_p too large for the singular kernel");
    // the factorised identical-pair sums need whole ns^2 groups per chunk and room for the univariate
    // basis values (4 ch (p+1) / ns doubles) where the grouped side's basis values go
    S.sing_fact = !S.hard && S.sing_ch % (S.ns * S.ns) == 0 &&
                  4 * (S.sing_ch / S.ns) * (p + 1) <= S.sing_nd * S.nloc && S.sing_ch / S.ns <= S.sing_nd;
  }

  // --- ansatz space: knot vector Xi_{p,m}, tables per element column ---
  std::vector<double> kn;
  for (int i = 0; i <= p; ++i) kn.push_back(0.0);
  for (int i = 1; i < S.n1; ++i) kn.push_back(double(i) / S.n1);
  for (int i = 0; i <= p; ++i) kn.push_back(1.0);
  S.phi1.assign((size_t)S.n1 * S.ng * (p + 1), 0.0);
  S.dphi1.assign(S.phi1.size(), 0.0);
  S.ext1.assign((size_t)S.n1 * (p + 1) * (p + 1), 0.0);
  std::vector<double> Vinv = bernstein_collocation_inverse(p);
  for (int ix = 0; ix < S.n1; ++ix) {
    double N[8], dN[8];
    for (int q = 0; q < S.ng; ++q) {
      span_basis(kn, p, ix + p, (ix + S.gx[q]) * S.h, N, dN);
      for (int a = 0; a <= p; ++a) {
        S.phi1[(ix * S.ng + q) * (p + 1) + a] = N[a];
        S.dphi1[(ix * S.ng + q) * (p + 1) + a] = dN[a];
      }
    }
    std::vector<double> smp((p + 1) * (p + 1));
    for (int i = 0; i <= p; ++i) {
      double u = p ? double(i) / p : 0.0;
      span_basis(kn, p, ix + p, (ix + u) * S.h, N, nullptr);
      for (int a = 0; a <= p; ++a) smp[i * (p + 1) + a] = N[a];
    }
    for (int a = 0; a <= p; ++a)
      for (int c = 0; c <= p; ++c) {
        double acc = 0;
        for (int i = 0; i <= p; ++i) acc += Vinv[c * (p + 1) + i] * smp[i * (p + 1) + a];
        S.ext1[(ix * (p + 1) + a) * (p + 1) + c] = acc;
      }
  }

  // --- touching element pairs ---
  if (hit) {
    S.touch = hit->touch;
  } else {
    const double tol = 1e-10 * S.scale;
    // sh: (e E + f, bitmask of e's corners shared with f) for every ordered pair e != f, sorted.  Element
    // corners coincide by construction at the grid vertices of a patch, so only the distinct vertices are
    // compared (coincidences across patch boundaries and of degenerate parametrisations): cells of a grid
    // much coarser than the tolerance, sorted, searched in every cell within the tolerance; coinciding vertices
    // are merged (union-find) and every pair of corners at one merged vertex marks its two elements.
    std::vector<std::pair<long long, int>> sh;
    std::vector<long> crep(4L * S.E);  // merged vertex of each element corner 4 e + c
    {
      const int nv1 = S.n1 + 1;
      const long NV = (long)np * nv1 * nv1;
      std::vector<double> vx(3 * NV);
      for (int j = 0; j < np; ++j)
        for (int a = 0; a < nv1; ++a)
          for (int b = 0; b < nv1; ++b) {
            const int ix = std::min(a, S.n1 - 1), iy = std::min(b, S.n1 - 1), c = (a - ix) + 2 * (b - iy);
            const long e = ((long)j * S.n1 + ix) * S.n1 + iy, v = ((long)j * nv1 + a) * nv1 + b;
            for (int k = 0; k < 3; ++k) vx[3 * v + k] = S.corners[(e * 4 + c) * 3 + k];
          }
      const double cell = std::max(1e-7 * S.scale, 1e-300);
      struct Key {
        long long a, b, c;
        long id;
        bool operator<(const Key &o) const {
          return a != o.a ? a < o.a : b != o.b ? b < o.b : c != o.c ? c < o.c : id < o.id;
        }
      };
      auto ci = [&](double x) { return (long long)std::floor(x / cell); };
      std::vector<Key> keys(NV);
      for (long v = 0; v < NV; ++v) keys[v] = {ci(vx[3 * v]), ci(vx[3 * v + 1]), ci(vx[3 * v + 2]), v};
      std::sort(keys.begin(), keys.end());
      std::vector<long> parent(NV);
      std::iota(parent.begin(), parent.end(), 0L);
      auto find = [&](long x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
      };
      for (long v = 0; v < NV; ++v) {
        // the cells a point within tol of this vertex can lie in (almost always the vertex's own)
        const double *x = &vx[3 * v];
        for (long long i = ci(x[0] - tol); i <= ci(x[0] + tol); ++i)
          for (long long jj = ci(x[1] - tol); jj <= ci(x[1] + tol); ++jj)
            for (long long k = ci(x[2] - tol); k <= ci(x[2] + tol); ++k) {
              auto it = std::lower_bound(keys.begin(), keys.end(), Key{i, jj, k, -1});
              for (; it != keys.end() && it->a == i && it->b == jj && it->c == k; ++it)
                if (it->id != v && dist3(&vx[3 * v], &vx[3 * it->id]) <= tol) parent[find(it->id)] = find(v);
            }
      }
      std::vector<std::pair<long, int>> inc(4L * S.E);  // (merged vertex, corner index 4 e + c)
      for (int j = 0; j < np; ++j)
        for (int ix = 0; ix < S.n1; ++ix)
          for (int iy = 0; iy < S.n1; ++iy) {
            const int e = (j * S.n1 + ix) * S.n1 + iy;
            for (int c = 0; c < 4; ++c) {
              crep[4L * e + c] = find(((long)j * nv1 + ix + (c & 1)) * nv1 + iy + (c >> 1));
              inc[4L * e + c] = {crep[4L * e + c], 4 * e + c};
            }
          }
      std::sort(inc.begin(), inc.end());
      // per element: its touching neighbours f with the mask of its corners shared with f
      constexpr int NBMAX = 64;
      std::vector<int> nbf((size_t)S.E * NBMAX), nbm((size_t)S.E * NBMAX), nbc(S.E, 0);
      for (size_t g0 = 0; g0 < inc.size();) {
        size_t g1 = g0;
        while (g1 < inc.size() && inc[g1].first == inc[g0].first) ++g1;
        for (size_t x = g0; x < g1; ++x)
          for (size_t y = g0; y < g1; ++y) {
            const int e = inc[x].second / 4, f = inc[y].second / 4;
            if (e == f) continue;
            int *lf = &nbf[(size_t)e * NBMAX], *lm = &nbm[(size_t)e * NBMAX];
            int k = 0;
            while (k < nbc[e] && lf[k] != f) ++k;
            if (k == nbc[e]) {
              if (k == NBMAX) fail(IGABEM_EINVAL, "an element touches more than 64 others");
              lf[k] = f;
              lm[k] = 0;
              ++nbc[e];
            }
            lm[k] |= 1 << (inc[x].second % 4);
          }
        g0 = g1;
      }
      for (int e = 0; e < S.E; ++e) {
        const size_t b0 = sh.size();
        for (int k = 0; k < nbc[e]; ++k)
          sh.push_back({(long long)e * S.E + nbf[(size_t)e * NBMAX + k], nbm[(size_t)e * NBMAX + k]});
        std::sort(sh.begin() + b0, sh.end());
      }
    }
    S.touch.clear();
    for (int e = 0; e < S.E; ++e) {
      S.touch.insert(S.touch.end(), {e, e, 0, 0, 0});
    }
    for (auto &kv : sh) {
      int e = int(kv.first / S.E), f = int(kv.first % S.E);
      int nsh = __builtin_popcount(kv.second);
      if (nsh > 2) fail(IGABEM_EINVAL, "two elements share more than an edge");
      int kind = nsh == 2 ? 2 : 1;
      int te = -1, tf = -1;
      for (int a = 0; a < 8 && te < 0; ++a)
        for (int b = 0; b < 8; ++b) {
          // corners coincide iff they were merged into one vertex above
          int u, v;
          d4(a, 0, 0, u, v); const long re0 = crep[e * 4L + u + 2 * v];
          d4(b, 0, 0, u, v); const long rf0 = crep[f * 4L + u + 2 * v];
          if (re0 != rf0) continue;
          if (kind == 2) {
            d4(a, 0, 1, u, v); const long re1 = crep[e * 4L + u + 2 * v];
            d4(b, 0, 1, u, v); const long rf1 = crep[f * 4L + u + 2 * v];
            if (re1 != rf1) continue;
          }
          te = a; tf = b;
          break;
        }
      if (te < 0) fail(IGABEM_EINVAL, "touching pair without a canonical position");
      S.touch.insert(S.touch.end(), {e, f, kind, te, tf});
    }
    if (fill) fill->touch = S.touch;
  }

  // --- continuous space: glue patch-wise functions with coinciding Greville anchors ---
  S.x2g.resize(S.NX);
  if (!S.hard) {
    std::iota(S.x2g.begin(), S.x2g.end(), 0);
    S.N = S.NX;
  } else {
    std::vector<double> grev(S.nb);
    for (int i = 0; i < S.nb; ++i) {
      double acc = 0;
      for (int k = 1; k <= p; ++k) acc += kn[i + k];
      grev[i] = acc / p;
    }
    std::vector<double> anchor(3 * S.NX);
    for (int j = 0; j < np; ++j)
      for (int i1 = 0; i1 < S.nb; ++i1)
        for (int i2 = 0; i2 < S.nb; ++i2)
          patch_eval(patches[j], grev[i1], grev[i2], &anchor[3 * (((long)j * S.nb + i1) * S.nb + i2)]);
    PointHash ah;
    ah.cell = 1e-6 * S.scale;
    for (long X = 0; X < S.NX; ++X) ah.insert(&anchor[3 * X], (int)X);
    std::vector<int> cls(S.NX);
    for (long X = 0; X < S.NX; ++X) {
      int best = (int)X;
      ah.near(&anchor[3 * X], [&](int k) {
        if (dist3(&anchor[3 * X], &anchor[3L * k]) <= 1e-9 * S.scale) best = std::min(best, k);
      });
      cls[X] = best;
    }
    std::vector<int> mins(cls.begin(), cls.end());
    std::sort(mins.begin(), mins.end());
    mins.erase(std::unique(mins.begin(), mins.end()), mins.end());
    for (long X = 0; X < S.NX; ++X)
      S.x2g[X] = int(std::lower_bound(mins.begin(), mins.end(), cls[X]) - mins.begin());
    S.N = (long)mins.size();
  }
  S.g2x_ptr.assign(S.N + 1, 0);
  for (long X = 0; X < S.NX; ++X) S.g2x_ptr[S.x2g[X] + 1]++;
  for (long i = 0; i < S.N; ++i) S.g2x_ptr[i + 1] += S.g2x_ptr[i];
  S.g2x_idx.assign(S.NX, 0);
  {
    std::vector<int> fill(S.g2x_ptr.begin(), S.g2x_ptr.end() - 1);
    for (long X = 0; X < S.NX; ++X) S.g2x_idx[fill[S.x2g[X]]++] = (int)X;
  }

  // --- cluster tree and block partition (Sec. 4.4) ---
  S.no_fmm = opt.no_fmm != 0;
  S.b = S.no_fmm ? m : opt.leaf_offset;
  if (S.b < 0 || S.b > m) fail(IGABEM_EINVAL, "leaf_offset must lie in 0..level_m");
  S.L = m - S.b;
  S.q = opt.cheb_q;
  if (S.q < 2 || S.q > 16) fail(IGABEM_EINVAL, "cheb_q must lie in 2..16");
  S.nL1 = (1 << S.b) + p;
  S.nL = S.nL1 * S.nL1;
  S.lev.assign(S.L + 1, TreeLevel{});
  const bool balls_hit = hit && hit->L >= S.L;
  for (int l = 0; l <= S.L; ++l) {
    TreeLevel &T = S.lev[l];
    int nl = 1 << l;
    T.n = np * nl * nl;
    if (balls_hit) {
      T.center = hit->center[l];
      T.radius = hit->radius[l];
      continue;
    }
    T.center.assign(3L * T.n, 0.0);
    T.radius.assign(T.n, 0.0);
    parallel_for((long)np * nl, [&](long jc) {
      const int j = (int)(jc / nl), cx = (int)(jc % nl);
        for (int cy = 0; cy < nl; ++cy) {
          int t = (j * nl + cx) * nl + cy;
          double *c = &T.center[3L * t];
          patch_point(patches[j], (cx + 0.5) / nl, (cy + 0.5) / nl, c);
          double r = 0;
          for (int a = 0; a <= 8; ++a)
            for (int b = 0; b <= 8; ++b) {
              double F[3];
              patch_point(patches[j], (cx + a / 8.0) / nl, (cy + b / 8.0) / nl, F);
              r = std::max(r, dist3(F, c));
            }
          T.radius[t] = r;
        }
    });
  }
  if (fill && !hit) {
    fill->L = S.L;
    for (int l = 0; l <= S.L; ++l) {
      fill->center.push_back(S.lev[l].center);
      fill->radius.push_back(S.lev[l].radius);
    }
  }
  // interpolation points and kappa cap per level (level-adaptive when q_max > cheb_q): the bound
  // eps(q, w) = w^q / (2^(q-1) q!) of q-point Chebyshev interpolation of exp(i w t) on [-1,1]; the
  // finest-level pair (cheb_q, kappa_cap) fixes eps_ref = eps(cheb_q, kappa_cap / 2); each level takes
  // the smallest q in [cheb_q, q_max] with eps(q, kappa D_l / 2) <= eps_ref (else q_max) and the cap
  // cap_l solving eps(q_l, cap_l / 2) = eps_ref.
  const double cap = opt.kappa_cap > 0 ? opt.kappa_cap : INFINITY;
  const int qmax = opt.q_max;
  const bool adaptive = qmax > S.q && !S.no_fmm;
  if (qmax != 0 && (qmax < S.q || qmax > 16)) fail(IGABEM_EINVAL, "q_max must be 0 or lie in cheb_q..16");
  if (adaptive && !(opt.kappa_cap > 0)) fail(IGABEM_EINVAL, "level-adaptive q (q_max > cheb_q) needs kappa_cap > 0");
  auto eps_bound = [](int q, double w) {
    double f = 1.0;
    for (int k = 2; k <= q; ++k) f *= k;
    return std::pow(w, q) / (std::pow(2.0, q - 1) * f);
  };
  for (int l = 0; l <= S.L; ++l) {
    TreeLevel &T = S.lev[l];
    T.q = S.q;
    T.cap = cap;
    if (!adaptive) continue;
    double D = 0;
    for (double r : T.radius) D = std::max(D, 2 * r);
    const double eps_ref = eps_bound(S.q, cap / 2);
    int q = qmax;
    for (int qq = S.q; qq <= qmax; ++qq)
      if (eps_bound(qq, opt.kappa * D / 2) <= eps_ref) {
        q = qq;
        break;
      }
    double f = 1.0;
    for (int k = 2; k <= q; ++k) f *= k;
    T.q = q;
    T.cap = q == S.q ? cap : 2.0 * std::pow(eps_ref * std::pow(2.0, q - 1) * f, 1.0 / q);
  }
  auto admissible = [&](int l, int t, int s) {
    if (S.no_fmm) return false;
    const TreeLevel &T = S.lev[l];
    double rt = T.radius[t], rs = T.radius[s];
    double diam = std::max(2 * rt, 2 * rs);
    double dist = dist3(&T.center[3L * t], &T.center[3L * s]) - rt - rs;
    if (dist <= 0 || diam > opt.eta_adm * dist) return false;
    return opt.kappa * diam <= T.cap;
  };
  std::vector<std::pair<int, int>> cand, nxt, near;
  for (int t = 0; t < np; ++t)
    for (int s = 0; s < np; ++s) cand.push_back({t, s});
  S.n_far = 0;
  S.lmin = S.L + 1;
  for (int l = 0; l <= S.L; ++l) {
    std::vector<std::pair<int, int>> far;
    nxt.clear();
    int nl = 1 << l, nc = 2 * nl;
    // the candidates in chunks on host threads (the CSR lists below do not depend on the order)
    const long nch = std::min<long>(64, ((long)cand.size() + 4095) / 4096);
    std::vector<std::vector<std::pair<int, int>>> cf(nch), cn(nch), cx(nch);
    parallel_for(nch, [&](long c) {
      const size_t i0 = cand.size() * c / nch, i1 = cand.size() * (c + 1) / nch;
      for (size_t i = i0; i < i1; ++i) {
        const int t = cand[i].first, s = cand[i].second;
        if (admissible(l, t, s)) {
          cf[c].push_back({t, s});
        } else if (l == S.L) {
          cn[c].push_back({t, s});
        } else {
          int jt = t / (nl * nl), xt = (t / nl) % nl, yt = t % nl;
          int js = s / (nl * nl), xs = (s / nl) % nl, ys = s % nl;
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
              cx[c].push_back({(jt * nc + 2 * xt + (a >> 1)) * nc + 2 * yt + (a & 1),
                               (js * nc + 2 * xs + (b >> 1)) * nc + 2 * ys + (b & 1)});
        }
      }
    });
    for (long c = 0; c < nch; ++c) {
      far.insert(far.end(), cf[c].begin(), cf[c].end());
      near.insert(near.end(), cn[c].begin(), cn[c].end());
      nxt.insert(nxt.end(), cx[c].begin(), cx[c].end());
    }
    TreeLevel &T = S.lev[l];
    csr_of_pairs(far, T.n, T.far_ptr, T.far_src);
    if (!far.empty()) S.lmin = std::min(S.lmin, l);
    S.n_far += (long)far.size();
    cand.swap(nxt);
  }
  int nleaf = S.lev[S.L].n;
  csr_of_pairs(near, nleaf, S.near_ptr, S.near_src);

  // touching pair -> near block
  int npt = (int)S.touch.size() / 5;
  if (hit) {
    S.nbr = hit->nbr;
    S.nbr_w = hit->nbr_w;
  } else {  // neighbour lists of the touching pairs (both directions), for the regular near-field kernel
    std::vector<std::vector<int>> nb(S.E);
    for (int i = 0; i < npt; ++i) {
      const int e = S.touch[5 * i], f = S.touch[5 * i + 1];
      if (e == f) continue;
      nb[e].push_back(f);
      nb[f].push_back(e);
    }
    S.nbr_w = 1;
    for (auto &v : nb) S.nbr_w = std::max<int>(S.nbr_w, (int)v.size());
    S.nbr.assign((size_t)S.E * S.nbr_w, -1);
    for (int e = 0; e < S.E; ++e)
      for (size_t c = 0; c < nb[e].size(); ++c) S.nbr[(size_t)e * S.nbr_w + c] = nb[e][c];
  }
  if (fill && fill->m >= 0) {
    fill->nbr = S.nbr;
    fill->nbr_w = S.nbr_w;
  }
  S.touch_blk.resize(npt);
  const int nlL = 1 << S.L, bsh = S.b;
  auto leaf_of = [&](int e) {
    int j = e / (S.n1 * S.n1), ix = (e / S.n1) % S.n1, iy = e % S.n1;
    return (j * nlL + (ix >> bsh)) * nlL + (iy >> bsh);
  };
  for (int i = 0; i < npt; ++i) {
    int te = leaf_of(S.touch[5 * i]), tf = leaf_of(S.touch[5 * i + 1]);
    auto b0 = S.near_src.begin() + S.near_ptr[te], b1 = S.near_src.begin() + S.near_ptr[te + 1];
    auto it = std::lower_bound(b0, b1, tf);
    if (it == b1 || *it != tf) fail(IGABEM_EINVAL, "touching pair outside the near field");
    S.touch_blk[i] = int(it - S.near_src.begin());
  }
  S.diag_blk.assign(nleaf, -1);
  for (int t = 0; t < nleaf; ++t)
    for (int k = S.near_ptr[t]; k < S.near_ptr[t + 1]; ++k)
      if (S.near_src[k] == t) S.diag_blk[t] = k;
  // unordered work list: identical pairs, and (e, f) with e < f for the others (the block of (f, e)
  // comes from the same quadrature points with the roles of x and y exchanged)
  S.sing.clear();
  // S.touch: the E identical pairs, then the other pairs (e, f) in ascending order of e E + f
  auto touch_index = [&](int e, int f) {
    int lo = S.E, hi = npt;  // the first entry whose key is not below e E + f
    const long long key = (long long)e * S.E + f;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if ((long long)S.touch[5 * mid] * S.E + S.touch[5 * mid + 1] < key) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= npt || S.touch[5 * lo] != e || S.touch[5 * lo + 1] != f) fail(IGABEM_EINVAL, "touching pair without its reverse");
    return lo;
  };
  for (int i = 0; i < npt; ++i) {
    const int *t = &S.touch[5 * i];
    if (t[2] == 0) {
      // identical pair: the rule's second half is the first with x and y exchanged, so its first half
      // gives the block from both orientations of every point (block of (f, e) = the same block)
      S.sing.insert(S.sing.end(), {t[0], t[1], 0, 0, 0, S.touch_blk[i], S.touch_blk[i]});
    } else if (t[0] < t[1]) {
      int back = S.touch_blk[touch_index(t[1], t[0])];
      S.sing.insert(S.sing.end(), {t[0], t[1], t[2], t[3], t[4], S.touch_blk[i], back});
    }
  }

  // --- interpolation tables (per level: its q; the leaf level's q is S.q of the leaf kernels) ---
  for (int l = 0; l <= S.L; ++l) {
    TreeLevel &T = S.lev[l];
    const int q = T.q;
    T.cheb.resize(q);
    for (int a = 0; a < q; ++a) T.cheb[a] = 0.5 + 0.5 * std::cos((2 * a + 1) * M_PI / (2 * q));
    auto lag = [&](int a, double x) {
      double v = 1.0;
      for (int k = 0; k < q; ++k)
        if (k != a) v *= (x - T.cheb[k]) / (T.cheb[a] - T.cheb[k]);
      return v;
    };
    // transfer to the children (same q): L_a(parent) at the child's node a2, child c of 2 per direction
    T.T1.assign(2L * q * q, 0.0);
    for (int c = 0; c < 2; ++c)
      for (int a = 0; a < q; ++a)
        for (int a2 = 0; a2 < q; ++a2) T.T1[(c * q + a) * q + a2] = lag(a, 0.5 * c + 0.5 * T.cheb[a2]);
    T.band_bottom = l < S.L && S.lev[l + 1].q != q;
    if (T.band_bottom || l == S.L) {  // Lagrange values at the Gauss points of the 2^(m-l) element columns
      const int ne = 1 << (m - l);
      T.LG.assign((size_t)ne * S.ng * q, 0.0);
      for (int o = 0; o < ne; ++o)
        for (int g = 0; g < S.ng; ++g)
          for (int a = 0; a < q; ++a) T.LG[((size_t)o * S.ng + g) * q + a] = lag(a, (o + S.gx[g]) / ne);
    }
  }
  S.q = S.lev[S.L].q;
  S.cheb = S.lev[S.L].cheb;
  S.T1 = S.lev[S.L].T1;
  S.LG1 = S.lev[S.L].LG;
}

}  // namespace igabem
