"""B-spline bases and NURBS patch maps (oracle; test infrastructure).

Follows Sec. 3.1 (p-open knot vectors, the Cox-de Boor recursion for b_j^p) and Sec. 3.2 (the NURBS
patch map F_j as a weighted quotient of tensor-product B-splines).  Everything is evaluated
directly from the knot vector at every point: no Bezier extraction, no tables.
"""
from __future__ import annotations

import numpy as np


def _degree0(knots: np.ndarray, x: np.ndarray) -> np.ndarray:
    """b_j^0(x) = 1 on [xi_j, xi_{j+1}), else 0.  The right end x == xi_last is assigned to the last
    non-empty span so that the basis is a partition of unity on the closed interval."""
    n = len(knots) - 1
    B = np.zeros((x.shape[0], n))
    for j in range(n):
        B[:, j] = (knots[j] <= x) & (x < knots[j + 1])
    last = max(j for j in range(n) if knots[j] < knots[j + 1])
    B[x >= knots[-1], last] = 1.0
    return B


def _raise(knots: np.ndarray, x: np.ndarray, B: np.ndarray, d: int) -> np.ndarray:
    """One step of the recursion: degree d-1 values B -> degree d values."""
    n = B.shape[1] - 1
    out = np.zeros((x.shape[0], n))
    for j in range(n):
        den1 = knots[j + d] - knots[j]
        den2 = knots[j + d + 1] - knots[j + 1]
        if den1 > 0:
            out[:, j] += (x - knots[j]) / den1 * B[:, j]
        if den2 > 0:
            out[:, j] += (knots[j + d + 1] - x) / den2 * B[:, j + 1]
    return out


def basis(knots, p: int, x) -> np.ndarray:
    """All k = len(knots)-p-1 B-splines b_j^p at the points x: array (len(x), k)."""
    knots = np.asarray(knots, float)
    x = np.atleast_1d(np.asarray(x, float))
    B = _degree0(knots, x)
    for d in range(1, p + 1):
        B = _raise(knots, x, B, d)
    return B


def basis_and_derivative(knots, p: int, x):
    """(b_j^p(x), d/dx b_j^p(x)) for all j, using
    d/dx b_j^p = p/(xi_{j+p}-xi_j) b_j^{p-1} - p/(xi_{j+p+1}-xi_{j+1}) b_{j+1}^{p-1}."""
    knots = np.asarray(knots, float)
    x = np.atleast_1d(np.asarray(x, float))
    k = len(knots) - p - 1
    B = _degree0(knots, x)
    for d in range(1, p):
        B = _raise(knots, x, B, d)
    if p == 0:
        return B, np.zeros_like(B)
    Bp = _raise(knots, x, B, p)
    dB = np.zeros((x.shape[0], k))
    for j in range(k):
        den1 = knots[j + p] - knots[j]
        den2 = knots[j + p + 1] - knots[j + 1]
        if den1 > 0:
            dB[:, j] += p / den1 * B[:, j]
        if den2 > 0:
            dB[:, j] -= p / den2 * B[:, j + 1]
    return Bp, dB


def span_index(knots, p: int, x) -> np.ndarray:
    """Index mu with xi_mu <= x < xi_{mu+1} (the last non-empty span for x at the right end)."""
    knots = np.asarray(knots, float)
    k = len(knots) - p - 1
    mu = np.searchsorted(knots, np.asarray(x, float), side="right") - 1
    return np.clip(mu, p, k - 1)


def local_basis_and_derivative(knots, p: int, x, mu=None):
    """The p+1 B-splines b_{mu-p}^p .. b_mu^p that are non-zero on the span mu of each point, and
    their derivatives: two arrays (n, p+1).  The same Cox-de Boor recursion as ``basis``, restricted
    to the functions that do not vanish on the span (the others are zero there)."""
    knots = np.asarray(knots, float)
    x = np.atleast_1d(np.asarray(x, float))
    mu = span_index(knots, p, x) if mu is None else np.asarray(mu)

    window = {off: knots[mu + off] for off in range(-p, p + 2)}

    def kn(off):
        return window[off]

    def safe_div(a, b):
        return np.where(b > 0, a / np.where(b > 0, b, 1.0), 0.0)

    prev = np.ones((x.shape[0], 1))                 # b_mu^0
    lower = prev
    for d in range(1, p + 1):
        new = np.zeros((x.shape[0], d + 1))
        for i in range(d + 1):                      # j = mu - d + i
            j = i - d
            if i >= 1:
                new[:, i] += safe_div(x - kn(j), kn(j + d) - kn(j)) * prev[:, i - 1]
            if i <= d - 1:
                new[:, i] += safe_div(kn(j + d + 1) - x, kn(j + d + 1) - kn(j + 1)) * prev[:, i]
        lower, prev = prev, new
    if p == 0:
        return prev, np.zeros_like(prev)
    dB = np.zeros_like(prev)
    for i in range(p + 1):                          # j = mu - p + i, lower holds degree p-1
        j = i - p
        if i >= 1:
            dB[:, i] += safe_div(p, kn(j + p) - kn(j)) * lower[:, i - 1]
        if i <= p - 1:
            dB[:, i] -= safe_div(p, kn(j + p + 1) - kn(j + 1)) * lower[:, i]
    return prev, dB


def nurbs_eval(patch, s, t):
    """F(s,t), d_s F, d_t F of a NURBS patch (Sec. 3.2) at points (s_i, t_i): three arrays (n, 3).

    F = N / W with N = sum c_{j1 j2} w_{j1 j2} b_{j1}(s) b_{j2}(t) and W = sum w b b;
    d F = (dN - F dW) / W.
    """
    s = np.atleast_1d(np.asarray(s, float))
    t = np.atleast_1d(np.asarray(t, float))
    p1, p2 = patch.p1, patch.p2
    m1 = span_index(patch.knots1, p1, s)
    m2 = span_index(patch.knots2, p2, t)
    bs, dbs = local_basis_and_derivative(patch.knots1, p1, s, m1)
    bt, dbt = local_basis_and_derivative(patch.knots2, p2, t, m2)
    w = patch.weights
    H = np.concatenate([patch.ctrl * w[..., None], w[..., None]], axis=-1)
    h = np.zeros((s.shape[0], 4)); hs = np.zeros_like(h); ht = np.zeros_like(h)
    for a, b in set(zip(m1.tolist(), m2.tolist())):          # points grouped by knot span
        sel = np.nonzero((m1 == a) & (m2 == b))[0]
        Hl = H[a - p1:a + 1, b - p2:b + 1].reshape(p1 + 1, -1)  # local homogeneous net

        def contract(b1, b2):      # sum_{i j} b1[n, i] b2[n, j] Hl[i, j, :]
            return np.einsum("nj,njc->nc", b2, (b1 @ Hl).reshape(-1, p2 + 1, 4))

        h[sel] = contract(bs[sel], bt[sel])
        hs[sel] = contract(dbs[sel], bt[sel])
        ht[sel] = contract(bs[sel], dbt[sel])
    N, W = h[:, :3], h[:, 3:]
    F = N / W
    return F, (hs[:, :3] - F * hs[:, 3:]) / W, (ht[:, :3] - F * ht[:, 3:]) / W
