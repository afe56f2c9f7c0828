"""Quadrature rules for Galerkin element pairs (oracle; test infrastructure).

The paper computes the Galerkin entries of Sec. 4.2-4.3 as integrals over pairs of parameter squares
but does not say how.  The rules used here (and, independently written, by the CUDA path) are:

  * regular pairs (no common point): the tensor Gauss-Legendre rule with 4 points per direction on
    each element, i.e. 16 x 16 point pairs;
  * touching pairs (identical element, common edge, common vertex): regularising transforms of the
    Sauter-Schwab type for quadrilaterals, derived below, with 5 Gauss points in each of the four
    transformed variables (identical: 8 regions, edge: 6, vertex: 4).

Each transform maps the unit 4-cube onto a piece of [0,1]^2 x [0,1]^2 = {(x, y)} with a Jacobian
that vanishes like the distance to the singular set raised to the power needed to cancel a 1/r
kernel.  Canonical positions: for a common edge both elements have the edge at x1 = 0 (resp.
y1 = 0) with x2 = y2 along it; for a common vertex both have it at the local origin.

Derivation (identical elements).  In each direction d put z_d = y_d - x_d and split by its sign; with
zeta_d = |z_d| and a base coordinate b_d in [0, 1 - zeta_d] the pair is (b_d, b_d + zeta_d) for a
positive sign and (b_d + zeta_d, b_d) for a negative one.  The singular set zeta = 0 is the corner of
the zeta square; splitting that square along its diagonal and writing (zeta1, zeta2) = (xi, xi eta)
or (xi eta, xi) gives the Jacobian xi; b_d = (1 - zeta_d) t_d adds (1 - zeta1)(1 - zeta2).

Common edge.  Along the edge the same sign split gives zeta = |y2 - x2| and b = (1 - zeta) t.  The
remaining singular point is the origin of (x1, y1, zeta); the cube is split into three pyramids by
its largest coordinate xi, the other two being xi eta1, xi eta2 in the order (x1, y1, zeta): Jacobian
xi^2 (1 - zeta).

Common vertex.  The singular point is the origin of (x1, x2, y1, y2); four pyramids by the largest
coordinate xi, the other three xi eta1, xi eta2, xi eta3 in the order (x1, x2, y1, y2): Jacobian xi^3.
"""
from __future__ import annotations

import itertools

import numpy as np


def gauss01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def tensor_rule(n: int):
    """Tensor Gauss rule on the unit square: (u, v, w) with point index q = a*n + b (u index major)."""
    x, w = gauss01(n)
    u = np.repeat(x, n)
    v = np.tile(x, n)
    return u, v, np.repeat(w, n) * np.tile(w, n)


def _cube(n: int):
    x, w = gauss01(n)
    g = np.array(list(itertools.product(range(n), repeat=4)))
    return [x[g[:, i]] for i in range(4)], np.prod(w[g], axis=1)


def rule_identical(n: int = 5):
    """(x1, x2, y1, y2, weight) for the integral over [0,1]^2 x [0,1]^2 with singularity at x = y."""
    (xi, eta, t1, t2), w0 = _cube(n)
    out = []
    for s1, s2, tri in itertools.product((1, -1), (1, -1), (0, 1)):
        z1, z2 = (xi, xi * eta) if tri == 0 else (xi * eta, xi)
        b1, b2 = (1.0 - z1) * t1, (1.0 - z2) * t2
        jac = xi * (1.0 - z1) * (1.0 - z2)
        x1, y1 = (b1, b1 + z1) if s1 > 0 else (b1 + z1, b1)
        x2, y2 = (b2, b2 + z2) if s2 > 0 else (b2 + z2, b2)
        out.append((x1, x2, y1, y2, w0 * jac))
    return tuple(np.concatenate(c) for c in zip(*out))


def rule_edge(n: int = 5):
    """Rule for a common edge in canonical position (x1 = y1 = 0 on the edge, x2 = y2 along it)."""
    (xi, e1, e2, t), w0 = _cube(n)
    out = []
    for sz, pyr in itertools.product((1, -1), (0, 1, 2)):
        if pyr == 0:
            x1, y1, z = xi, xi * e1, xi * e2
        elif pyr == 1:
            y1, x1, z = xi, xi * e1, xi * e2
        else:
            z, x1, y1 = xi, xi * e1, xi * e2
        b = (1.0 - z) * t
        jac = xi * xi * (1.0 - z)
        x2, y2 = (b, b + z) if sz > 0 else (b + z, b)
        out.append((x1, x2, y1, y2, w0 * jac))
    return tuple(np.concatenate(c) for c in zip(*out))


def rule_vertex(n: int = 5):
    """Rule for a common vertex in canonical position (both elements at their local origin)."""
    (xi, e1, e2, e3), w0 = _cube(n)
    out = []
    for big in range(4):
        coords = [None] * 4
        coords[big] = xi
        rest = [i for i in range(4) if i != big]
        for i, e in zip(rest, (e1, e2, e3)):
            coords[i] = xi * e
        out.append((coords[0], coords[1], coords[2], coords[3], w0 * xi ** 3))
    return tuple(np.concatenate(c) for c in zip(*out))


# The eight symmetries of the unit square in the fixed order used to bring a touching pair into
# canonical position: identity, rotations by 90, 180, 270 degrees, then the same four composed with
# the diagonal reflection (u, v) -> (v, u).
D4 = (
    lambda u, v: (u, v),
    lambda u, v: (1.0 - v, u),
    lambda u, v: (1.0 - u, 1.0 - v),
    lambda u, v: (v, 1.0 - u),
    lambda u, v: (v, u),
    lambda u, v: (1.0 - u, v),
    lambda u, v: (1.0 - v, 1.0 - u),
    lambda u, v: (u, 1.0 - v),
)
