"""Pins of the oracle's quadrature rules (CPU): polynomial exactness, closed-form singular integrals
over flat squares, and independence of the canonical orientation."""
import itertools

import numpy as np
import pytest

from oracle import assemble as A
from oracle import quadrature as Q
from oracle import space as S
from paper_2306_11324_gb300 import inputs


def test_gauss_rule_exactness():
    for n in (1, 3, 4, 5, 8):
        x, w = Q.gauss01(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
        if n <= 4:
            assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("rule", [Q.rule_identical, Q.rule_edge, Q.rule_vertex])
def test_singular_rules_integrate_polynomials(rule):
    """The transforms are polynomial maps with polynomial Jacobians, so polynomials in (x, y) of
    total degree <= 4 become polynomials of degree <= 9 per transformed variable, which the 5-point
    Gauss rule integrates exactly over [0,1]^4."""
    x1, x2, y1, y2, w = rule(5)
    assert abs(w.sum() - 1) < 1e-14
    for a, b, c, d in itertools.product(range(3), repeat=4):
        if a + b + c + d > 4:
            continue
        exact = 1.0 / ((a + 1) * (b + 1) * (c + 1) * (d + 1))
        assert abs(np.sum(w * x1 ** a * x2 ** b * y1 ** c * y2 ** d) - exact) < 1e-13


def _rect_potential(px, py, x0, x1, y0, y1):
    """int_{x0}^{x1} int_{y0}^{y1} dx dy / |(x, y) - (px, py)| in closed form."""
    def F(x, y):
        r = np.sqrt(x * x + y * y)
        return x * np.log(y + r) + y * np.log(x + r)
    a0, a1, b0, b1 = x0 - px, x1 - px, y0 - py, y1 - py
    return F(a1, b1) - F(a0, b1) - F(a1, b0) + F(a0, b0)


def _semi_analytic(x0, x1, y0, y1, n=200):
    """int over [0,1]^2 of the closed-form inner integral over [x0,x1] x [y0,y1]."""
    x, w = Q.gauss01(n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.sum(np.outer(w, w) * _rect_potential(X, Y, x0, x1, y0, y1))


def test_identical_rule_on_the_unit_square():
    """int_{[0,1]^2} int_{[0,1]^2} 1/|x-y| = 4 ln(1+sqrt2) - 4/3 (sqrt2 - 1)."""
    exact = 4 * np.log(1 + np.sqrt(2)) - 4.0 / 3.0 * (np.sqrt(2) - 1)
    x1, x2, y1, y2, w = Q.rule_identical(5)
    assert abs(np.sum(w / np.hypot(x1 - y1, x2 - y2)) / exact - 1) < 3e-8
    x1, x2, y1, y2, w = Q.rule_identical(10)
    assert abs(np.sum(w / np.hypot(x1 - y1, x2 - y2)) / exact - 1) < 1e-12


def test_edge_and_vertex_rules_on_adjacent_squares():
    ref_edge = _semi_analytic(-1, 0, 0, 1)          # squares [0,1]^2 and [-1,0] x [0,1]
    x1, x2, y1, y2, w = Q.rule_edge(5)
    assert abs(np.sum(w / np.hypot(x1 + y1, x2 - y2)) / ref_edge - 1) < 3e-8
    ref_vert = _semi_analytic(-1, 0, -1, 0)         # squares [0,1]^2 and [-1,0]^2
    x1, x2, y1, y2, w = Q.rule_vertex(5)
    assert abs(np.sum(w / np.hypot(x1 + y1, x2 + y2)) / ref_vert - 1) < 3e-8


def _two_squares(kind, orient):
    """Two unit squares in the plane z=0 meeting in an edge (kind 2) or a vertex (kind 1); the
    second patch's parametrisation is turned by the square symmetry `orient`."""
    sq1 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)]
    if kind == 2:
        c = {(0, 0): (-1, 0, 0), (1, 0): (0, 0, 0), (0, 1): (-1, 1, 0), (1, 1): (0, 1, 0)}
    else:
        c = {(0, 0): (-1, -1, 0), (1, 0): (0, -1, 0), (0, 1): (-1, 0, 0), (1, 1): (0, 0, 0)}
    T = Q.D4[orient]
    corners = []
    for u, v in ((0, 0), (1, 0), (0, 1), (1, 1)):
        a, b = T(u, v)
        corners.append(c[(int(round(a)), int(round(b)))])
    if np.cross(np.subtract(corners[1], corners[0]), np.subtract(corners[2], corners[0]))[2] < 0:
        return None                                   # keep the normals of both patches equal
    return [inputs.flat_patch(sq1), inputs.flat_patch(corners)]


@pytest.mark.parametrize("kind", [2, 1])
def test_touching_pairs_do_not_depend_on_parametrisation(kind):
    """Single-element patches with the constant function (p = 0): the Laplace single layer entry
    between two touching unit squares equals the closed-form value for every orientation of the
    second square's parametrisation."""
    ref = (_semi_analytic(-1, 0, 0, 1) if kind == 2 else _semi_analytic(-1, 0, -1, 0)) / (4 * np.pi)
    seen = 0
    for orient in range(8):
        patches = _two_squares(kind, orient)
        if patches is None:
            continue
        sp = S.Space(S.Mesh(patches, 0), 0)
        V = A.dense_operator(sp, 0.0, "V")
        assert abs(V[0, 1] / ref - 1) < 3e-8 and abs(V[1, 0] / ref - 1) < 3e-8
        seen += 1
    assert seen == 4
