"""Pins of the oracle's geometry, B-spline and space code (CPU)."""
import os

import numpy as np
import pytest

from oracle import bspline
from oracle import space as S
from oracle import quadrature as Q
from paper_2306_11324_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_sphere_patches_lie_on_unit_sphere():
    rng = np.random.default_rng(0)
    for p in inputs.unit_sphere_patches():
        s, t = rng.uniform(0, 1, 500), rng.uniform(0, 1, 500)
        F, Fs, Ft = bspline.nurbs_eval(p, s, t)
        assert np.abs(np.linalg.norm(F, axis=1) - 1).max() < 1e-13
        # tangents are tangent: F . dF = 0 on the unit sphere
        assert np.abs(np.sum(F * Fs, axis=1)).max() < 1e-12
        assert (p.weights > 0).all()


def _edge_samples(patch, n=7):
    g = np.linspace(0, 1, n)
    z, o = np.zeros(n), np.ones(n)
    return [bspline.nurbs_eval(patch, a, b)[0] for a, b in ((z, g), (o, g), (g, z), (g, o))]


@pytest.mark.parametrize("deformed", [False, True])
def test_patches_conform_on_interfaces(deformed):
    patches = inputs.deformed_sphere_patches(spans=4) if deformed else inputs.unit_sphere_patches()
    edges = [e for p in patches for e in _edge_samples(p)]
    matched = 0
    for i, a in enumerate(edges):
        partners = [b for j, b in enumerate(edges) if j // 4 != i // 4 and
                    (np.allclose(a, b, atol=1e-13) or np.allclose(a, b[::-1], atol=1e-13))]
        assert len(partners) == 1, "every patch edge is shared, with equal parametrisation"
        matched += 1
    assert matched == 24


@pytest.mark.parametrize("deformed", [False, True])
def test_normals_point_outward(deformed):
    """int_Gamma x . n dsigma = 3 vol(Omega) > 0 (divergence theorem); 4 pi for the unit sphere."""
    patches = inputs.deformed_sphere_patches(spans=4) if deformed else inputs.unit_sphere_patches()
    u, v, w = Q.tensor_rule(12)
    total = 0.0
    for p in patches:
        F, Fs, Ft = bspline.nurbs_eval(p, u, v)
        total += np.sum(w * np.sum(F * np.cross(Fs, Ft), axis=1))
    if deformed:
        assert total > 0.5 * 4 * np.pi
    else:
        assert abs(total - 4 * np.pi) < 1e-10


def test_deformed_sphere_is_seeded_and_bounded():
    a = inputs.deformed_sphere_patches(spans=4)
    b = inputs.deformed_sphere_patches(spans=4)
    assert all(np.array_equal(x.ctrl, y.ctrl) for x, y in zip(a, b))
    rng = np.random.default_rng(1)
    r = np.concatenate([np.linalg.norm(bspline.nurbs_eval(p, rng.uniform(0, 1, 200),
                                                          rng.uniform(0, 1, 200))[0], axis=1)
                        for p in a])
    assert 0.8 < r.min() and r.max() < 1.2 and r.std() > 0.01


def test_knot_insertion_keeps_the_surface():
    p = inputs.unit_sphere_patches()[2]
    q = inputs.refine_patch(p, 4)
    rng = np.random.default_rng(2)
    s, t = rng.uniform(0, 1, 300), rng.uniform(0, 1, 300)
    for a, b in zip(bspline.nurbs_eval(p, s, t), bspline.nurbs_eval(q, s, t)):
        assert np.abs(a - b).max() < 1e-13


def test_bspline_partition_of_unity_and_bernstein_case():
    x = np.linspace(0, 1, 101)
    for p, m in ((1, 2), (2, 3), (3, 1), (4, 0)):
        B = bspline.basis(S.knot_vector(p, m), p, x)
        assert np.abs(B.sum(axis=1) - 1).max() < 1e-14
        assert B.min() >= -1e-15
    # a single span is the Bernstein basis
    B = bspline.basis(S.knot_vector(3, 0), 3, x)
    bern = np.stack([1 * (1 - x) ** 3, 3 * x * (1 - x) ** 2, 3 * x ** 2 * (1 - x), x ** 3], axis=1)
    assert np.abs(B - bern).max() < 1e-14
    # p = 1 on Xi_{1,2}: hat functions with peaks at the knots
    B = bspline.basis(S.knot_vector(1, 2), 1, x)
    hats = np.maximum(0, 1 - np.abs(4 * x[:, None] - np.arange(5)[None, :]))
    assert np.abs(B - hats).max() < 1e-14


def test_bspline_derivative_matches_finite_differences():
    kn = S.knot_vector(3, 2)
    x = np.array([0.1, 0.3, 0.55, 0.8, 0.93])
    B, dB = bspline.basis_and_derivative(kn, 3, x)
    e = 1e-6
    fd = (bspline.basis(kn, 3, x + e) - bspline.basis(kn, 3, x - e)) / (2 * e)
    assert np.abs(dB - fd).max() < 1e-6
    b, db = bspline.local_basis_and_derivative(kn, 3, x)
    mu = bspline.span_index(kn, 3, x)
    idx = (mu - 3)[:, None] + np.arange(4)[None, :]
    rows = np.arange(len(x))[:, None]
    assert np.abs(B[rows, idx] - b).max() < 1e-15 and np.abs(dB[rows, idx] - db).max() < 1e-13


@pytest.mark.parametrize("m,p", [(1, 1), (2, 2), (2, 3), (1, 4)])
def test_dimension_of_spaces_on_the_sphere(m, p):
    mesh = S.Mesh(inputs.unit_sphere_patches(), m)
    assert S.Space(mesh, p).N == 6 * (2 ** m + p) ** 2
    # closed surface of quadrilateral patches: n (2^m+p-1)^2 + Euler characteristic (2)
    assert S.Space(mesh, p, continuous=True).N == 6 * (2 ** m + p - 1) ** 2 + 2


@pytest.mark.parametrize("m,p", [(0, 1), (1, 2), (1, 3)])
def test_dimension_of_spaces_on_a_torus(m, p):
    mesh = S.Mesh(inputs.polyhedral_torus_patches(), m)
    assert S.Space(mesh, p).N == 16 * (2 ** m + p) ** 2
    assert S.Space(mesh, p, continuous=True).N == 16 * (2 ** m + p - 1) ** 2   # Euler char. 0


def test_dimension_formulas_reproduce_the_turbine_example():
    """The counts checked above (S^2: n (2^m+p)^2; S^0: n (2^m+p-1)^2 + Euler characteristic, shown
    for the sphere and the torus) give the paper's turbine numbers; 12'000 = 120 * 10^2 means the
    turbine's closed patch layout has Euler characteristic 0."""
    row = np.loadtxt(os.path.join(GOLDEN, "turbine_dofs.txt"))
    n, p, m, d2, d0 = (int(v) for v in row)
    assert n * (2 ** m + p) ** 2 == d2
    assert n * (2 ** m + p - 1) ** 2 + 0 == d0


def test_continuous_space_traces_agree_across_interfaces():
    """A random S^0 function has equal values from both sides of every interface."""
    mesh = S.Mesh(inputs.deformed_sphere_patches(spans=2), 1)
    sp = S.Space(mesh, 2, continuous=True)
    c = np.random.default_rng(3).standard_normal(sp.N)
    cX = c[sp.x2g]
    g = np.linspace(0.05, 0.95, 5)
    pts, vals = [], []
    for e in range(mesh.E):
        for uu, vv in ((np.zeros(5), g), (np.ones(5), g), (g, np.zeros(5)), (g, np.ones(5))):
            phi, _, _ = sp.eval(np.full(5, e), uu, vv)
            x, _, _ = mesh.geometry(np.full(5, e), uu, vv)
            pts.append(x); vals.append(phi @ cX[sp.l2x[e]])
    pts, vals = np.concatenate(pts), np.concatenate(vals)
    from scipy.spatial import cKDTree
    for a, b in cKDTree(pts).query_pairs(1e-11):
        assert abs(vals[a] - vals[b]) < 1e-12


def test_exact_torus_lies_on_the_torus_conforms_and_points_outward():
    """The 16 rational biquadratic patches of the convergence workload (Sec. 5.2: torus R = 2, r = 0.5):
    every point satisfies (rho - R)^2 + z^2 = r^2, shared edges carry equal parametrisations, the
    normals point out (int x . n = 3 vol = 6 pi^2 R r^2) and S^0 has dimension 16 (2^m+p-1)^2 (Euler
    characteristic 0)."""
    patches = inputs.torus_patches(2.0, 0.5)
    rng = np.random.default_rng(3)
    for p in patches:
        s, t = rng.uniform(0, 1, 300), rng.uniform(0, 1, 300)
        F, _, _ = bspline.nurbs_eval(p, s, t)
        rho = np.hypot(F[:, 0], F[:, 1])
        assert np.abs((rho - 2.0) ** 2 + F[:, 2] ** 2 - 0.25).max() < 1e-13
    edges = [e for p in patches for e in _edge_samples(p)]
    for i, a in enumerate(edges):
        partners = [b for j, b in enumerate(edges) if j // 4 != i // 4 and
                    (np.allclose(a, b, atol=1e-13) or np.allclose(a, b[::-1], atol=1e-13))]
        assert len(partners) == 1
    u, v, w = Q.tensor_rule(14)
    total = 0.0
    for p in patches:
        F, Fs, Ft = bspline.nurbs_eval(p, u, v)
        total += np.sum(w * np.sum(F * np.cross(Fs, Ft), axis=1))
    assert abs(total - 6 * np.pi ** 2 * 2.0 * 0.25) < 1e-9
    for m, p in ((1, 1), (2, 2)):
        mesh = S.Mesh(patches, m)
        assert S.Space(mesh, p, continuous=True).N == 16 * (2 ** m + p - 1) ** 2
