"""Pins of the oracle's boundary integral operators (CPU): symmetries, Laplace-limit identities,
Calderon identities and the far field of an interior point source, all exact for the continuous
operators and reproduced up to discretisation error that falls with h."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import farfield
from tests import oracle_cache as C
from paper_2306_11324_gb300 import inputs

Z0 = np.array([0.1, -0.2, 0.15])          # point source inside the unit sphere
KAPPA = 2.0


def _load(sp, rules, vals):
    """X-space vector <f, psi_i> for f given at the Gauss points."""
    pts = rules.pts
    wq = np.tile(rules.w, sp.mesh.E)
    b = np.zeros(sp.NX, dtype=complex)
    np.add.at(b, sp.l2x[pts.e], (wq * pts.a * vals)[:, None] * pts.phi)
    return b


def _point_source(m, deformed=False):
    sp = C.sphere_space(m, 1, False, deformed)
    sp0 = C.sphere_space(m, 1, True, deformed)
    rules = A.ElementRules(sp)
    d = rules.pts.x - Z0
    r = np.linalg.norm(d, axis=1)
    G = np.exp(1j * KAPPA * r) / (4 * np.pi * r)
    dGdn = G * (1j * KAPPA * r - 1) / r ** 2 * np.sum(d * rules.pts.n, axis=1) / rules.pts.a
    ops = C.operators(m, 1, KAPPA, ("M", "V", "K", "Kp", "W"), False, deformed)
    M = ops["M"]
    t = np.linalg.solve(M, _load(sp, rules, dGdn))             # L2 projection of du/dn on S^2
    gX = np.linalg.solve(M, _load(sp, rules, G))               # ... of u on S^2
    P = sp0.prolongation()
    g0 = np.linalg.solve(P.T @ M @ P, P.T @ _load(sp, rules, G))   # ... of u on S^0
    return sp, sp0, ops, t, gX, g0, P


@pytest.fixture(scope="module")
def ps():
    return {m: _point_source(m) for m in (1, 2)}


def test_single_layer_symmetric_and_double_layer_adjoint(ps):
    sp, sp0, ops, *_ = ps[1]
    P = sp0.prolongation()
    V, K, Kp = ops["V"], ops["K"], ops["Kp"]
    W0 = P.T @ ops["W"] @ P
    assert np.abs(V - V.T).max() < 1e-13 * np.abs(V).max()          # complex symmetric
    assert np.abs(K - Kp.T).max() < 1e-13 * np.abs(K).max()         # K on S^2 = (K')^T
    assert np.abs(W0 - W0.T).max() < 1e-13 * np.abs(W0).max()
    assert np.abs(V - V.conj().T).max() > 1e-3 * np.abs(V).max()    # not Hermitian for kappa > 0


def test_laplace_limit_identities():
    """kappa = 0: int dG/dn_y = -1/2 on a smooth surface, so K 1 = -1/2 M 1 (Galerkin, exact up
    to quadrature); the curl of a constant vanishes, so W 1 = 0 exactly."""
    for m in (1, 2):
        sp0 = C.sphere_space(m, 1, True)
        ops = C.operators(m, 1, 0.0, ("M", "K", "W"))
        one = np.ones(ops["M"].shape[0])
        res = np.linalg.norm(ops["K"] @ one + 0.5 * ops["M"] @ one) / np.linalg.norm(ops["M"] @ one)
        assert res < 1e-6
        P = sp0.prolongation()
        assert np.abs(P.T @ ops["W"] @ P @ np.ones(sp0.N)).max() < 1e-13


def test_calderon_identities_of_an_interior_point_source(ps):
    """u = G(., z0), z0 inside: V t = (K - 1/2) g and (1/2 + K') t = -W g on the boundary."""
    res1, res2 = [], []
    for m in (1, 2):
        sp, sp0, ops, t, gX, g0, P = ps[m]
        r1 = ops["V"] @ t - (ops["K"] - 0.5 * ops["M"]) @ gX
        res1.append(np.linalg.norm(r1) / np.linalg.norm(ops["V"] @ t))
        lhs = P.T @ (0.5 * ops["M"] + ops["Kp"]) @ t
        r2 = lhs + P.T @ ops["W"] @ (P @ g0)
        res2.append(np.linalg.norm(r2) / np.linalg.norm(lhs))
    assert res1[1] < 5e-5 and res1[0] / res1[1] > 6
    assert res2[1] < 1e-3 and res2[0] / res2[1] > 3


def test_far_field_of_an_interior_point_source(ps):
    """DL(u) - SL(du/dn) reproduces u outside, so u_inf(x^) = exp(-i kappa x^.z0) / (4 pi)."""
    xh = inputs.fibonacci_directions(20)
    exact = np.exp(-1j * KAPPA * xh @ Z0) / (4 * np.pi)
    errs = []
    for m in (1, 2):
        sp, sp0, ops, t, gX, g0, P = ps[m]
        u = farfield.far_field(sp0, KAPPA, g0, xh, True) + farfield.far_field(sp, KAPPA, t, xh, False)
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 8
