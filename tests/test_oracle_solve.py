"""Pins of the oracle's full CFIE solves (CPU): the far field of the sound-soft and sound-hard unit
sphere against the Mie series, the convergence rate in h, GMRES against LU, and the Mie series
against its own closed-form limits."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import farfield, mie, solve
from tests import oracle_cache as C
from paper_2306_11324_gb300 import inputs

D = np.array([0.0, 0.0, 1.0])


def _solve(m, p, kappa, hard):
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard)
    b = A.rhs(sp, kappa, kappa, D, hard)
    return sp, Amat, b, solve.lu_solve(Amat, b)


def _err(sp, kappa, x, hard):
    xh = inputs.fibonacci_directions(100)
    u = farfield.far_field(sp, kappa, x, xh, hard)
    um = mie.mie_far_field(kappa, xh, D, hard)
    return np.abs(u - um).max() / np.abs(um).max()


def test_sound_soft_sphere_matches_mie_with_rate():
    """p = 1: the far-field error falls like h^(2p+2) = h^4 (Sec. 5.2)."""
    e1 = _err(*_solve(1, 1, 1.0, False)[0:1], 1.0, _solve(1, 1, 1.0, False)[3], False)
    e2 = _err(*_solve(2, 1, 1.0, False)[0:1], 1.0, _solve(2, 1, 1.0, False)[3], False)
    assert e2 < 2e-4
    assert e1 / e2 > 10                     # 2^4 = 16 asymptotically


def test_sound_hard_sphere_matches_mie():
    sp, _, _, x = _solve(2, 1, 1.0, True)
    assert _err(sp, 1.0, x, True) < 3e-3
    sp1, _, _, x1 = _solve(1, 1, 1.0, True)
    assert _err(sp1, 1.0, x1, True) / _err(sp, 1.0, x, True) > 4     # h^(2p+1) = h^3


def test_sign_of_the_single_layer_representation():
    """With the paper's '+' in front of the single layer the far field would be -u_inf: the Mie
    comparison fails by O(1)."""
    sp, _, _, x = _solve(1, 1, 1.0, False)
    xh = inputs.fibonacci_directions(50)
    um = mie.mie_far_field(1.0, xh, D)
    wrong = -farfield.far_field(sp, 1.0, x, xh, False)
    assert np.abs(wrong - um).max() / np.abs(um).max() > 1.0


def test_gmres_matches_lu():
    sp, Amat, b, x = _solve(2, 1, 1.0, False)
    xg, it, res = solve.gmres(lambda v: Amat @ v, b, tol=1e-10, restart=30)
    assert res <= 1e-10
    assert np.linalg.norm(Amat @ xg - b) <= 1.1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(xg - x) < 1e-8 * np.linalg.norm(x)
    xr, it_r, _ = solve.gmres(lambda v: Amat @ v, b, tol=1e-10, restart=5)
    assert it_r > it and np.linalg.norm(xr - x) < 1e-8 * np.linalg.norm(x)


def test_mie_limits_and_optical_theorem():
    xh = inputs.fibonacci_directions(2000)
    # sound-soft, kappa -> 0: u_s -> -1/r, so u_inf -> -1
    assert np.abs(mie.mie_far_field(1e-4, xh[:5]) + 1).max() < 1e-3
    for hard in (False, True):
        for kappa in (0.5, 3.0, 10.0):
            u = mie.mie_far_field(kappa, xh, D, hard)
            u0 = mie.mie_far_field(kappa, D[None, :], D, hard)[0]
            # optical theorem: int_S2 |u_inf|^2 = (4 pi / kappa) Im u_inf(d)
            assert abs(4 * np.pi * np.mean(np.abs(u) ** 2) / (4 * np.pi / kappa * u0.imag) - 1) < 2e-3
    # sound-hard, kappa -> 0: no monopole; u_inf = O(kappa^2)
    assert np.abs(mie.mie_far_field(1e-3, xh[:5], D, True)).max() < 1e-5


def test_point_source_right_hand_side_tends_to_the_plane_wave_one():
    """A point source far away in the direction -d is a plane wave of direction d times
    G(|z|) = exp(i kappa |z|)/(4 pi |z|), up to O(1/|z|): the point-source load vectors divided by G(|z|)
    approach the plane-wave ones at that rate (sound-soft and sound-hard)."""
    d = np.array([0.0, 0.6, 0.8])
    k = 2.0
    for hard in (False, True):
        sp = C.sphere_space(1, 1, hard)
        ref = A.rhs(sp, k, k, d, hard)
        errs = []
        for Rz in (1e3, 1e5):
            b = A.rhs_point_sources(sp, k, k, -Rz * d, hard)[:, 0]
            g = np.exp(1j * k * Rz) / (4 * np.pi * Rz)
            errs.append(np.abs(b / g - ref).max() / np.abs(ref).max())
        assert errs[0] < 10.0 / 1e3 and 50 < errs[0] / errs[1] < 200


@pytest.mark.parametrize("hard", [False, True])
def test_potential_matches_the_mie_near_field(hard):
    """The scattered field at points off the unit sphere (Sec. 5.3's potential evaluation) from the
    oracle's LU density, against the Mie series near field (r = 1.5 .. 5); the error shrinks under
    refinement like the far field's."""
    rng = np.random.default_rng(4)
    P = rng.standard_normal((12, 3))
    P *= (rng.uniform(1.5, 5.0, 12) / np.linalg.norm(P, axis=1))[:, None]
    ref = mie.mie_scattered_field(1.0, P, D, hard)
    errs = []
    for m in (1, 2):
        sp, Amat, b, x = _solve(m, 1, 1.0, hard)
        u = farfield.potential(sp, 1.0, x, P, hard)
        errs.append(np.abs(u - ref).max() / np.abs(ref).max())
    assert errs[1] < 2e-3 and errs[1] < errs[0] / 4
