"""Potential evaluation at many points (NEXT-1: the physical-space interpolation FMM of rank q^3 of
Sec. 4.4 / 5.3) through the C ABI: the direct sum equals the oracle's representation formula at every
point, the fast method agrees with the direct sum to its interpolation accuracy, and a solved density's
scattered field approaches the Mie near field."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import farfield, mie, solve
from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G
from tests import oracle_cache as C

pytestmark = pytest.mark.gpu


def _shell(n, r0, r1, seed):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n, 3))
    return P * (rng.uniform(r0, r1, n) / np.linalg.norm(P, axis=1))[:, None]


@pytest.mark.parametrize("hard", [False, True])
def test_direct_potential_matches_oracle(hard):
    prob, info = G.problem(level_m=2, degree_p=1, kappa=2.0, eta_cfie=2.0, bc=int(hard), no_fmm=1)
    sp = C.sphere_space(2, 1, hard)
    x = inputs.random_complex(sp.N, seed=21, cols=2)
    P = _shell(20, 1.3, 5.0, 8)
    u = B.igabem_potential(prob, x, P)
    ref = np.stack([farfield.potential(sp, 2.0, x[:, r], P, hard) for r in range(2)], axis=1)
    assert G.rel(u, ref) < 1e-10
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard,prec", [(False, B.FP64), (True, B.FP64), (False, B.MIXED_FP32)])
def test_fast_potential_matches_direct_sum(hard, prec):
    """24576 Gauss points, 6000 points in the shell 1.2 < r < 5: the octree FMM (7^3 nodes per box)
    against the direct sum."""
    kw = dict(level_m=4, degree_p=2, kappa=4.0, eta_cfie=4.0, bc=int(hard), cheb_q=7, leaf_offset=2, eta_adm=0.5)
    fast, info = G.problem(precision=prec, **kw)
    direct, _ = G.problem(no_fmm=1, **kw)
    x = inputs.random_complex(info["n_dofs"], seed=22, cols=3)
    P = _shell(6000, 1.2, 5.0, 9)
    uf = B.igabem_potential(fast, x, P)
    ud = B.igabem_potential(direct, x, P)
    err = G.rel(uf, ud)
    print(f"fast potential vs direct: {err:.2e}")
    assert err < 1e-4
    B.igabem_problem_destroy(fast)
    B.igabem_problem_destroy(direct)


def test_solved_scattered_field_approaches_mie():
    """Sound-soft unit sphere, kappa = 2, degree 2, 16 x 16 elements per patch: GMRES density, the fast
    potential at 2000 points against the Mie near field."""
    prob, info = G.problem(level_m=4, degree_p=2, kappa=2.0, eta_cfie=2.0, cheb_q=7, leaf_offset=2, tol=1e-9,
                           precond=1)
    d = np.array([[0.0, 0.0, 1.0]])
    x, _ = B.igabem_solve(prob, d, info["n_dofs"])
    P = _shell(2000, 1.5, 5.0, 10)
    u = B.igabem_potential(prob, x, P)[:, 0]
    ref = mie.mie_scattered_field(2.0, P, d[0])
    err = G.rel(u, ref)
    print(f"scattered field vs Mie: {err:.2e}")
    assert err < 1e-4
    B.igabem_problem_destroy(prob)
