"""The torus of the paper's convergence study (Sec. 5.2: R = 2, r = 0.5, 16 exact rational patches,
kappa = 2.5, plane wave d = x^) and incident point sources: the CUDA path through the C ABI against
the oracle (point-source load vectors; the dense Galerkin matrix on the torus) and the far field's
convergence in h."""
import functools

import numpy as np
import pytest

from oracle import assemble as A
from oracle import space as S
from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G
from tests import oracle_cache as C

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _torus_geom():
    return B.igabem_geometry_create(G.ctx(), inputs.torus_patches(2.0, 0.5))


@pytest.mark.parametrize("hard", [False, True])
def test_point_source_right_hand_sides_match_oracle(hard):
    prob, info = G.problem(level_m=2, degree_p=1, kappa=2.0, eta_cfie=2.0, bc=int(hard), no_fmm=1)
    z = np.array([[3.0, -1.0, 2.0], [0.0, 0.0, -4.0]])
    b = B.igabem_rhs_sources(prob, z, info["n_dofs"])
    ref = A.rhs_point_sources(C.sphere_space(2, 1, hard), 2.0, 2.0, z, hard)
    assert G.rel(b, ref) < 1e-10
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard", [False, True])
def test_torus_dense_matvec_matches_exact_galerkin_matrix(hard):
    """Degree-2 rational patches, a closed surface of Euler characteristic 0: the exact Galerkin matrix
    (every pair near) on the torus with 4 elements per patch."""
    opt = B.igabem_default_options(level_m=1, degree_p=1, kappa=2.5, eta_cfie=2.5, bc=int(hard), no_fmm=1)
    prob = B.igabem_problem_create(_torus_geom(), opt)
    info = B.igabem_problem_info(prob)
    sp = S.Space(S.Mesh(inputs.torus_patches(2.0, 0.5), 1), 1, continuous=hard)
    Amat = A.cfie_matrix(sp, 2.5, 2.5, hard)
    assert info["n_dofs"] == sp.N
    x = inputs.random_complex(sp.N, seed=12, cols=2)
    assert G.rel(B.igabem_matvec(prob, x), Amat @ x) < 1e-10
    B.igabem_problem_destroy(prob)


def test_torus_far_field_converges_like_h_to_the_2p_plus_2():
    """Sec. 5.2: kappa = 2.5, d = x^, p = 1, sound-soft, FP64 with level-adaptive interpolation; the far
    field at 100 directions at m = 1..3 against m = 5: the error falls like h^(2p+2) = h^4."""
    xh = inputs.fibonacci_directions(100)
    d = np.array([[1.0, 0.0, 0.0]])
    u = {}
    for m in (1, 2, 3, 5):
        opt = B.igabem_default_options(level_m=m, degree_p=1, kappa=2.5, eta_cfie=2.5, cheb_q=8, kappa_cap=2.0,
                                       q_max=14, leaf_offset=min(m, 1), eta_adm=0.5, tol=1e-11, precond=1)
        prob = B.igabem_problem_create(_torus_geom(), opt)
        info = B.igabem_problem_info(prob)
        x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
        u[m] = B.igabem_farfield(prob, x, xh)[:, 0]
        B.igabem_problem_destroy(prob)
    e = [np.abs(u[m] - u[5]).max() / np.abs(u[5]).max() for m in (1, 2, 3)]
    rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    print("torus far-field errors", e, "orders", rates)
    assert e[2] < e[1] < e[0]
    assert rates[-1] > 3.0
