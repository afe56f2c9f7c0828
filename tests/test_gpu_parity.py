"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element, on
small seeded problems that span several clusters and leaf blocks."""
import functools

import numpy as np
import pytest

from oracle import assemble as A
from oracle import farfield, fmm, mie, solve
from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G
from tests import oracle_cache as C

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10        # same definitions in FP64: only rounding order differs
DIRS = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, -1.0, 0.0]])


@pytest.mark.parametrize("hard", [False, True])
def test_rhs(hard):
    prob, info = G.problem(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, bc=int(hard), no_fmm=1)
    b = B.igabem_rhs(prob, DIRS, info["n_dofs"])
    sp = C.sphere_space(2, 1, hard)
    ref = A.rhs(sp, 1.0, 1.0, DIRS, hard)
    assert info["n_dofs"] == sp.N
    assert G.rel(b, ref) < FP64_TOL
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard", [False, True])
def test_dense_matvec_matches_exact_galerkin_matrix(hard):
    """no_fmm: every element pair in the near field, i.e. the exact ("mode A") Galerkin matrix."""
    prob, info = G.problem(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, bc=int(hard), no_fmm=1)
    sp = C.sphere_space(2, 1, hard)
    Amat = C.cfie(2, 1, 1.0, 1.0, hard)
    x = inputs.random_complex(sp.N, seed=1234, cols=2)
    y = B.igabem_matvec(prob, x)
    assert G.rel(y, Amat @ x) < FP64_TOL
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard,leaf,q", [(False, 2, 3), (False, 1, 5), (True, 2, 3)])
def test_fmm_matvec_matches_interpolated_kernel_matrix(hard, leaf, q):
    """FMM matvec = the oracle's mode-B matrix (interpolated kernel on admissible blocks)."""
    m, p, kappa = 2, 1, 1.0
    prob, info = G.problem(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard),
                           cheb_q=q, leaf_offset=m - leaf, eta_adm=0.5)
    assert info["n_far_pairs"] == sum(len(f) for f in C.tree(m, p, leaf, 0.5, q, kappa, hard).far)
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard, mode_b=(leaf, 0.5, q))
    x = inputs.random_complex(sp.N, seed=1234)
    y = B.igabem_matvec(prob, x)
    assert G.rel(y, Amat @ x) < FP64_TOL
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard", [False, True])
def test_farfield(hard):
    prob, info = G.problem(level_m=2, degree_p=1, kappa=2.0, eta_cfie=2.0, bc=int(hard), no_fmm=1)
    sp = C.sphere_space(2, 1, hard)
    x = inputs.random_complex(sp.N, seed=7, cols=2)
    xh = inputs.fibonacci_directions(37)
    u = B.igabem_farfield(prob, x, xh)
    ref = np.stack([farfield.far_field(sp, 2.0, x[:, r], xh, hard) for r in range(2)], axis=1)
    assert G.rel(u, ref) < FP64_TOL
    B.igabem_problem_destroy(prob)


def test_solve_sound_soft_sphere():
    """GMRES(30) on the GPU reaches the oracle's LU solution; the far field matches Mie."""
    prob, info = G.problem(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, no_fmm=1, tol=1e-10)
    sp = C.sphere_space(2, 1)
    Amat = C.cfie(2, 1, 1.0, 1.0, False)
    d = np.array([[0.0, 0.0, 1.0]])
    x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
    ref = solve.lu_solve(Amat, A.rhs(sp, 1.0, 1.0, d[0], False))
    assert sinfo["rel_residual"] <= 1e-10
    assert G.rel(x[:, 0], ref) < 1e-8
    xh = inputs.fibonacci_directions(100)
    u = B.igabem_farfield(prob, x, xh)[:, 0]
    assert G.rel(u, mie.mie_far_field(1.0, xh)) < 2e-4
    B.igabem_problem_destroy(prob)


MIXED_MATVEC_TOL = 2e-6   # FP32 far field (phase-split kernel samples, FP32 accumulation)
# tensor-core M2L: FP16 split products (hi hi + hi lo + lo hi, each scaled operand to ~2^-22 of its
# largest entry) summed by the tensor core into FP32 per pair, pairs added in FP32
MIXED_TC_TOL = 1e-5


@pytest.mark.parametrize("hard,kappa", [(False, 1.0), (False, 6.0), (True, 3.0)])
def test_mixed_fmm_matvec_matches_interpolated_kernel_matrix(hard, kappa):
    """FP32 M2L (mixed precision) against the FP64 mode-B matrix of the oracle."""
    m, p, leaf, q = 2, 1, 2, 5
    prob, info = G.problem(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=q,
                           leaf_offset=m - leaf, eta_adm=0.5, precision=B.MIXED_FP32)
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard, mode_b=(leaf, 0.5, q))
    x = inputs.random_complex(sp.N, seed=1234)
    y = B.igabem_matvec(prob, x)
    assert G.rel(y, Amat @ x) < MIXED_MATVEC_TOL
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard", [False, True])
def test_mixed_solve_far_field_matches_fp64(hard):
    """The mixed-precision solve reproduces the FP64 far field to 1e-5."""
    kw = dict(level_m=3, degree_p=2, kappa=4.0, eta_cfie=4.0, bc=int(hard), cheb_q=7, leaf_offset=1)
    xh = inputs.fibonacci_directions(100)
    d = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    u = {}
    # FP64 to 1e-8; the mixed operator carries FP32 rounding (~1e-7 of ||A x||), so its GMRES stops
    # at 1e-6
    for prec, tol in ((B.FP64, 1e-8), (B.MIXED_FP32, 1e-6)):
        prob, info = G.problem("deformed" if hard else "sphere", precision=prec, tol=tol, **kw)
        x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
        assert sinfo["rel_residual"] <= tol
        u[prec] = B.igabem_farfield(prob, x, xh)
        B.igabem_problem_destroy(prob)
    assert G.rel(u[B.MIXED_FP32], u[B.FP64]) < 1e-5


@pytest.mark.parametrize("R", [6, 16])
@pytest.mark.parametrize("prec,hard", [(B.FP64, False), (B.FP64, True), (B.MIXED_FP32, False),
                                       (B.MIXED_FP32, True)])
def test_multi_rhs_fmm_matvec(prec, hard, R):
    """Several right-hand sides at once (the multi-column M2L; from 8 columns on also the many-column
    near-field SpMV and the moment-matrix P2M / L2P): every column against the oracle."""
    m, p, leaf, q, kappa = 2, 1, 2, 5, 3.0
    prob, info = G.problem(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=q,
                           leaf_offset=m - leaf, eta_adm=0.5, precision=prec)
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard, mode_b=(leaf, 0.5, q))
    x = inputs.random_complex(sp.N, seed=77, cols=R)
    y = B.igabem_matvec(prob, x)
    tol = FP64_TOL if prec == B.FP64 else MIXED_MATVEC_TOL
    assert G.rel(y, Amat @ x) < tol
    # the same columns one at a time give the same result
    y0 = B.igabem_matvec(prob, np.ascontiguousarray(x[:, 2]))
    assert G.rel(y0, y[:, 2]) < (1e-13 if prec == B.FP64 else MIXED_MATVEC_TOL)
    B.igabem_problem_destroy(prob)


def _m2l_launches(prob):
    return B.igabem_profile_get(prob, reset=True)["phases"]["m2l"]["launches"]


@pytest.mark.parametrize("hard,R", [(False, 16), (False, 64), (True, 16), (True, 32)])
def test_tensor_core_m2l_matches_oracle(hard, R):
    """tcgen05 M2L (FP16 hi/lo split, FP32 accumulation) against the oracle's mode-B matrix, every column."""
    m, p, leaf, q, kappa = 2, 1, 2, 5, 3.0
    prob, info = G.problem(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=q,
                           leaf_offset=m - leaf, eta_adm=0.5, precision=B.MIXED_TC)
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard, mode_b=(leaf, 0.5, q))
    x = inputs.random_complex(sp.N, seed=78, cols=R)
    _m2l_launches(prob)
    y = B.igabem_matvec(prob, x)
    launches = _m2l_launches(prob)
    assert launches >= 2            # operand packing per level + the tensor-core kernel
    ref = Amat @ x
    # the same product with the FP32 CUDA-core M2L, for the record
    prob32, _ = G.problem(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=q,
                          leaf_offset=m - leaf, eta_adm=0.5, precision=B.MIXED_FP32)
    y32 = B.igabem_matvec(prob32, x)
    B.igabem_problem_destroy(prob32)
    print(f"tensor-core M2L rel. error {G.rel(y, ref):.2e}, FP32 M2L {G.rel(y32, ref):.2e}")
    assert G.rel(y32, ref) < MIXED_MATVEC_TOL
    assert G.rel(y, ref) < MIXED_TC_TOL
    # a column count the tensor-core path does not take (not a multiple of 16) runs the FP32 M2L
    y5 = B.igabem_matvec(prob, np.ascontiguousarray(x[:, :5]))
    assert _m2l_launches(prob) == 1
    assert G.rel(y5, ref[:, :5]) < MIXED_MATVEC_TOL
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("hard", [False, True])
def test_tensor_core_m2l_q7_against_fp64(hard):
    """q = 7 (the benchmark's interpolation degree), many clusters and pairs: tcgen05 M2L against the
    FP64 GPU path and against the FP32 CUDA-core M2L."""
    m, R = 4, (32 if hard else 64)
    kw = dict(level_m=m, degree_p=2, kappa=6.0, eta_adm=0.5, eta_cfie=6.0, bc=int(hard), cheb_q=7, leaf_offset=1)
    kind = "deformed" if hard else "sphere"
    ys = {}
    for prec in (B.FP64, B.MIXED_FP32, B.MIXED_TC):
        prob, info = G.problem(kind, precision=prec, **kw)
        if prec == B.FP64:
            x = inputs.random_complex(info["n_dofs"], seed=79, cols=R)
        _m2l_launches(prob)
        ys[prec] = B.igabem_matvec(prob, x)
        if prec == B.MIXED_TC:
            assert _m2l_launches(prob) >= 2
        B.igabem_problem_destroy(prob)
    print(f"q=7: tensor-core vs FP64 {G.rel(ys[B.MIXED_TC], ys[B.FP64]):.2e}, "
          f"FP32 vs FP64 {G.rel(ys[B.MIXED_FP32], ys[B.FP64]):.2e}")
    assert G.rel(ys[B.MIXED_FP32], ys[B.FP64]) < MIXED_MATVEC_TOL
    assert G.rel(ys[B.MIXED_TC], ys[B.FP64]) < MIXED_TC_TOL


@functools.lru_cache(maxsize=None)
def _three_level_rows(hard, col):
    """Oracle rows of the mode-B product on a three-level tree (far pairs on levels 2 and 3)."""
    sp = C.sphere_space(3, 1, hard)
    x = inputs.random_complex(sp.N, seed=91, cols=16)
    rows = np.array([0, 77, sp.N // 2, sp.N - 1])
    tree = C.tree(3, 1, 3, 0.5, 4, 2.0, hard)
    return rows, fmm.cfie_rows(sp, 2.0, 2.0, hard, x[:, col], rows, tree=tree)


@pytest.mark.parametrize("prec,hard", [(B.FP64, False), (B.FP64, True), (B.MIXED_TC, True)])
def test_transfers_three_levels(prec, hard):
    """M2M / L2L between two levels with many columns (separable transfers): sampled rows of two
    columns against the oracle, every column against the one-column path."""
    prob, info = G.problem(level_m=3, degree_p=1, kappa=2.0, eta_cfie=2.0, bc=int(hard), cheb_q=4,
                           leaf_offset=0, eta_adm=0.5, precision=prec)
    sp = C.sphere_space(3, 1, hard)
    assert info["n_far_pairs"] == sum(len(f) for f in C.tree(3, 1, 3, 0.5, 4, 2.0, hard).far)
    x = inputs.random_complex(sp.N, seed=91, cols=16)
    y = B.igabem_matvec(prob, x)
    tol = FP64_TOL if prec == B.FP64 else MIXED_MATVEC_TOL
    for col in (0, 9):
        rows, ref = _three_level_rows(hard, col)
        assert np.abs(y[rows, col] - ref).max() / np.abs(y[:, col]).max() < tol
    for col in (0, 5, 15):
        y1 = B.igabem_matvec(prob, np.ascontiguousarray(x[:, col]))
        assert G.rel(y[:, col], y1) < (1e-12 if prec == B.FP64 else MIXED_MATVEC_TOL)
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("n_dirs", [1, 8])
@pytest.mark.parametrize("hard", [False, True])
def test_preconditioned_solve_matches_lu(hard, n_dirs):
    """The block-Jacobi right preconditioner changes the iterations, not the solution (one column,
    and eight columns through the many-column SpMV and block apply)."""
    kappa = 2.0
    sp = C.sphere_space(2, 1, hard)
    Amat = C.cfie(2, 1, kappa, kappa, hard)
    d = inputs.fibonacci_directions(n_dirs) if n_dirs > 1 else np.array([[0.0, 0.6, 0.8]])
    ref = solve.lu_solve(Amat, A.rhs(sp, kappa, kappa, d, hard)).reshape(sp.N, n_dirs)
    its = {}
    for pc in (0, 1):
        prob, info = G.problem(level_m=2, degree_p=1, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=4,
                               leaf_offset=1, eta_adm=0.5, no_fmm=1, tol=1e-10, precond=pc)
        x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
        assert sinfo["rel_residual"] <= 1e-10
        for r in range(n_dirs):
            assert G.rel(x[:, r], ref[:, r]) < 1e-8
        its[pc] = sinfo["iterations"]
        B.igabem_problem_destroy(prob)
    if not hard:                   # second-kind equation: the local blocks capture it well
        assert its[1] < its[0]


@functools.lru_cache(maxsize=None)
def _adaptive_rows():
    """Oracle rows of the mode-B product with level-adaptive q: unit sphere m = 3, kappa = 16,
    cheb_q = 4, cap 2, q_max = 10, element leaves: far blocks on level 2 with 10 x 10 points and on
    level 3 with 6 x 6 (three columns)."""
    sp = C.sphere_space(3, 1)
    x = inputs.random_complex(sp.N, seed=93, cols=3)
    tree = fmm.ClusterTree(sp.mesh, 3, 0.5, 4, 16.0, kappa_cap=2.0, q_max=10)
    rows = np.array([0, 123, sp.N // 2, sp.N - 1])
    return tree, rows, fmm.cfie_rows(sp, 16.0, 16.0, False, x, rows, tree=tree)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED_FP32])
def test_level_adaptive_interpolation_matches_oracle(prec):
    """Level-adaptive q (NEXT-4): the per-level q and far-pair counts equal the oracle tree's; the
    product with 10 x 10 nodes on level 2 (more than 64 per cluster: row chunks in the M2L), formed
    from and evaluated at the Gauss points there (its children use 6 x 6), against the oracle rows,
    for one column and three columns."""
    prob, info = G.problem(level_m=3, degree_p=1, kappa=16.0, eta_cfie=16.0, cheb_q=4, kappa_cap=2.0, q_max=10,
                           leaf_offset=0, eta_adm=0.5, precision=prec)
    tree, rows, ref3 = _adaptive_rows()
    assert info["level_q"][2:] == tree.ql[2:] == [10, 6]
    assert info["level_far"] == [len(f) for f in tree.far]
    sp = C.sphere_space(3, 1)
    x = inputs.random_complex(sp.N, seed=93, cols=3)
    tol = FP64_TOL if prec == B.FP64 else MIXED_MATVEC_TOL
    y3 = B.igabem_matvec(prob, x)
    for col in range(3):
        ref = ref3[:, col]
        y1 = B.igabem_matvec(prob, np.ascontiguousarray(x[:, col]))
        assert np.abs(y1[rows] - ref).max() / np.abs(ref).max() < tol
        assert np.abs(y3[rows, col] - ref).max() / np.abs(ref).max() < tol
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("pc", [0, 1])
def test_graph_captured_gmres_equals_eager_launches(pc):
    """The GMRES iteration captured once as a CUDA graph (state on the device, flags read one iteration
    behind) gives the same iterates as the same kernels launched one by one: equal iteration counts and
    densities equal to rounding, for three directions that converge at different iterations."""
    d = inputs.fibonacci_directions(3)
    out = {}
    for ng in (0, 1):
        prob, info = G.problem(level_m=3, degree_p=2, kappa=4.0, eta_cfie=4.0, cheb_q=5, leaf_offset=1, eta_adm=0.5,
                               tol=1e-9, gmres_restart=8, precond=pc, no_graph=ng)
        x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
        assert sinfo["rel_residual"] <= 1e-9
        out[ng] = (x, sinfo)
        B.igabem_problem_destroy(prob)
    assert out[0][1]["iterations"] == out[1][1]["iterations"] > 8     # more than one restart cycle
    assert G.rel(out[0][0], out[1][0]) < 1e-12


@pytest.mark.parametrize("prec,hard,R", [(B.FP64, False, 1), (B.FP64, True, 3), (B.MIXED_FP32, False, 4),
                                         (B.MIXED_FP32, True, 1), (B.MIXED_TC, False, 16)])
def test_stored_coupling_blocks_match_oracle(prec, hard, R):
    """NEXT-2: the M2L coupling blocks generated once at set-up and streamed by every product (the
    paper's stored H^2 operator) give the oracle's mode-B product, and the same product as the
    blocks generated on the fly."""
    m, p, leaf, q, kappa = 2, 1, 2, 5, 3.0
    kw = dict(level_m=m, degree_p=p, kappa=kappa, eta_cfie=kappa, bc=int(hard), cheb_q=q, leaf_offset=m - leaf,
              eta_adm=0.5, precision=prec)
    prob, info = G.problem(m2l_stored=1, **kw)
    fly, _ = G.problem(**kw)
    sp = C.sphere_space(m, p, hard)
    Amat = C.cfie(m, p, kappa, kappa, hard, mode_b=(leaf, 0.5, q))
    x = inputs.random_complex(sp.N, seed=95, cols=R)
    y = B.igabem_matvec(prob, x)
    tol = FP64_TOL if prec == B.FP64 else MIXED_MATVEC_TOL
    assert G.rel(y, Amat @ x) < tol
    assert G.rel(y, B.igabem_matvec(fly, x)) < (1e-12 if prec == B.FP64 else MIXED_MATVEC_TOL)
    B.igabem_problem_destroy(prob)
    B.igabem_problem_destroy(fly)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED_FP32])
def test_stored_coupling_blocks_with_level_adaptive_q(prec):
    """Stored blocks of 10 x 10 and 6 x 6 nodes (level-adaptive q) against the oracle's mode-B rows."""
    prob, info = G.problem(level_m=3, degree_p=1, kappa=16.0, eta_cfie=16.0, cheb_q=4, kappa_cap=2.0, q_max=10,
                           leaf_offset=0, eta_adm=0.5, precision=prec, m2l_stored=1)
    tree, rows, ref3 = _adaptive_rows()
    sp = C.sphere_space(3, 1)
    x = inputs.random_complex(sp.N, seed=93, cols=3)
    y3 = B.igabem_matvec(prob, x)
    tol = FP64_TOL if prec == B.FP64 else MIXED_MATVEC_TOL
    assert np.abs(y3[rows] - ref3).max() / np.abs(ref3).max() < tol
    B.igabem_problem_destroy(prob)


def test_set_up_reused_across_wavenumbers_equals_a_fresh_set_up():
    """Problems on one geometry at the same level share its wavenumber-independent host set-up (element
    nets, touching pairs, cluster balls): the product of a problem whose set-up came from that cache
    equals the product of the same problem on a fresh geometry object."""
    patches = inputs.deformed_sphere_patches(spans=4)
    kw = dict(level_m=4, degree_p=2, eta_cfie=1.0, cheb_q=6, leaf_offset=2, eta_adm=0.5, kappa_cap=4.0, q_max=9,
              precision=B.FP64)
    g = B.igabem_geometry_create(G.ctx(), patches)
    p1 = B.igabem_problem_create(g, B.igabem_default_options(kappa=3.0, **kw))      # fills the cache
    p2 = B.igabem_problem_create(g, B.igabem_default_options(kappa=5.0, **kw))      # reuses it
    g2 = B.igabem_geometry_create(G.ctx(), patches)
    p3 = B.igabem_problem_create(g2, B.igabem_default_options(kappa=5.0, **kw))     # fresh
    i2, i3 = B.igabem_problem_info(p2), B.igabem_problem_info(p3)
    for k in ("n_dofs", "n_far_pairs", "n_near_pairs", "n_touching_pairs", "n_singular_points", "level_q"):
        assert i2[k] == i3[k], k
    x = inputs.random_complex(i2["n_dofs"], seed=77, cols=2)
    y2, y3 = B.igabem_matvec(p2, x), B.igabem_matvec(p3, x)
    assert G.rel(y2, y3) < 1e-13
    for p in (p1, p2, p3):
        B.igabem_problem_destroy(p)
    B.igabem_geometry_destroy(g)
    B.igabem_geometry_destroy(g2)
