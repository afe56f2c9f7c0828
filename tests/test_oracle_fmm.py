"""Pins of the oracle's cluster tree and interpolated-kernel matrix (CPU)."""
import numpy as np
import pytest

from oracle import fmm
from tests import oracle_cache as C
from paper_2306_11324_gb300 import inputs


@pytest.mark.parametrize("leaf,eta", [(2, 0.5), (1, 0.5), (2, 1.6)])
def test_block_partition_covers_every_element_pair_once(leaf, eta):
    t = C.tree(2, 1, leaf, eta, 5, 1.0)
    cnt = t.cover_check()
    assert cnt.min() == 1 and cnt.max() == 1
    for l, pairs in enumerate(t.far):
        for a, b in pairs:
            assert t.admissible(l, a, b)
    for a, b in t.near:
        assert not t.admissible(t.L, a, b)


def test_lagrange_interpolation_reproduces_polynomials():
    for q in (3, 5, 7):
        nodes = fmm.cheb_nodes(q, 0.25, 0.5)
        s = np.linspace(0.25, 0.5, 17)
        L = fmm.lagrange(nodes, s)
        assert np.abs(L.sum(axis=1) - 1).max() < 1e-13
        for k in range(q):
            assert np.abs(L @ nodes ** k - s ** k).max() < 1e-13
        assert np.abs(L @ nodes ** q - s ** q).max() > 1e-10


@pytest.mark.parametrize("hard", [False, True])
def test_mode_b_converges_to_the_exact_matrix_in_q(hard):
    """Sec. 4.4: the interpolated kernel tends to the exact one as q grows, so every operator's mode-B
    matrix tends to its exact Galerkin matrix.  Sound-soft checks V and K'; sound-hard checks K (the
    pull-back kernel a_x dG/dn_y with the normal at the source nodes) and W (G alone interpolated, the
    curl and normal factors of Maue's form kept at the quadrature points).  A transposed normal, a
    wrong channel factor or a dropped term would leave an O(1) far-block error that does not decay."""
    ops = ("K", "W") if hard else ("V", "Kp")
    ex = C.operators(2, 1, 1.0, ops, hard)
    errs = []
    for q in (3, 5):
        mb = C.modeb(2, 1, 1.0, ops, 2, 0.5, q, hard=hard)
        errs.append(max(np.abs(mb[o] - ex[o]).max() / np.abs(ex[o]).max() for o in ops))
    assert errs[0] < 1e-4 and errs[1] < 1e-7 and errs[0] / errs[1] > 100


@pytest.mark.parametrize("hard", [False, True])
def test_sampled_rows_equal_the_dense_mode_b_matrix(hard):
    """cfie_rows (the row-by-row reference of the large GPU parity tests) equals the dense mode-B CFIE
    matrix: sound-soft 1/2 M + K' - i eta V on S^2, sound-hard 1/2 M - K - i eta W on S^0 (Sec. 4.1)."""
    sp = C.sphere_space(2, 1, hard)
    Amat = C.cfie(2, 1, 1.0, 1.0, hard, mode_b=(2, 0.5, 3))
    x = inputs.random_complex(sp.N)
    rows = np.array([0, 7, 33, sp.N - 1])
    r = fmm.cfie_rows(sp, 1.0, 1.0, hard, x, rows, C.tree(2, 1, 2, 0.5, 3, 1.0, hard))
    assert np.abs(r - (Amat @ x)[rows]).max() < 1e-13 * np.abs(Amat @ x).max()


def test_chebyshev_error_bound_of_the_level_rule():
    """eps(q, omega) = omega^q / (2^(q-1) q!) bounds the error of q-point Chebyshev interpolation of
    exp(i omega t) on [-1, 1], and is within a factor 2 of the true error (brute force on a fine grid):
    a wrong power of two or factorial in the level rule fails here."""
    t = np.linspace(-1.0, 1.0, 4001)
    checked = 0
    for q in (3, 5, 7, 10, 12):
        nodes = fmm.cheb_nodes(q, -1.0, 1.0)
        L = fmm.lagrange(nodes, t)
        for omega in (0.5, 1.0, 2.0, 3.0, 5.0):
            bound = fmm.cheb_error_bound(q, omega)
            if not 1e-12 < bound < 1e-2:
                continue
            err = np.abs(L @ np.exp(1j * omega * nodes) - np.exp(1j * omega * t)).max()
            assert err <= bound * (1 + 1e-6), (q, omega, err, bound)
            assert err >= bound / 2, (q, omega, err, bound)
            checked += 1
    assert checked >= 8


def test_level_rule_takes_the_smallest_q_that_meets_the_finest_levels_accuracy():
    kappa, q0, cap0, qmax = 60.0, 7, 6.0, 12
    diam = [2.5 / 2 ** l for l in range(8)]
    qs, caps = fmm.level_q_and_caps(kappa, diam, q0, cap0, qmax)
    eps_ref = fmm.cheb_error_bound(q0, cap0 / 2)
    for D, q, c in zip(diam, qs, caps):
        if q < qmax:
            assert fmm.cheb_error_bound(q, kappa * D / 2) <= eps_ref
        if q > q0:
            assert fmm.cheb_error_bound(q - 1, kappa * D / 2) > eps_ref
        assert abs(fmm.cheb_error_bound(q, c / 2) - eps_ref) <= 1e-9 * eps_ref
    assert qs == sorted(qs, reverse=True) and qs[0] == qmax and qs[-1] == q0 and caps[-1] == cap0
    assert len(set(qs)) >= 3
    # q_max = q0 (or no cap) is the fixed-q tree of Sec. 4.4
    assert fmm.level_q_and_caps(kappa, diam, q0, cap0, q0) == ([q0] * 8, [cap0] * 8)
    assert fmm.level_q_and_caps(kappa, diam, q0, np.inf, qmax) == ([q0] * 8, [np.inf] * 8)


def test_adaptive_tree_covers_every_pair_once_with_far_blocks_of_two_degrees():
    """The unit sphere at m = 3, kappa = 8, q0 = 4, cap 2, q_max = 8: far blocks on level 2 take 6 points
    per direction and on level 3 take 5; the block partition still covers every element pair once, and
    every far block meets its level's cap."""
    sp = C.sphere_space(3, 1)
    t = fmm.ClusterTree(sp.mesh, 3, 0.5, 4, 8.0, kappa_cap=2.0, q_max=8)
    assert t.ql[2:] == [6, 5]
    assert len(t.far[2]) > 0 and len(t.far[3]) > 0
    cnt = t.cover_check()
    assert cnt.min() == 1 and cnt.max() == 1
    for l, pairs in enumerate(t.far):
        for a, b in pairs:
            assert 8.0 * 2 * max(t.radius[l][a], t.radius[l][b]) <= t.caps[l]
