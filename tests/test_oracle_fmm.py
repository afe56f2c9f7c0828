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


def test_mode_b_converges_to_the_exact_matrix_in_q():
    ex = C.operators(2, 1, 1.0, ("V", "Kp"))
    errs = []
    for q in (3, 5):
        mb = C.modeb(2, 1, 1.0, ("V", "Kp"), 2, 0.5, q)
        errs.append(max(np.abs(mb[o] - ex[o]).max() / np.abs(ex[o]).max() for o in ("V", "Kp")))
    assert errs[0] < 1e-4 and errs[1] < 1e-7 and errs[0] / errs[1] > 100


def test_sampled_rows_equal_the_dense_mode_b_matrix():
    sp = C.sphere_space(2, 1)
    Amat = C.cfie(2, 1, 1.0, 1.0, False, mode_b=(2, 0.5, 3))
    x = inputs.random_complex(sp.N)
    rows = np.array([0, 7, 33, 149])
    r = fmm.cfie_rows(sp, 1.0, 1.0, False, x, rows, C.tree(2, 1, 2, 0.5, 3, 1.0))
    assert np.abs(r - (Amat @ x)[rows]).max() < 1e-13 * np.abs(Amat @ x).max()
