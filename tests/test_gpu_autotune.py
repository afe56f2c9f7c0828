"""The layout autotuner (igabem_autotune): it times the candidate leaf sizes and M2L storage modes on
the device, returns one of them, serves the same key from its cache (memory and file), and the tuned
options give the same operator as the caller's."""
import os

import numpy as np
import pytest

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_caches_it_and_keeps_the_operator(tmp_path):
    kw = dict(level_m=4, degree_p=2, kappa=6.0, eta_cfie=6.0, cheb_q=7, kappa_cap=4.0, eta_adm=0.5,
              precision=B.MIXED_FP32, leaf_offset=2)
    opt = B.igabem_default_options(**kw)
    path = str(tmp_path / "tune.txt")
    tuned, info = B.igabem_autotune(G.geometry("sphere"), opt, 4, 30, path)
    print(info)
    assert info["from_cache"] == 0 and info["candidates"] >= 4
    assert tuned.leaf_offset in (1, 2, 3) and tuned.m2l_stored in (0, 1)
    assert info["score_ms"] == pytest.approx(info["setup_ms"] + 30 * info["matvec_ms"], rel=1e-9)
    assert os.path.exists(path) and open(path).read().strip()
    again, info2 = B.igabem_autotune(G.geometry("sphere"), opt, 4, 30, path)
    assert info2["from_cache"] == 1
    assert (again.leaf_offset, again.m2l_stored) == (tuned.leaf_offset, tuned.m2l_stored)
    # every option other than the layout is the caller's, and the operator is the same up to the
    # interpolation of the different tree (compare with the caller's layout at the FP32 level)
    assert tuned.kappa == opt.kappa and tuned.cheb_q == opt.cheb_q and tuned.precision == opt.precision
    p0 = B.igabem_problem_create(G.geometry("sphere"), opt)
    p1 = B.igabem_problem_create(G.geometry("sphere"), tuned)
    N = B.igabem_problem_info(p0)["n_dofs"]
    x = inputs.random_complex(N, seed=5, cols=4)
    y0, y1 = B.igabem_matvec(p0, x), B.igabem_matvec(p1, x)
    assert G.rel(y1, y0) < 1e-4
    B.igabem_problem_destroy(p0)
    B.igabem_problem_destroy(p1)
