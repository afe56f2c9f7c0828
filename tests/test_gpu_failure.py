"""Failure detection on the device without a fault: a bounded device wait that runs out (on a barrier
nothing arrives at) is reported as IGABEM_ETIMEOUT, and the context keeps working."""
import time

import numpy as np
import pytest

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

ETIMEOUT, EINVAL = -6, -1


def test_bounded_wait_reports_timeout_and_the_context_survives():
    t0 = time.perf_counter()
    rc = B.igabem_wait_selftest(G.ctx(), 0.2)
    elapsed = time.perf_counter() - t0
    assert rc == ETIMEOUT
    assert "gave up" in B.igabem_last_error()
    assert 0.2 <= elapsed < 5.0
    prob, info = G.problem(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, no_fmm=1)
    y = B.igabem_matvec(prob, inputs.random_complex(info["n_dofs"], seed=5))
    assert np.isfinite(y).all() and np.abs(y).max() > 0
    B.igabem_problem_destroy(prob)
    assert B.igabem_wait_selftest(G.ctx(), 0.0) == EINVAL
