"""Serving loop (continuous admission of concurrent requests): every request's result equals the same
request solved alone, admission by memory, timeouts and statistics."""
import numpy as np
import pytest

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

XH = inputs.fibonacci_directions(24)

# (geometry, options, incident directions)
MIX = [
    ("sphere", dict(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, bc=0, cheb_q=5, leaf_offset=0), 1),
    ("deformed", dict(level_m=3, degree_p=2, kappa=3.0, eta_cfie=3.0, bc=1, cheb_q=6, leaf_offset=1), 3),
    ("sphere", dict(level_m=3, degree_p=2, kappa=5.0, eta_cfie=5.0, bc=0, cheb_q=7, leaf_offset=1,
                    precision=B.MIXED_FP32), 2),
    ("deformed", dict(level_m=2, degree_p=2, kappa=2.0, eta_cfie=2.0, bc=0, cheb_q=5, leaf_offset=0), 1),
    ("sphere", dict(level_m=3, degree_p=1, kappa=4.0, eta_cfie=4.0, bc=1, cheb_q=6, leaf_offset=1), 4),
    ("deformed", dict(level_m=3, degree_p=2, kappa=6.0, eta_cfie=6.0, bc=0, cheb_q=7, leaf_offset=1,
                      precision=B.MIXED_FP32), 2),
]


def _tol(kw):
    """GMRES tolerance: 1e-8 in FP64; the mixed form stops at its FP32 rounding floor."""
    return 1e-8 if kw.get("precision", B.FP64) == B.FP64 else 1e-6


def _alone(kind, kw, R):
    prob, info = G.problem(kind, tol=_tol(kw), **kw)
    d = inputs.fibonacci_directions(R)
    x, _ = B.igabem_solve(prob, d, info["n_dofs"])
    u = B.igabem_farfield(prob, x, XH)
    B.igabem_problem_destroy(prob)
    return u


def test_each_result_is_the_same_alone_and_in_the_mix():
    srv = B.igabem_server_create(G.ctx(), 0, 3)
    reqs = []
    for rep in range(2):                       # twice the mix: more requests than slots
        for kind, kw, R in MIX:
            opt = B.igabem_default_options(tol=_tol(kw), **kw)
            reqs.append(B.igabem_submit(srv, G.geometry(kind), opt, inputs.fibonacci_directions(R), XH))
    for r in reqs:
        B.igabem_wait(r, 600.0)
    results = [B.igabem_result(r) for r in reqs]
    stats = B.igabem_server_get_stats(srv)
    for r in reqs:
        B.igabem_request_destroy(r)
    B.igabem_server_destroy(srv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_active"] >= 2                 # requests did run concurrently
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    for i, (kind, kw, R) in enumerate(MIX):
        ref = _alone(kind, kw, R)
        # equal up to the solver tolerance (reduction order may differ between runs)
        tol = 1e-7 if kw.get("precision", B.FP64) == B.FP64 else 1e-5
        for rep in range(2):
            u, info, rc = results[rep * len(MIX) + i]
            assert rc == 0 and info["rel_residual"] <= _tol(kw)
            assert G.rel(u, ref) < tol, (i, rep, G.rel(u, ref))


def test_admission_refuses_a_request_larger_than_the_budget():
    srv = B.igabem_server_create(G.ctx(), 8 << 20, 1)          # 8 MiB budget
    opt = B.igabem_default_options(level_m=3, degree_p=2, kappa=2.0, eta_cfie=2.0, leaf_offset=1)
    r = B.igabem_submit(srv, G.geometry("sphere"), opt, [[0.0, 0.0, 1.0]], XH)
    B.igabem_wait(r, 120.0)
    u, info, rc = B.igabem_result(r, raise_errors=False)
    assert rc == -2 and "budget" in B.igabem_last_error()
    B.igabem_request_destroy(r)
    st = B.igabem_server_get_stats(srv)
    assert st["failed"] == 1 and st["completed"] == 0 and st["peak_bytes"] == 0
    B.igabem_server_destroy(srv)


def test_wait_times_out_and_poll_reports_progress():
    srv = B.igabem_server_create(G.ctx(), 0, 1)
    opt = B.igabem_default_options(level_m=4, degree_p=2, kappa=4.0, eta_cfie=4.0, leaf_offset=2)
    r = B.igabem_submit(srv, G.geometry("sphere"), opt, [[0.0, 0.0, 1.0]], XH)
    with pytest.raises(B.IgabemError) as ei:
        B.igabem_wait(r, 0.0)
    assert ei.value.code == -6
    B.igabem_wait(r, 600.0)
    assert B.igabem_poll(r)
    u, info, rc = B.igabem_result(r)
    assert rc == 0 and np.isfinite(u).all() and info["solve_ms"] > 0
    B.igabem_request_destroy(r)
    B.igabem_server_destroy(srv)


def test_requests_for_one_problem_are_merged_and_the_problem_stays_resident():
    """Three requests for the same problem that wait together are solved as one multi-column GMRES
    run (shared matrix-vector products); a later request for it reuses the resident set-up.  Each
    request's far field equals the same request solved alone."""
    srv = B.igabem_server_create(G.ctx(), 0, 1)        # one slot: the requests queue behind the first
    first = B.igabem_submit(srv, G.geometry("deformed"),
                            B.igabem_default_options(level_m=4, degree_p=2, kappa=3.0, eta_cfie=3.0, leaf_offset=2),
                            [[0.0, 0.0, 1.0]], XH)
    kw = dict(level_m=3, degree_p=2, kappa=4.0, eta_cfie=4.0, bc=0, cheb_q=6, leaf_offset=1)
    opt = B.igabem_default_options(tol=1e-8, **kw)
    dirs = inputs.fibonacci_directions(6)
    parts = [dirs[0:1], dirs[1:3], dirs[3:6]]
    reqs = [B.igabem_submit(srv, G.geometry("sphere"), opt, d, XH) for d in parts]
    for r in [first] + reqs:
        B.igabem_wait(r, 600.0)
    late = B.igabem_submit(srv, G.geometry("sphere"), opt, dirs[4:5], XH)
    B.igabem_wait(late, 600.0)
    stats = B.igabem_server_get_stats(srv)
    out = [B.igabem_result(r) for r in reqs + [late]]
    for r in [first] + reqs + [late]:
        B.igabem_request_destroy(r)
    B.igabem_server_destroy(srv)
    assert stats["merged"] >= 2 and stats["cache_hits"] >= 1 and stats["failed"] == 0
    prob, info = G.problem("sphere", tol=1e-8, **kw)
    for d, (u, sinfo, rc) in zip(parts + [dirs[4:5]], out):
        x, _ = B.igabem_solve(prob, d, info["n_dofs"])
        ref = B.igabem_farfield(prob, x, XH)
        assert rc == 0 and G.rel(u, ref) < 1e-7, G.rel(u, ref)
    B.igabem_problem_destroy(prob)
