"""Host-side pieces of bench.py: the oracle sampler of the CPU baseline and of the reference arm (a
pool of spawned processes that build the mesh once and time bounded samples of element rows), and the
serving stream's request recipe."""
import numpy as np

import bench


def test_oracle_sampler_times_repeated_bounded_samples():
    wl = dict(geometry="sphere", level_m=2, degree_p=1, kappa=1.0, bc=0)
    with bench.OracleSampler(wl) as smp:
        smp.cores = min(smp.cores, 2)
        a = smp.sample(budget_s=0.5, with_lu=False)
        b = smp.sample(budget_s=0.5, with_lu=True)
    for cb in (a, b):
        assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
        assert np.isclose(cb["value"] * cb["extrapolated_s_per_solve"], 1.0)
    assert "dense LU" in b["sample"]


def test_serving_requests_keep_eight_unknowns_per_wavelength():
    for r in bench.serving_requests(64, seed=5):
        assert 4 <= r["m"] <= 6 and 1.0 <= r["kappa"] <= (2 ** r["m"] + 2) / 2
        assert 1 <= len(r["dirs"]) <= 32 and np.allclose(np.linalg.norm(r["dirs"], axis=1), 1.0)
        assert r["bc"] in (0, 1) and r["gap"] >= 0
