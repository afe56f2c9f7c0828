"""The measured-rate probe behind the roofline fractions (igabem_measure_peaks) returns plausible
rates for one GB300-class GPU, and the default workload's far field agrees with the Mie series."""
import numpy as np
import pytest

from oracle import mie
from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    p = B.igabem_measure_peaks(G.ctx())
    print(p)
    # FP32: lanes x 2 flops x clock, between a tenth of and twice the nominal 152 x 128 x 2 x 2.07 GHz
    nominal32 = p["sm_count"] * 128 * 2 * 2.07e9 / 1e12
    assert 0.1 * nominal32 < p["fp32_tflops"] < 2 * nominal32
    assert 0.0 < p["fp64_tflops"] < p["fp32_tflops"]
    assert 0.0 < p["sincosf_gops"] and 0.0 < p["rsqrtf_gops"] and 0.0 < p["sincos_fp64_gops"]
    # a special-function call is slower than an FMA
    assert p["sincosf_gops"] * 1e9 < p["fp32_tflops"] * 1e12 / 2


def test_default_workload_far_field_matches_mie():
    """Unit sphere, 32 x 32 elements per patch, degree 2, kappa = 8, mixed precision with the block
    preconditioner: the GMRES solution's far field against the Mie series (the discretisation, FMM
    and solver errors together)."""
    prob, info = G.problem("sphere", level_m=5, degree_p=2, kappa=8.0, eta_cfie=8.0, bc=0, cheb_q=7,
                           leaf_offset=2, eta_adm=0.5, precision=B.MIXED_FP32, precond=1, tol=1e-6)
    d = np.array([[0.0, 0.0, 1.0]])
    x, sinfo = B.igabem_solve(prob, d, info["n_dofs"])
    xh = inputs.fibonacci_directions(100)
    u = B.igabem_farfield(prob, x, xh)[:, 0]
    err = G.rel(u, mie.mie_far_field(8.0, xh))
    print(f"far field vs Mie: {err:.2e} after {sinfo['iterations']} iterations")
    assert sinfo["rel_residual"] <= 1e-6
    assert err < 1e-4
    B.igabem_problem_destroy(prob)
