"""Parity at the discretisations the benchmark runs: degree-2 B-splines, 7 x 7 Chebyshev points per
cluster, leaves of 4 x 4 elements, admissibility eta_adm = 0.5 (Sec. 4.4), including the default
workload (unit sphere, 32 x 32 elements per patch, kappa = 8) and the 64-direction sound-hard workload
(deformed multi-span sphere, 64 x 64 elements per patch, kappa = 20).

The CUDA path runs through the C ABI; the expected values are sampled rows of the oracle's mode-B
product on the same seeded vectors, stored in tests/golden/rows_*.txt by make_parity_rows.py (which
imports only oracle/ and the input generator).  Every stored entry is compared."""
import numpy as np
import pytest

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G
from tests.golden import make_parity_rows as golden

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-6, "tc": 1e-5}   # as in test_gpu_parity.py


def _prec(name):
    return {"fp64": B.FP64, "mixed": B.MIXED_FP32, "tc": B.MIXED_TC}[name]


def _problem(c, prec, stored=0):
    return G.problem(c["geometry"], level_m=c["m"], degree_p=c["p"], kappa=c["kappa"], eta_cfie=c["eta"],
                     bc=int(c["hard"]), cheb_q=c["q"], leaf_offset=c["m"] - c["leaf"], eta_adm=0.5,
                     kappa_cap=0.0 if not np.isfinite(c["cap"]) else c["cap"], precision=_prec(prec),
                     m2l_stored=stored, q_max=c.get("q_max") or 0)


def _check(name, prec, single_column=True, stored=0):
    c, rows, ref, N, n_far = golden.load(name)
    prob, info = _problem(c, prec, stored)
    assert info["n_dofs"] == N and info["n_far_pairs"] == n_far
    x = inputs.random_complex(N, seed=c["seed"], cols=c["cols"])
    y = B.igabem_matvec(prob, x if c["cols"] > 1 else x[:, 0])
    y = y.reshape(N, -1)
    err = np.abs(y[rows] - ref).max() / np.abs(ref).max()
    print(f"{name} {prec}: {c['cols']} columns, rel. error {err:.2e}")
    assert err < TOL[prec]
    if single_column and c["cols"] > 1:         # the one-column path (R = 1 M2L, SpMV, P2M / L2P)
        y1 = B.igabem_matvec(prob, np.ascontiguousarray(x[:, 0]))
        err1 = np.abs(y1[rows] - ref[:, 0]).max() / np.abs(ref[:, 0]).max()
        print(f"{name} {prec}: one column, rel. error {err1:.2e}")
        assert err1 < TOL[prec if prec != "tc" else "mixed"]
    B.igabem_problem_destroy(prob)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "tc"])
def test_sphere_16x16_p2_q7_leaves4x4(prec):
    _check("sphere_soft_m4_p2_q7_b2_k8", prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "tc"])
def test_deformed_multispan_sound_hard_p2_q7_capped(prec):
    """Sound-hard on S^0 over the deformed sphere, whose degree-4 patches have 4 knot spans per
    direction (multi-span Bezier extraction), with the hypersingular operator and a kappa cap."""
    _check("deformed_hard_m4_p2_q7_b2_k8_cap6", prec)


@pytest.mark.parametrize("prec,stored", [("fp64", 0), ("mixed", 0), ("fp64", 1), ("mixed", 1)])
def test_6x32x32_workload_matvec_against_oracle_rows(prec, stored):
    """The 32 x 32-element workload's operator (6936 unknowns, kappa = 8) on a seeded vector: the plain
    FP64 GPU matvec and the mixed-precision one, with the coupling blocks generated on the fly and
    stored, against the oracle's rows."""
    _check("sphere_soft_6x32x32_p2_k8", prec, stored=stored)


@pytest.mark.parametrize("prec", ["tc", "mixed"])
def test_64_direction_sound_hard_workload_against_oracle_rows(prec):
    """The 64-direction sound-hard workload's operator (25352 unknowns, kappa = 20, 64 columns) in the
    tensor-core and FP32 M2L precisions against the oracle's rows."""
    _check("deformed_hard_6x64x64_p2_k20", prec, single_column=False)


@pytest.mark.parametrize("prec,stored", [("fp64", 0), ("mixed", 1)])
def test_large_scatterer_discretisation_at_16x16_against_oracle_rows(prec, stored):
    """The large scatterer's discretisation at 16 x 16 elements per patch: deformed multi-span sphere,
    sound-soft, kappa = 20, level-adaptive q (7 .. 12 under the kappa * diameter <= 6 cap, band-bottom
    levels), 8 columns; FP64 with the blocks generated on the fly, and the benchmark's mixed precision
    with stored FP32 blocks."""
    _check("deformed_soft_m4_p2_q7-12_b2_k20_cap6", prec, single_column=False, stored=stored)
