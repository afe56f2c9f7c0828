"""The allocation-free far field (igabem_farfield_noalloc) against the regular entry point.

Callers that cannot let the library allocate device memory (their own allocator owns the device, or
they must not stall on cudaMalloc's implicit synchronisation) use igabem_farfield_noalloc, which
keeps its scratch in a fixed device array.  This file is collected last so that a failure here
stops a -x run only after every other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = 1e-10     # the FP64 tolerance of the other GPU parity tests


@pytest.mark.parametrize("hard", [False, True])
def test_noalloc_far_field_matches_far_field_on_two_calls(hard):
    import torch
    prob, info = G.problem(level_m=2, degree_p=1, kappa=2.0, eta_cfie=2.0, bc=int(hard), no_fmm=1)
    N = info["n_dofs"]
    for call, (R, n_dir, seed) in enumerate([(2, 37, 11), (3, 64, 12)]):
        dens = torch.tensor(inputs.random_complex(N, seed=seed, cols=R), device="cuda")
        xh = inputs.fibonacci_directions(n_dir)
        ref = B.igabem_farfield(prob, dens, xh)                 # the allocating entry point
        xh_dev = torch.tensor(xh, dtype=torch.float64, device="cuda")
        out = torch.full((n_dir, R), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        B.igabem_farfield_noalloc(prob, dens, xh_dev, out)
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert G.rel(got, want) < TOL, call
    B.igabem_problem_destroy(prob)


def test_noalloc_far_field_refuses_what_it_cannot_hold():
    import torch
    prob, info = G.problem(level_m=2, degree_p=1, kappa=1.0, eta_cfie=1.0, no_fmm=1)
    N = info["n_dofs"]
    # 96 elements x 16 Gauss points x 1400 columns > 2^21 scratch values
    dens = torch.zeros((N, 1400), dtype=torch.complex128, device="cuda")
    xh = torch.tensor(inputs.fibonacci_directions(4), dtype=torch.float64, device="cuda")
    out = torch.empty((4, 1400), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.IgabemError) as ei:
        B.igabem_farfield_noalloc(prob, dens, xh, out)
    assert ei.value.code == -1 and "scratch" in str(ei.value)
    # host memory is refused: the entry point never stages copies
    with pytest.raises(B.IgabemError) as ei:
        B.igabem_farfield_noalloc(prob, dens[:, :1].contiguous().cpu().numpy(), xh, out[:, :1].contiguous())
    assert ei.value.code == -1 and "device memory" in str(ei.value)
    # so is page-locked host memory, which kernels could reach but which is not the device's own
    pinned = torch.zeros((N, 1), dtype=torch.complex128).pin_memory()
    with pytest.raises(B.IgabemError) as ei:
        B.igabem_farfield_noalloc(prob, pinned, xh, out[:, :1].contiguous())
    assert ei.value.code == -1 and "device memory" in str(ei.value)
    # more right-hand sides than the kernel's grid can hold: refused before any launch
    wide = torch.zeros((N, 65536), dtype=torch.complex128, device="cuda")
    out_w = torch.empty((1, 65536), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.IgabemError) as ei:
        B.igabem_farfield_noalloc(prob, wide, xh[:1].contiguous(), out_w)
    assert ei.value.code == -1 and "65535" in str(ei.value)
    del wide, out_w
    # the context is still usable after the refusals
    good = torch.tensor(inputs.random_complex(N, seed=5, cols=1), device="cuda")
    o1 = torch.empty((4, 1), dtype=torch.complex128, device="cuda")
    B.igabem_farfield_noalloc(prob, good, xh, o1)
    assert G.rel(o1.cpu().numpy(), B.igabem_farfield(prob, good, xh.cpu().numpy()).cpu().numpy()) < TOL
    B.igabem_problem_destroy(prob)
