"""Helpers of the GPU tests: one CUDA context per session, problems built through the C ABI."""
import functools

import numpy as np

from paper_2306_11324_gb300 import binding as B
from paper_2306_11324_gb300 import inputs


@functools.lru_cache(maxsize=None)
def ctx():
    return B.igabem_create(0, None)


@functools.lru_cache(maxsize=None)
def geometry(kind="sphere"):
    if kind == "sphere":
        patches = inputs.unit_sphere_patches()
    elif kind == "deformed":
        patches = inputs.deformed_sphere_patches(spans=4)
    elif kind == "deformed8":
        patches = inputs.deformed_sphere_patches(spans=8)
    else:
        raise ValueError(kind)
    return B.igabem_geometry_create(ctx(), patches)


def problem(kind="sphere", **kw):
    opt = B.igabem_default_options(**kw)
    prob = B.igabem_problem_create(geometry(kind), opt)
    return prob, B.igabem_problem_info(prob)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()
