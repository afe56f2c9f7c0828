"""Session cache of oracle matrices shared by the CPU pin tests and the GPU parity tests."""
import functools

import numpy as np

from oracle import assemble as A
from oracle import fmm
from oracle import space as S
from paper_2306_11324_gb300 import inputs


@functools.lru_cache(maxsize=None)
def sphere_space(m, p, hard=False, deformed=False):
    patches = inputs.deformed_sphere_patches(spans=4) if deformed else inputs.unit_sphere_patches()
    return S.Space(S.Mesh(patches, m), p, continuous=hard)


@functools.lru_cache(maxsize=None)
def operators(m, p, kappa, ops, hard=False, deformed=False):
    sp = sphere_space(m, p, hard, deformed)
    return A.dense_operators(sp, kappa, list(ops))


@functools.lru_cache(maxsize=None)
def tree(m, p, leaf, eta, q, kappa, hard=False, deformed=False):
    sp = sphere_space(m, p, hard, deformed)
    return fmm.ClusterTree(sp.mesh, leaf, eta, q, kappa)


@functools.lru_cache(maxsize=None)
def modeb(m, p, kappa, ops, leaf, eta, q, hard=False, deformed=False):
    sp = sphere_space(m, p, hard, deformed)
    return fmm.modeB_operators(sp, kappa, list(ops), tree(m, p, leaf, eta, q, kappa, hard, deformed))


def cfie(m, p, kappa, eta, hard, mode_b=None, deformed=False):
    """Global CFIE matrix; mode_b = (leaf, eta_adm, q) selects the interpolated-kernel matrix."""
    sp = sphere_space(m, p, hard, deformed)
    names = ("K", "W") if hard else ("Kp", "V")
    ops = dict(operators(m, p, kappa, ("M",), hard, deformed))
    if mode_b is None:
        ops.update(operators(m, p, kappa, names, hard, deformed))
    else:
        ops.update(modeb(m, p, kappa, names, *mode_b, hard=hard, deformed=deformed))
    return A.cfie_matrix(sp, kappa, eta, hard, ops)
