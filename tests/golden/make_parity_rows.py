"""Writes the oracle's sampled rows of the mode-B CFIE product for the large GPU parity tests.

Only the oracle (``oracle/``) and the seeded input generator are used: the expected values are the
interpolated-kernel ("mode B") Galerkin matrix of Sec. 4.4 applied to a seeded vector, entry by entry
(``oracle.fmm.cfie_rows``), for the discretisations the benchmark runs -- degree 2 B-splines,
7 x 7 Chebyshev points per cluster, leaves of 4 x 4 elements, admissibility eta_adm = 0.5 -- which the
oracle needs minutes for, so they are stored instead of recomputed in every GPU run.

    python tests/golden/make_parity_rows.py [case ...]

Each case writes ``rows_<case>.txt``: a header of ``# key = value`` lines (the case's parameters) and
then one line per entry ``row column re im``.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fmm  # noqa: E402
from oracle import space as S  # noqa: E402
from paper_2306_11324_gb300 import inputs  # noqa: E402

# name -> parameters; leaf = leaf level of the cluster tree (m - b), eta = CFIE coupling (Sec. 2),
# cap = kappa * cluster diameter bound of the admissibility (inf: none), cols = columns of the seeded x
CASES = {
    # unit sphere, 16 x 16 elements per patch, the benchmark's discretisation at kappa = 8
    "sphere_soft_m4_p2_q7_b2_k8": dict(geometry="sphere", m=4, p=2, leaf=2, q=7, kappa=8.0, eta=8.0,
                                       hard=False, cap=np.inf, cols=16, seed=2101, nrows=8),
    # the default benchmark workload itself: unit sphere, 32 x 32 elements per patch, kappa = 8
    "sphere_soft_6x32x32_p2_k8": dict(geometry="sphere", m=5, p=2, leaf=3, q=7, kappa=8.0, eta=8.0,
                                      hard=False, cap=np.inf, cols=1, seed=2026, nrows=6),
    # deformed (multi-span) sphere, continuous space, hypersingular operator, capped admissibility
    "deformed_hard_m4_p2_q7_b2_k8_cap6": dict(geometry="deformed", m=4, p=2, leaf=2, q=7, kappa=8.0,
                                              eta=0.125, hard=True, cap=6.0, cols=16, seed=2102, nrows=6),
    # the 64-direction sound-hard workload: deformed sphere, 64 x 64 elements per patch, kappa = 20
    "deformed_hard_6x64x64_p2_k20": dict(geometry="deformed", m=6, p=2, leaf=4, q=7, kappa=20.0, eta=0.05,
                                         hard=True, cap=6.0, cols=64, seed=2027, nrows=2),
    # the large scatterer's discretisation at 16 x 16 elements per patch: deformed multi-span sphere,
    # sound-soft, kappa = 20, level-adaptive q (7 .. 12 under the kappa * diameter <= 6 cap)
    "deformed_soft_m4_p2_q7-12_b2_k20_cap6": dict(geometry="deformed", m=4, p=2, leaf=2, q=7, q_max=12,
                                                  kappa=20.0, eta=20.0, hard=False, cap=6.0, cols=8,
                                                  seed=2103, nrows=6),
    # the large single scatterer at the sweep's first kappa: deformed sphere, 256 x 256 elements per
    # patch (399384 unknowns), kappa = 50, 8 columns, level-adaptive q (7 .. 12, capped admissibility).
    # Not stored: two rows take the oracle more than four hours on one core (every far cluster's mode-B
    # block of the row's element is formed); run it explicitly to produce the file
    "deformed_soft_6x256x256_p2_k50": dict(geometry="deformed", m=8, p=2, leaf=6, q=7, q_max=12, kappa=50.0,
                                           eta=50.0, hard=False, cap=6.0, cols=8, seed=2029, nrows=2),
}


def patches(kind):
    return inputs.unit_sphere_patches() if kind == "sphere" else inputs.deformed_sphere_patches(spans=4)


def rows_of(c, N):
    """Sampled rows: the first and last unknowns (patch corners) and evenly spread ones between."""
    return np.unique(np.linspace(0, N - 1, c["nrows"]).round().astype(int))


def make(name):
    c = CASES[name]
    t0 = time.time()
    sp = S.Space(S.Mesh(patches(c["geometry"]), c["m"]), c["p"], continuous=c["hard"])
    tree = fmm.ClusterTree(sp.mesh, c["leaf"], 0.5, c["q"], c["kappa"], kappa_cap=c["cap"], q_max=c.get("q_max"))
    x = inputs.random_complex(sp.N, seed=c["seed"], cols=c["cols"])
    rows = rows_of(c, sp.N)
    y = fmm.cfie_rows(sp, c["kappa"], c["eta"], c["hard"], x, rows, tree)
    path = os.path.join(HERE, f"rows_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# sampled rows of the mode-B CFIE product (Sec. 4.4), written by make_parity_rows.py\n")
        for k, v in c.items():
            f.write(f"# {k} = {v}\n")
        f.write(f"# N = {sp.N}\n# n_far_pairs = {sum(len(l) for l in tree.far)}\n")
        for i, r in enumerate(rows):
            for j in range(c["cols"]):
                f.write(f"{r} {j} {float(y[i, j].real)!r} {float(y[i, j].imag)!r}\n")
    print(f"{name}: N = {sp.N}, {len(rows)} rows x {c['cols']} columns, {time.time() - t0:.0f} s -> {path}")


def load(name):
    """(parameters, rows, values[rows, cols], N, n_far_pairs) of a stored case."""
    c = dict(CASES[name])
    path = os.path.join(HERE, f"rows_{name}.txt")
    meta, data = {}, []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                if " = " in line:
                    k, v = line[1:].split(" = ", 1)
                    meta[k.strip()] = v.strip()
            elif line.strip():
                r, j, re, im = line.split()
                data.append((int(r), int(j), float(re), float(im)))
    rows = sorted({d[0] for d in data})
    y = np.zeros((len(rows), c["cols"]), dtype=complex)
    for r, j, re, im in data:
        y[rows.index(r), j] = complex(re, im)
    return c, np.array(rows), y, int(meta["N"]), int(meta["n_far_pairs"])


if __name__ == "__main__":
    for name in sys.argv[1:] or [c for c in CASES if c != "deformed_soft_6x256x256_p2_k50"]:
        make(name)
