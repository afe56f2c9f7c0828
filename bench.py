#!/usr/bin/env python
"""Benchmark of the isogeometric CFIE solver on one GB300 (or N replicas of it under torchrun).

Default workload, the large single scatterer: seeded deformed sphere (6 degree-4 patches with 4 knot
spans per direction, control points displaced radially with amplitude 0.15), 256 x 256 elements per
patch (393216 elements), B-splines of degree 2 (399384 unknowns), sound-soft, eta = kappa, a frequency
sweep of 16 kappa in [50, 60] with 8 incident directions each and the far field at 2048 directions.
A step is one kappa of the sweep through the whole hot path: problem set-up (geometry tables, cluster
tree with level-adaptive Chebyshev orders 7 .. 12, stored FP32 coupling blocks, near-field Galerkin
quadrature), right-hand sides, GMRES(30) with the block preconditioner to 1e-5 for the 8 directions at
once, far field; solves/s counts every direction.  Timed in the mixed precision; the product is
compared with the plain FP64 operator's on a seeded vector beside the steps.

--workload sphere_soft_6x32x32_p2_k8: sound-soft unit sphere, 32 x 32 elements per patch (6936
unknowns), kappa = 8, one plane wave; a step is one request (set-up, GMRES(30) to 1e-6, far field at 100
directions), the FP64 form timed beside it and the far fields of the two compared.
--workload deformed_hard_6x64x64_p2_k20_64dirs: sound-hard deformed sphere, 24576 elements, kappa = 20,
64 incident directions; a step is one operator application to the 64 columns (tensor-core M2L by
default), one full solve timed beside the steps, the product checked against the FP64 operator.
--workload serving_stream: Poisson arrivals of mixed requests into the library's server.
--workload torus_convergence: observed convergence orders on the exact torus.

Prints one JSON line (see the keys below).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CFIE matvecs/s & solves/s at far-field err≤1e-5 vs FP64; p50/p99 solve latency"

WORKLOADS = {
    # leaf offset b (leaves of 2^b x 2^b elements) per precision: the faster set-up + solve on GB300;
    # the mixed form's GMRES stops at its FP32 rounding floor
    "sphere_soft_6x32x32_p2_k8": dict(geometry="sphere", level_m=5, degree_p=2, kappa=8.0, bc=0,
                                      cheb_q=7, eta_adm=0.5, leaf_offset={"fp64": 2, "mixed": 2},
                                      tol={"fp64": 1e-6, "mixed": 1e-6}, n_dir=100, n_rhs=1, kappa_cap=0.0,
                                      restart=30, precond={"fp64": 1, "mixed": 1}, precision="mixed", eta=8.0),
    # sound-hard deformed sphere (amplitude 0.15, seed 1), 64 x 64 elements per patch, kappa = 20,
    # 64 incident directions on a Fibonacci sphere solved as one multi-RHS request; admissibility capped
    # at kappa * diameter <= 6 (FMM truncation ~1e-5 against the dense matrix at q = 7)
    # GMRES(30) stagnates on this sound-hard system (the hypersingular part is unbounded and kappa is
    # large): restart 300, eta = 1/kappa and the block preconditioner (~300 iterations to 1e-5 at 16
    # directions, against ~860 unpreconditioned).
    # A step of this workload is one operator application to all 64 columns; one solve (capped at 1500
    # iterations) is timed beside the steps.
    "deformed_hard_6x64x64_p2_k20_64dirs": dict(geometry="deformed", level_m=6, degree_p=2, kappa=20.0, bc=1,
                                                cheb_q=7, eta_adm=0.5, leaf_offset={"fp64": 2, "mixed": 2, "tc": 2},
                                                tol={"fp64": 1e-5, "mixed": 1e-5, "tc": 1e-5}, n_dir=100, n_rhs=64,
                                                kappa_cap=6.0, restart=300, precond={"fp64": 1, "mixed": 1, "tc": 1},
                                                precision="tc", step="matvec", solve_max_iter=1500, eta=0.05),
    # the large single scatterer: deformed sphere (amplitude 0.15, seed 1), 256 x 256 elements per patch
    # (393216 elements, 399384 unknowns), sound-soft, a frequency sweep of 16 kappa in [50, 60] with 8
    # incident directions each, far field at 2048 directions.  A step is one kappa of the sweep: problem
    # set-up (near field, tree, tables), GMRES(30) with the block preconditioner to 1e-5 for the 8
    # directions at once, far field.  Level-adaptive interpolation: 7 points per direction where
    # kappa * diameter <= 6, up to 12 on coarser levels (the Chebyshev bound of the finest level's accuracy).
    "deformed_soft_6x256x256_p2_k50-60_8dirs": dict(geometry="deformed", level_m=8, degree_p=2, kappa=50.0, bc=0,
                                                    cheb_q=7, q_max=12, eta_adm=0.5, kappa_cap=6.0,
                                                    leaf_offset={"fp64": 2, "mixed": 2, "tc": 2},
                                                    tol={"fp64": 1e-5, "mixed": 1e-5, "tc": 1e-5}, n_dir=2048,
                                                    n_rhs=8, restart=30, precond={"fp64": 1, "mixed": 1, "tc": 1},
                                                    precision="mixed", step="sweep", eta="kappa",
                                                    m2l_stored={"fp64": 0, "mixed": 1, "tc": 1},
                                                    kappas=[50.0 + 10.0 * i / 15 for i in range(16)],
                                                    solve_max_iter=2000),
    # the same step at 32 x 32 elements per patch (6144 elements), kappa in [10, 12]: a small case of the
    # large scatterer's kernels (profiling, quick checks)
    "deformed_soft_6x32x32_p2_k10-12_8dirs": dict(geometry="deformed", level_m=5, degree_p=2, kappa=10.0, bc=0,
                                                  cheb_q=7, q_max=12, eta_adm=0.5, kappa_cap=6.0,
                                                  leaf_offset={"fp64": 2, "mixed": 2, "tc": 2},
                                                  tol={"fp64": 1e-5, "mixed": 1e-5, "tc": 1e-5}, n_dir=2048,
                                                  n_rhs=8, restart=30, precond={"fp64": 1, "mixed": 1, "tc": 1},
                                                  precision="mixed", step="sweep", eta="kappa",
                                                  m2l_stored={"fp64": 0, "mixed": 1, "tc": 1},
                                                  kappas=[10.0 + 2.0 * i / 15 for i in range(16)],
                                                  solve_max_iter=2000),
}
DEFAULT = "deformed_soft_6x256x256_p2_k50-60_8dirs"
PRECISIONS = {}                              # name -> igabem_precision (filled once the binding is loaded)
FLOPS_PER_SAMPLE = {False: 40, True: 52}     # FP32 M2L kernel-sample arithmetic: soft 40 flops, hard 52 per pair of samples
FLOPS_PER_MAC = 8                            # one complex multiply-add
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_near_singular launch per 4-D point,
# from one ncu capture of the small sweep case (29.6 + 22.7 MB for 92,130,000 points); the traffic of a
# launch grows with its points (block writes per pair, rule and net reads per chunk)
SINGULAR_DRAM_BYTES_PER_POINT = 52.274424e6 / 92130000


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"])
    return 6800.0


def singular_flops(info, p, hard, pg=4):
    """FP64 operations of the touching pairs' quadrature (the model behind the roofline of
    k_near_singular), from the counts the library reports.  Per element net contracted along its second
    coordinate (once per distinct value in a chunk of the rule): the homogeneous rows of the rational
    Bezier net of degree pg with their derivatives, 2 (pg+1)^2 4 2 flops.  Per distinct element point:
    the columns with value, d/du, d/dv ((pg+1) 4 3 2), the rational quotient, normal and Jacobian (30).
    Per 4-D point: the kernel (distance, sincos, G, G'/r, the two orientations and the weight, 60), the
    (p+1)^2 B-splines of the side that is not grouped by Bernstein extraction (5 per function; the surface
    curls 6 more for sound-hard) and the group sums (the kernel value of each orientation times each
    function, 8 per function; sound-hard adds w gc times the curls, 12).  Per group of points sharing an
    element point: that side's B-splines (and curls) and the accumulation of the (p+1)^2 x (p+1)^2 entries
    of both blocks (8 per entry; sound-hard 16 more for the curl products).  Identical sound-soft pairs
    summed in factorised form (groups of ns^2 points, ns = 5): per point the kernel alone; per group the
    univariate basis values (4 ns of them, 5 (p+1) each), the inner sums (ns (p+1)^2 ns, 10 flops each:
    the product of two basis values and two complex-by-real multiply-adds) and the outer sums
    ((p+1)^4 ns, 10 each)."""
    n = (p + 1) ** 2
    ns = 5
    per_column = 2 * (pg + 1) ** 2 * 4 * 2
    per_geo_point = (pg + 1) * 4 * 3 * 2 + 30
    basis = 5 * n + (6 * n if hard else 0)
    per_point = 60 + basis + 8 * n + (12 * n if hard else 0)
    per_group = basis + n * n * (8 + (16 if hard else 0))
    fact = info.get("n_singular_factored_points", 0)
    per_fact_group = 4 * ns * 5 * (p + 1) + ns * n * ns * 10 + n * n * ns * 10
    return (info["n_singular_geo_columns"] * per_column + info["n_singular_geo_points"] * per_geo_point
            + (info["n_singular_points"] - fact) * per_point + fact * 60
            + info["n_singular_groups"] * per_group + fact / ns ** 2 * per_fact_group)


def mie_soft_far_field(kappa, xhat, d=(0.0, 0.0, 1.0)):
    """Far field of a plane wave scattered by the sound-soft unit sphere (the Mie series, a textbook
    closed form; e^{-i omega t}, outgoing Hankel functions): u_inf = (i/kappa) sum_n (2n+1)
    j_n(kappa)/h_n(kappa) P_n(x^.d), summed to n = kappa + 4 kappa^(1/3) + 20."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn
    c = np.clip(np.asarray(xhat, float) @ np.asarray(d, float), -1.0, 1.0)
    out = np.zeros(c.shape, dtype=complex)
    for n in range(int(kappa + 4 * kappa ** (1 / 3) + 20) + 1):
        j = spherical_jn(n, kappa)
        out += (2 * n + 1) * (j / (j + 1j * spherical_yn(n, kappa))) * eval_legendre(n, c)
    return 1j / kappa * out


def m2l_alu_roofline(kernel, far_pairs, Q, hard, R, ms, peaks, fp64):
    """Roofline of an M2L of kernel samples generated on the fly (R columns per sample pass): FP flops
    (sample arithmetic + complex contraction) against the measured FMA rate, and the special-function
    work (one sincos and one rsqrt per node pair) against the measured XU rates; the bound is the
    larger of the two fractions."""
    C = 7 if hard else 1
    samples = far_pairs * Q * Q
    flops = samples * (FLOPS_PER_SAMPLE[hard] * (2 if hard else 1) + FLOPS_PER_MAC * C * R)
    achieved = flops / (ms / 1e3) / 1e12
    fpk = "fp64_tflops" if fp64 else "fp32_tflops"
    out = {"kernel": kernel, "achieved": achieved, "unit": "TFLOP/s", "peak": peaks[fpk],
           "frac": achieved / peaks[fpk], "algorithmic_flops_per_matvec": flops, "avg_ms_per_matvec": ms,
           "peak_source": f"measured {'FP64' if fp64 else 'FP32'} FMA rate (igabem_measure_peaks, this run)",
           "node_pairs_per_matvec": samples}
    if fp64:
        t_sfu = samples / (peaks["sincos_fp64_gops"] * 1e9)
        out["sincos_fp64_frac"] = t_sfu / (ms / 1e3)
        out["bound"] = "alu"
    else:
        t_xu = samples / (peaks["sincosf_gops"] * 1e9) + samples / (peaks["rsqrtf_gops"] * 1e9)
        out["xu_frac"] = t_xu / (ms / 1e3)
        out["xu_source"] = "one __sincosf and one rsqrtf per node pair at the measured rates"
        out["bound"] = "alu" if out["frac"] >= out["xu_frac"] else "xu"
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + ["serving_stream", "torus_convergence"])
    ap.add_argument("--requests", type=int, default=64, help="serving_stream: requests in the stream")
    ap.add_argument("--rate", type=float, default=2.0, help="serving_stream: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving_stream: concurrent requests")
    ap.add_argument("--max-iter", type=int, default=1000, help="serving_stream: GMRES iterations per request")
    ap.add_argument("--precision", choices=["fp64", "mixed", "tc"], default=None,
                    help="fp64, mixed (FP32 far field) or tc (mixed with the tensor-core M2L); default: the "
                         "workload's own")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--one-form", action="store_true", help="time only --precision (no second form)")
    return ap.parse_args()


def patches_of(kind):
    from paper_2306_11324_gb300 import inputs
    return inputs.unit_sphere_patches() if kind == "sphere" else inputs.deformed_sphere_patches(spans=4)


# ---------------------------------------------------------------------------------------------
# clocks during the timed region

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(", ") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# the oracle on the host cores (bounded sample)

_ORACLE_STATE = None


def _oracle_init(wl, n_trial):
    """Per host process of the oracle sample, once: the mesh, space and element rules of the workload
    and the trial elements each test row is integrated against."""
    global _ORACLE_STATE
    from oracle import assemble as A
    from oracle import space as S
    mesh = S.Mesh(patches_of(wl["geometry"]), wl["level_m"])
    sp = S.Space(mesh, wl["degree_p"], continuous=bool(wl["bc"]))
    rules = A.ElementRules(sp)
    touch = {}
    for e, f, k in mesh.touching():
        touch.setdefault(e, []).append((f, k))
    trial = np.arange(mesh.E) if n_trial >= mesh.E else np.arange(0, mesh.E, mesh.E // n_trial)
    _ORACLE_STATE = (wl, mesh, sp, rules, touch, trial)


def _oracle_rows_worker(job):
    """One host process of the oracle sample: the exact Galerkin rows of the test elements job[0]
    (against the trial elements), until job[1] seconds have passed; returns (rows done, seconds scaled
    to rows against all elements)."""
    from oracle import assemble as A
    elems, budget = job
    wl, mesh, sp, rules, touch, trial = _ORACLE_STATE
    ops = ["K", "W"] if wl["bc"] else ["Kp", "V"]
    t0 = time.perf_counter()
    k = 0
    for e in elems:
        pairs = [(e, e, 0)] + [(e, f, kk) for f, kk in touch.get(e, [])]
        A.singular_blocks(ops, wl["kappa"], sp, pairs)
        reg = np.setdiff1d(trial, [f for _, f, _ in pairs])
        for op in ops:
            A.regular_row_blocks(op, wl["kappa"], rules, e, reg)
        k += 1
        if time.perf_counter() - t0 > budget:
            break
    return k, (time.perf_counter() - t0) * mesh.E / len(trial)


class OracleSampler:
    """The CPU oracle timed on a bounded sample of the workload on the host cores, scaled to solves/s.

    Sample: the exact Galerkin rows of some test elements against the trial elements (dense FP64
    assembly, regular and singular quadrature), computed by one spawned process per host core (each
    process builds the mesh, space and rules once, when the sampler opens, outside every timed
    region), the rows per second of all processes together scaled to the E rows of the full matrix;
    plus the dense LU of an n x n complex matrix (n = 1536) on the BLAS threads, scaled by (N/n)^3 to
    the N x N system."""

    def __init__(self, wl):
        self.wl = wl
        self.E = 6 * 4 ** wl["level_m"]
        self.N = 6 * (2 ** wl["level_m"] + wl["degree_p"]) ** 2
        # one process per host core, as many as half the host memory holds: each process keeps the
        # oracle's mesh, space and Gauss-point tables of all E elements (~12.5 kB per element measured,
        # 4.9 GB on 393216 elements)
        cores = os.cpu_count() or 1
        try:
            mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        except (ValueError, OSError, AttributeError):
            mem = 64 << 30
        per_proc = 12.5e3 * self.E + 0.5e9
        self.cores = max(1, min(cores, int(0.5 * mem / per_proc)))
        self.n_trial = min(self.E, 6144)   # rows against at most 6144 trial elements, scaled to all E
        self.calls = 0

    def __enter__(self):
        import multiprocessing
        self.env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")   # one thread per process
        self.pool = multiprocessing.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                              initargs=(self.wl, self.n_trial))
        return self

    def __exit__(self, *exc):
        self.pool.close()
        self.pool.join()
        for k, v in self.env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def sample(self, budget_s=20.0, with_lu=True):
        import scipy.linalg
        cores, E, N = self.cores, self.E, self.N
        off = 13 * self.calls
        self.calls += 1
        jobs = [(list(range(off + 97 * w, E, 97 * cores)), budget_s * 0.5) for w in range(cores)]
        res = self.pool.map(_oracle_rows_worker, jobs, chunksize=1)
        rows = sum(k for k, _ in res)
        rate = sum(k / t for k, t in res if t > 0)          # rows per second of all processes together
        t_rows = 1.0 / rate
        n = 1536
        t_lu = 0.0
        if with_lu:
            M = (np.random.default_rng(0).standard_normal((n, n))
                 + 1j * np.random.default_rng(1).standard_normal((n, n)))
            t1 = time.perf_counter()
            scipy.linalg.lu_factor(M)
            t_lu = (time.perf_counter() - t1) * (N / n) ** 3
        t_solve = t_rows * E + t_lu
        return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"{rows} of {E} element rows of the exact Galerkin matrix on {cores} processes "
                          f"(each row against {self.n_trial} of the {E} trial elements, its time scaled by "
                          f"{E / self.n_trial:.0f}; {rate:.3f} full rows/s together, scaled by E) + dense LU "
                          f"of a {n}^2 complex matrix scaled by (N/{n})^3 = {t_lu:.1f} s on the BLAS threads",
                "extrapolated_s_per_solve": t_solve}


def oracle_sample(wl, budget_s=20.0, with_lu=True):
    """One bounded sample of the oracle (OracleSampler) for the workload."""
    with OracleSampler(wl) as smp:
        return smp.sample(budget_s, with_lu)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    times = []
    with OracleSampler(wl) as smp:
        for i in range(args.warmup + args.steps):
            cb = smp.sample(budget_s=6.0)
            if i >= args.warmup:
                times.append(cb["extrapolated_s_per_solve"])
    # a direct solve serves all of a step's incident directions at once: each counts as a solve, as in
    # the GPU arm
    R = wl.get("n_rhs", 1)
    value = R / statistics.mean(times)
    cb["value"] = value
    if R > 1:
        cb["sample"] += f"; {R} directions per solve counted as {R} solves"
    print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": {"workload": args.workload},
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------------------------

def replica_share(items, rank, world):
    """The units of work of one rank: replicas deal whole requests round-robin (no data-path exchange)."""
    return items[rank::world]


def max_over_ranks(value, dist, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def serving_requests(n, seed=0):
    """The serving stream: n requests, each a seeded deformed sphere with 16x16 .. 64x64 elements per
    patch, kappa ~ U[1, 30] rejected until there are >= 8 degree-2 unknowns per wavelength
    ((2^m + 2) / 2 >= kappa along a patch edge of arc pi/2), random boundary condition, 1..32
    incident directions; exponential inter-arrival gaps of mean 1 (scaled by the arrival rate)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        m = int(rng.integers(4, 7))
        while True:
            kappa = float(rng.uniform(1.0, 30.0))
            if kappa <= (2 ** m + 2) / 2:
                break
        dirs = rng.standard_normal((int(rng.integers(1, 33)), 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        out.append(dict(m=m, kappa=kappa, bc=int(rng.integers(0, 2)), dirs=dirs, geom_seed=int(rng.integers(1, 10**6)),
                        gap=float(rng.exponential(1.0))))
    return out


def _report_done(B, reqs, handles, reported, t0):
    """Progress of the serving stream on stderr: one line per finished request."""
    for i, h in enumerate(handles):
        if i not in reported and B.igabem_poll(h):
            reported.add(i)
            _, info, rc = B.igabem_result(h, raise_errors=False)
            r = reqs[i]
            print(f"[{time.perf_counter() - t0:8.1f} s] request {i}: m={r['m']} kappa={r['kappa']:.1f} "
                  f"bc={r['bc']} R={len(r['dirs'])} rc={rc} its={info['iterations']} "
                  f"solve {info['solve_ms']:.0f} ms", file=sys.stderr, flush=True)


def run_serving(args):
    """Continuous-batching serving run: Poisson arrivals into the library's server."""
    import torch
    from paper_2306_11324_gb300 import binding as B
    from paper_2306_11324_gb300 import inputs
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    reqs = replica_share(serving_requests(args.requests), rank, world)
    ctx = B.igabem_create(local, None)
    xhat = inputs.fibonacci_directions(100)
    geoms = {}

    def geom(seed):
        if seed not in geoms:
            geoms[seed] = B.igabem_geometry_create(ctx, inputs.deformed_sphere_patches(seed=seed, spans=4))
        return geoms[seed]

    def opt(r):
        # block preconditioner; sound-soft GMRES(30), sound-hard GMRES(300) (see the C2 workload);
        # level-adaptive q (7 .. 12) under the kappa * diameter <= 6 cap, as in the large-scatterer
        # workload (the cap alone leaves only the finest level admissible at kappa ~ 30); the M2L
        # coupling blocks stored in FP32 (set up once, read by every product: the many-iteration
        # sound-hard solves gain most).  A request that has not reached the tolerance after max_iter
        # iterations is reported as failed.
        return B.igabem_default_options(level_m=r["m"], degree_p=2, kappa=r["kappa"],
                                        eta_cfie=1.0 / r["kappa"] if r["bc"] else r["kappa"],
                                        bc=r["bc"], cheb_q=7, q_max=12, eta_adm=0.5, leaf_offset=2, kappa_cap=6.0,
                                        precision=B.MIXED_FP32, tol=1e-5, max_iter=args.max_iter,
                                        gmres_restart=300 if r["bc"] else 30, precond=1,
                                        m2l_stored=1)
    for r in reqs:
        geom(r["geom_seed"])
    srv = B.igabem_server_create(ctx, 0, args.slots)
    reported = set()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        handles, t_next = [], t0
        for r in reqs:
            t_next += r["gap"] / args.rate
            while time.perf_counter() < t_next:
                time.sleep(min(0.005, max(0.0, t_next - time.perf_counter())))
            handles.append(B.igabem_submit(srv, geom(r["geom_seed"]), opt(r), r["dirs"], xhat))
            _report_done(B, reqs, handles, reported, t0)
        while len(reported) < len(handles):
            time.sleep(0.05)
            _report_done(B, reqs, handles, reported, t0)
        wall = time.perf_counter() - t0
    status = [B.igabem_result(h, raise_errors=False)[2] for h in handles]
    st = B.igabem_server_get_stats(srv)
    for h in handles:
        B.igabem_request_destroy(h)
    B.igabem_server_destroy(srv)
    ok = sum(1 for c in status if c == 0)
    out = {"metric": METRIC, "value": ok / wall * world, "unit": "solves/s", "n_gpus": world, "steps": len(reqs),
           "warmup": 0, "ms_per_step": 1e3 * wall / max(1, len(reqs)), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded deformed spheres, Poisson arrivals)",
           "config": {"workload": "serving_stream", "requests": len(reqs), "arrival_rate_per_s": args.rate,
                      "slots": args.slots, "precision": "mixed, stored M2L blocks", "cheb_q": "7 .. 12 by level", "tol": 1e-5,
                      "max_iter": args.max_iter},
           "solve_latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean": st["mean_ms"]},
           "completed": st["completed"], "failed": st["failed"], "peak_active": st["peak_active"],
           "peak_bytes": st["peak_bytes"], "statuses": sorted(set(status)), "clocks": clk.summary(),
           "rhs_total": int(sum(len(r["dirs"]) for r in reqs))}
    if rank == 0:
        print(json.dumps(out))


def run_matvec_steps(args, wl, B, inputs, geom, options, stream, flush, local, world, rank, dist, peaks):
    """Workloads whose step is one operator application to all right-hand-side columns (64 for the
    sound-hard deformed sphere): matvecs/s counts every column; one full solve is timed beside."""
    import torch
    R = wl["n_rhs"]
    dirs = inputs.fibonacci_directions(R)
    opt = options(args.precision, max_iter=wl["solve_max_iter"])
    prob = B.igabem_problem_create(geom, opt)
    info = B.igabem_problem_info(prob)
    N = info["n_dofs"]
    x_host = inputs.random_complex(N, seed=2026, cols=R)
    x = torch.tensor(x_host, device="cuda")
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        B.igabem_matvec(prob, x, y)
    B.igabem_profile_get(prob, reset=True)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            B.igabem_matvec(prob, x, y)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist)
    pr = B.igabem_profile_get(prob, reset=True)
    phases = {k: round(v["ms"] / max(1, v["calls"]), 3) for k, v in pr["phases"].items() if v["calls"]}
    m2l_ms = pr["phases"]["m2l"]["ms"] / max(1, pr["phases"]["m2l"]["calls"])
    y_dev = y.cpu().numpy()
    # end to end through the public API with host buffers (x in, y out every step)
    ke = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(ke):
        y_h = B.igabem_matvec(prob, x_host)
    e2e_s = (time.perf_counter() - t0) / ke
    # one full solve of the R directions and the far field
    t0 = time.perf_counter()
    dens, sinfo = B.igabem_solve(prob, dirs, N, raise_on_not_converged=False)
    u = B.igabem_farfield(prob, dens, inputs.fibonacci_directions(wl["n_dir"]))
    solve_s = time.perf_counter() - t0
    B.igabem_problem_destroy(prob)
    # the same product through the FP64 path (the accuracy of this precision), rank 0 only
    err = None
    if rank == 0 and args.precision != "fp64":
        p64 = B.igabem_problem_create(geom, options("fp64"))
        y64 = B.igabem_matvec(p64, x_host)
        B.igabem_problem_destroy(p64)
        err = float(np.abs(y_dev - y64).max() / np.abs(y64).max())
    far = info["n_far_pairs"]
    Q = wl["cheb_q"] ** 2
    C = 7 if wl["bc"] else 1
    useful = far * Q * Q * FLOPS_PER_MAC * C * R                    # complex contraction of the M2L
    samples = far * Q * Q * FLOPS_PER_SAMPLE[bool(wl["bc"])] * (2 if wl["bc"] else 1)
    achieved = (useful + samples) / (m2l_ms / 1e3) / 1e12
    tc = args.precision == "tc"
    peak = (json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
            if tc and os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else peaks["fp32_tflops"])
    kh = (Q + 7) // 8 * 8
    executed = far * 3 * 2 * 128 * (2 * kh) * C * R                  # tensor-core flops issued (split, padding)
    roofline = {"bound": "tensor" if tc else "alu", "kernel": "k_m2l_tc" if tc else "k_m2l_gemm<float>",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": ("measured dense BF16 burst (FP16 has the same tensor rate), MEASURED_PEAKS.json"
                                if tc else "measured FP32 FMA rate (igabem_measure_peaks, this run)"),
                "algorithmic_flops_per_matvec": useful + samples, "avg_ms_per_matvec": m2l_ms,
                "executed_tensor_flops_per_matvec": executed if tc else None,
                "executed_tensor_tflops": executed / (m2l_ms / 1e3) / 1e12 if tc else None}
    value = R * args.steps * world / (total_ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "tc": "f16x2+f32+f64"}[args.precision],
           "data": "synthetic (seeded deformed sphere, seeded complex vectors, Fibonacci directions)",
           "config": {"workload": args.workload, "n_dofs": N, "n_elements": info["n_elements"], "n_rhs": R,
                      "step": f"one operator application to {R} columns (counted as {R} matvecs)",
                      "precision": args.precision, "cheb_q": wl["cheb_q"], "eta_adm": wl["eta_adm"],
                      "kappa": wl["kappa"], "kappa_cap": wl["kappa_cap"], "leaf_offset": wl["leaf_offset"][args.precision],
                      "n_far_pairs": far, "parallelism": f"replicas x{world}",
                      "l2": "flushed (256 MB write) before each step"},
           "phase_ms_per_matvec": phases, "setup_ms": info["setup_ms"], "measured_peaks": peaks,
           "matvec_rel_err_vs_fp64": err,
           "solve": {"gmres_iterations": sinfo["iterations"], "rel_residual": sinfo["rel_residual"],
                     "converged": sinfo["rel_residual"] <= wl["tol"][args.precision],
                     "max_iter": wl["solve_max_iter"],
                     "gmres_restart": wl["restart"], "tol": wl["tol"][args.precision],
                     "seconds": solve_s, "solves_per_s": 1.0 / solve_s, "n_dir": wl["n_dir"],
                     "farfield_finite": bool(np.isfinite(u).all())},
           "gpu_launches": pr["launches"] // max(1, args.steps) * args.steps,
           "clocks": clk.summary(),
           "e2e": {"value": R / e2e_s * world, "unit": "matvecs/s", "h2d_bytes_per_step": int(x_host.nbytes),
                   "d2h_bytes_per_step": int(x_host.nbytes), "ms_per_step": 1e3 * e2e_s},
           "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(wl, with_lu=False)
        t_mv = 1.0 / cb["value"]
        cb.update(value=R / t_mv, unit="matvecs/s",
                  sample=cb["sample"] + f"; the oracle applies the operator by assembling it (no fast method), so "
                                        f"one application to {R} columns costs one assembly")
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_torus_convergence(args):
    """The convergence study of Sec. 5.2 on its geometry: the torus R = 2, r = 0.5 as 16 exact rational
    patches, kappa = 2.5, plane wave d = x^, far field at 100 directions, FP64 with level-adaptive
    interpolation (cheb_q 8, cap 2, up to 14 points), GMRES(30) with the block preconditioner to 1e-11;
    for p = 1, 2 (sound-soft) and p = 1 (sound-hard) the error at m = 1..4 against m = 5 and the
    observed orders in h (expected 2p + 2 for sound-soft, 2p + 1 for sound-hard).  The paper's own
    reference solutions and data logs are not available; the finest level stands in for them."""
    import torch
    from paper_2306_11324_gb300 import binding as B
    from paper_2306_11324_gb300 import inputs
    torch.cuda.set_device(0)
    ctx = B.igabem_create(0, torch.cuda.current_stream().cuda_stream)
    geom = B.igabem_geometry_create(ctx, inputs.torus_patches(2.0, 0.5))
    xh = inputs.fibonacci_directions(100)
    d = np.array([[1.0, 0.0, 0.0]])
    table, orders = [], {}
    for p, hard in ((1, False), (2, False), (1, True)):
        u, info_m = {}, {}
        for m in (1, 2, 3, 4, 5):
            opt = B.igabem_default_options(level_m=m, degree_p=p, kappa=2.5, eta_cfie=(1 / 2.5) if hard else 2.5,
                                           bc=int(hard), cheb_q=8, kappa_cap=2.0, q_max=14, leaf_offset=min(m, 1),
                                           eta_adm=0.5, tol=1e-11, precond=0 if hard else 1,
                                           gmres_restart=300 if hard else 30, max_iter=3000)
            t0 = time.perf_counter()
            prob = B.igabem_problem_create(geom, opt)
            info = B.igabem_problem_info(prob)
            x, sinfo = B.igabem_solve(prob, d, info["n_dofs"], raise_on_not_converged=False)
            u[m] = B.igabem_farfield(prob, x, xh)[:, 0]
            B.igabem_problem_destroy(prob)
            info_m[m] = (info["n_dofs"], sinfo["iterations"], sinfo["rel_residual"], time.perf_counter() - t0)
        errs = {m: float(np.abs(u[m] - u[5]).max() / np.abs(u[5]).max()) for m in (1, 2, 3, 4)}
        for m in (1, 2, 3, 4):
            order = float(np.log2(errs[m - 1] / errs[m])) if m > 1 else None
            table.append({"p": p, "bc": "hard" if hard else "soft", "m": m, "n_dofs": info_m[m][0],
                          "gmres_iterations": info_m[m][1], "rel_residual": info_m[m][2], "seconds": info_m[m][3],
                          "farfield_err_vs_m5": errs[m], "order": order})
        orders[f"p{p}_{'hard' if hard else 'soft'}"] = float(np.log2(errs[2] / errs[3]))
    print(json.dumps({"metric": "far-field self-convergence on the torus (Sec. 5.2)", "value": orders["p1_soft"],
                      "unit": "observed order in h (m = 2 -> 3, against m = 5)", "n_gpus": 1, "steps": 1, "warmup": 0,
                      "higher_is_better": True, "dtype": "f64", "data": "synthetic (exact torus, plane wave d = x^)",
                      "config": {"workload": "torus_convergence", "kappa": 2.5, "R": 2.0, "r": 0.5,
                                 "expected_orders": {"p1_soft": 4, "p2_soft": 6, "p1_hard": 3}},
                      "orders": orders, "table": table}))


def run_sweep_steps(args, wl, B, inputs, geom, patches, stream, flush, local, world, rank, dist, peaks, ctx):
    """The frequency-sweep workload: a step is one kappa of the sweep (set-up, GMRES for all incident
    directions at once, far field); solves/s counts every incident direction.  Beside the timed steps:
    operator applications on a resident problem, the product against the plain FP64 operator on the
    same seeded vector (the FP64 form is compared by matrix-vector products only), and the same steps
    through the public API with host buffers."""
    import torch
    R = wl["n_rhs"]
    dirs = inputs.fibonacci_directions(R)
    xhat = inputs.fibonacci_directions(wl["n_dir"])
    kappas = wl["kappas"]

    def options(precision, kappa, **kw):
        o = dict(level_m=wl["level_m"], degree_p=wl["degree_p"], kappa=kappa,
                 eta_cfie=kappa if wl["eta"] == "kappa" else wl["eta"], bc=wl["bc"], cheb_q=wl["cheb_q"],
                 q_max=wl["q_max"], eta_adm=wl["eta_adm"], leaf_offset=wl["leaf_offset"][precision],
                 tol=wl["tol"][precision], kappa_cap=wl["kappa_cap"], gmres_restart=wl["restart"],
                 max_iter=wl["solve_max_iter"], precond=wl["precond"][precision],
                 precision=PRECISIONS[precision], profile=1,
                 m2l_stored=wl.get("m2l_stored", {}).get(precision, 0))
        o.update(kw)
        return B.igabem_default_options(**o)

    def step(i, host=False):
        kappa = kappas[i % len(kappas)]
        g = B.igabem_geometry_create(ctx, patches) if host else geom
        prob = B.igabem_problem_create(g, options(args.precision, kappa))
        info = B.igabem_problem_info(prob)
        N = info["n_dofs"]
        dens = None if host else torch.empty((N, R), dtype=torch.complex128, device="cuda")
        dens, sinfo = B.igabem_solve(prob, dirs, N, density=dens, raise_on_not_converged=False)
        u = B.igabem_farfield(prob, dens, xhat)
        return g, prob, info, sinfo, u, kappa

    for i in range(args.warmup):
        _, prob, *_ = step(i)
        B.igabem_problem_destroy(prob)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    prof_tot, launches, steps_rec = {}, 0, []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, prob, info, sinfo, u, kappa = step(args.warmup + k)
            ev[k][1].record(stream)
            pr = B.igabem_profile_get(prob)
            launches += pr["launches"]
            for name, v in pr["phases"].items():
                a = prof_tot.setdefault(name, {"ms": 0.0, "calls": 0, "launches": 0})
                for key in a:
                    a[key] += v[key]
            steps_rec.append({"kappa": kappa, "gmres_iterations": sinfo["iterations"],
                              "rel_residual": sinfo["rel_residual"], "matvecs": sinfo["n_matvecs"],
                              "converged": sinfo["rel_residual"] <= wl["tol"][args.precision],
                              "farfield_finite": bool(torch.isfinite(torch.view_as_real(u)).all().item())
                              if hasattr(u, "device") else bool(np.isfinite(u).all())})
            B.igabem_problem_destroy(prob)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist)
    phases = {k: round(v["ms"] / args.steps, 3) for k, v in prof_tot.items() if v["ms"] > 0}
    # operator applications on a resident problem (kappa of the sweep's first value)
    prob = B.igabem_problem_create(geom, options(args.precision, kappas[0]))
    info = B.igabem_problem_info(prob)
    N = info["n_dofs"]
    x_host = inputs.random_complex(N, seed=2028, cols=R)
    x = torch.tensor(x_host, device="cuda")
    y = torch.empty_like(x)
    B.igabem_matvec(prob, x, y)
    B.igabem_profile_get(prob, reset=True)
    nmv = 5
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(nmv):
        B.igabem_matvec(prob, x, y)
    b.record(stream)
    torch.cuda.synchronize()
    mv_ms = a.elapsed_time(b) / nmv
    mv_prof = B.igabem_profile_get(prob, reset=True)
    mv_phases = {k: round(v["ms"] / max(1, v["calls"]), 3) for k, v in mv_prof["phases"].items() if v["calls"]}
    y_mixed = y.cpu().numpy()
    B.igabem_problem_destroy(prob)
    # the plain FP64 operator on the same vector (rank 0)
    err64, fp64_mv_ms = None, None
    if rank == 0 and args.precision != "fp64" and not args.one_form:
        p64 = B.igabem_problem_create(geom, options("fp64", kappas[0]))
        y64 = torch.empty_like(x)
        B.igabem_matvec(p64, x, y64)
        torch.cuda.synchronize()
        a.record(stream)
        B.igabem_matvec(p64, x, y64)
        b.record(stream)
        torch.cuda.synchronize()
        fp64_mv_ms = a.elapsed_time(b)
        y64h = y64.cpu().numpy()
        err64 = float(np.abs(y_mixed - y64h).max() / np.abs(y64h).max())
        B.igabem_problem_destroy(p64)
    # end to end through the public API with host buffers (geometry, problem, solve, far field)
    ke = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(ke):
        g2, p2, *_ = step(args.warmup + i, host=True)
        B.igabem_problem_destroy(p2)
        B.igabem_geometry_destroy(g2)
    e2e_s = (time.perf_counter() - t0) / ke
    _, _, knots, ctrl, w = inputs.patches_to_arrays(patches)
    h2d = int(knots.nbytes + ctrl.nbytes + w.nbytes + 8 * 2 * 2 * len(patches) + dirs.nbytes + xhat.nbytes)
    d2h = int(N * 16 * R + len(xhat) * 16 * R)
    # roofline: the FP64 singular quadrature of the set-up and the M2L of a product
    hard = bool(wl["bc"])
    sing = prof_tot.get("setup_singular", {"ms": 0.0, "calls": 0})
    sing_ms = sing["ms"] / max(1, sing["calls"])
    sing_flops = singular_flops(info, wl["degree_p"], hard)
    sing_ach = sing_flops / (sing_ms / 1e3) / 1e12 if sing_ms > 0 else 0.0
    m2l_ms = mv_phases.get("m2l", 0.0)
    qs = info["level_q"]
    far_by_level = info["level_far"]
    C = 7 if hard else 1
    m2l_samples = sum(f * q ** 4 for f, q in zip(far_by_level, qs))
    m2l_flops = sum(f * q ** 4 * (FLOPS_PER_SAMPLE[hard] * (2 if hard else 1) + FLOPS_PER_MAC * C * R)
                    for f, q in zip(far_by_level, qs))
    m2l_ach = m2l_flops / (m2l_ms / 1e3) / 1e12 if m2l_ms > 0 else 0.0
    stored = wl.get("m2l_stored", {}).get(args.precision, 0)
    if stored:
        # the stored blocks are read once per product: q^4 FP32 complex entries per far pair (x 2 hard)
        ebytes = 8 if args.precision != "fp64" else 16
        m2l_bytes = sum(f * q ** 4 for f, q in zip(far_by_level, qs)) * (2 if hard else 1) * ebytes
        hbm = hbm_peak_gbs()
        m2l_gbs = m2l_bytes / (m2l_ms / 1e3) / 1e9 if m2l_ms > 0 else 0.0
        m2l_roof = {"kernel": "k_m2l_stored<float>", "bound": "hbm", "achieved": m2l_gbs, "unit": "GB/s",
                    "peak": hbm, "frac": m2l_gbs / hbm if hbm else None,
                    "algorithmic_bytes_per_matvec": m2l_bytes, "avg_ms_per_matvec": m2l_ms,
                    "peak_source": "measured copy bandwidth, MEASURED_PEAKS.json"}
    else:
        m2l_roof = {"kernel": "k_m2l_rows<float> / k_m2l_gemm<float>", "achieved": m2l_ach, "unit": "TFLOP/s",
                    "peak": peaks["fp32_tflops"], "frac": m2l_ach / peaks["fp32_tflops"],
                    "xu_frac": (m2l_samples / (peaks["sincosf_gops"] * 1e9) + m2l_samples / (peaks["rsqrtf_gops"] * 1e9))
                    / (m2l_ms / 1e3) if m2l_ms > 0 else None,
                    "algorithmic_flops_per_matvec": m2l_flops, "avg_ms_per_matvec": m2l_ms,
                    "node_pairs_per_matvec": m2l_samples,
                    "peak_source": "measured FP32 FMA rate (igabem_measure_peaks, this run)"}
    roofline = {"bound": "alu", "kernel": "k_near_singular (FP64)", "achieved": sing_ach,
                "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": sing_ach / peaks["fp64_tflops"],
                "traffic": SINGULAR_DRAM_BYTES_PER_POINT * info["n_singular_points"],
                "traffic_source": "DRAM bytes per 4-D point of one ncu capture of the small sweep case, "
                                  "times this launch's points",
                "peak_source": "measured FP64 FMA rate (igabem_measure_peaks, this run; 2 flops per FMA)",
                "algorithmic_flops_per_setup": sing_flops, "avg_ms_per_setup": sing_ms,
                "singular_points": info["n_singular_points"],
                "singular_geometry_points": info["n_singular_geo_points"],
                "singular_geometry_columns": info["n_singular_geo_columns"],
                "singular_groups": info["n_singular_groups"],
                "singular_factored_points": info["n_singular_factored_points"],
                "m2l": m2l_roof}
    lat = sorted(step_ms)
    value = R * args.steps * world / (total_ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "tc": "f16x2+f32+f64"}[args.precision],
           "data": "synthetic (seeded deformed sphere, Fibonacci directions, seeded complex vectors)",
           "config": {"workload": args.workload, "n_dofs": N, "n_elements": info["n_elements"], "n_rhs": R,
                      "step": f"one kappa of the sweep: set-up, GMRES for {R} directions, far field at "
                              f"{wl['n_dir']} directions (counted as {R} solves)",
                      "kappas": [kappas[(args.warmup + k) % len(kappas)] for k in range(args.steps)],
                      "precision": args.precision, "cheb_q": wl["cheb_q"], "q_max": wl["q_max"],
                      "level_q": qs, "level_far": far_by_level, "eta_adm": wl["eta_adm"],
                      "kappa_cap": wl["kappa_cap"], "leaf_offset": wl["leaf_offset"][args.precision],
                      "gmres_restart": wl["restart"], "tol": wl["tol"][args.precision],
                      "precond": wl["precond"][args.precision], "n_far_pairs": info["n_far_pairs"],
                      "m2l_stored": wl.get("m2l_stored", {}).get(args.precision, 0),
                      "parallelism": f"replicas x{world}",
                      "l2": "working set far above L2 (and a 256 MB write before each step)"},
           "steps_detail": steps_rec,
           "solve_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "phase_ms_per_step": phases, "setup_ms": info["setup_ms"], "host_setup_ms": info["host_setup_ms"],
           "device_bytes": info["device_bytes"],
           "matvecs_per_s": R * 1e3 / mv_ms * world, "matvec_ms": mv_ms, "phase_ms_per_matvec": mv_phases,
           "matvec_rel_err_vs_fp64": err64, "fp64_matvec_ms": fp64_mv_ms,
           "fp64_matvecs_per_s": R * 1e3 / fp64_mv_ms if fp64_mv_ms else None,
           "gpu_launches": launches, "clocks": clk.summary(), "measured_peaks": peaks,
           "e2e": {"value": R / e2e_s * world, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s},
           "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(wl, with_lu=True)
        cb.update(value=R * cb["value"],
                  sample=cb["sample"] + f"; {R} directions per solve counted as {R} solves")
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving_stream":
        return run_serving(args)
    if args.workload == "torus_convergence":
        return run_torus_convergence(args)
    import torch
    from paper_2306_11324_gb300 import binding as B
    from paper_2306_11324_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    PRECISIONS.update(fp64=B.FP64, mixed=B.MIXED_FP32, tc=B.MIXED_TC)
    if args.precision is None:
        args.precision = wl["precision"]
    stream = torch.cuda.current_stream()
    ctx = B.igabem_create(local, stream.cuda_stream)
    patches = patches_of(wl["geometry"])
    geom = B.igabem_geometry_create(ctx, patches)
    dirs = np.array([[0.0, 0.0, 1.0]]) if wl["n_rhs"] == 1 else inputs.fibonacci_directions(wl["n_rhs"])
    xhat = inputs.fibonacci_directions(wl["n_dir"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # larger than the 129 MB L2

    def options(precision, max_iter=5000):
        leaf = wl["leaf_offset"][precision]
        return B.igabem_default_options(level_m=wl["level_m"], degree_p=wl["degree_p"], kappa=wl["kappa"],
                                        eta_cfie=wl["eta"], bc=wl["bc"], cheb_q=wl["cheb_q"],
                                        eta_adm=wl["eta_adm"], leaf_offset=leaf, tol=wl["tol"][precision],
                                        kappa_cap=wl["kappa_cap"], gmres_restart=wl["restart"],
                                        max_iter=max_iter, precond=wl["precond"][precision],
                                        precision=PRECISIONS[precision], profile=1, q_max=wl.get("q_max", 0))

    def request(opt, host=False):
        """One request through the public API; returns (problem, info, solve info, far field)."""
        prob = B.igabem_problem_create(geom, opt)
        info = B.igabem_problem_info(prob)
        N = info["n_dofs"]
        dens = None if host else torch.empty((N, len(dirs)), dtype=torch.complex128, device="cuda")
        dens, sinfo = B.igabem_solve(prob, dirs, N, density=dens)
        u = B.igabem_farfield(prob, dens, xhat)
        return prob, info, sinfo, u

    def run_form(precision, steps, warmup, timed_clocks):
        opt = options(precision)
        for _ in range(warmup):
            prob, *_ = request(opt)
            B.igabem_problem_destroy(prob)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        prof_tot, launches, iters, mvs, u_last = {}, 0, [], [], None
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                prob, info, sinfo, u = request(opt)
                ev[k][1].record(stream)
                pr = B.igabem_profile_get(prob)
                launches += pr["launches"]
                for name, v in pr["phases"].items():
                    a = prof_tot.setdefault(name, {"ms": 0.0, "calls": 0, "launches": 0})
                    for key in a:
                        a[key] += v[key]
                iters.append(sinfo["iterations"])
                mvs.append(sinfo["n_matvecs"])
                u_last = u
                B.igabem_problem_destroy(prob)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_ms = max_over_ranks(sum(step_ms), dist)
        # operator applications on a resident problem
        prob = B.igabem_problem_create(geom, opt)
        info = B.igabem_problem_info(prob)
        x = torch.tensor(inputs.random_complex(info["n_dofs"], cols=len(dirs)), device="cuda")
        y = torch.empty_like(x)
        B.igabem_matvec(prob, x, y)
        nmv = 20
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nmv):
            B.igabem_matvec(prob, x, y)
        b.record(stream)
        torch.cuda.synchronize()
        B.igabem_problem_destroy(prob)
        lat = sorted(step_ms)
        return {"precision": precision, "solves_per_s": steps * world / (total_ms / 1e3),
                "ms_per_step": total_ms / steps, "matvec_ms": a.elapsed_time(b) / nmv,
                "matvecs_per_s": 1e3 / (a.elapsed_time(b) / nmv) * world,
                "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "iters": iters[-1], "mvs": mvs[-1], "launches": launches, "info": info,
                "phases": {k: round(v["ms"] / steps, 3) for k, v in prof_tot.items() if v["ms"] > 0},
                "prof": prof_tot, "u": u_last.cpu().numpy(), "clocks": clk.summary(),
                "leaf_offset": wl["leaf_offset"][precision], "tol": wl["tol"][precision]}

    peaks = B.igabem_measure_peaks(ctx)
    if wl.get("step") == "sweep":
        return run_sweep_steps(args, wl, B, inputs, geom, patches, stream, flush, local, world, rank, dist, peaks,
                               ctx)
    if wl.get("step") == "matvec":
        return run_matvec_steps(args, wl, B, inputs, geom, options, stream, flush, local, world, rank, dist, peaks)
    main_form = run_form(args.precision, args.steps, args.warmup, True)
    other = "mixed" if args.precision == "fp64" else "fp64"
    other_form = run_form(other, max(1, min(args.steps, 3)), 1, False) if not args.one_form else None
    if other_form is not None:
        fp64_u = (main_form if args.precision == "fp64" else other_form)["u"]
        mix_u = (other_form if args.precision == "fp64" else main_form)["u"]
        far_err = float(np.abs(mix_u - fp64_u).max() / np.abs(fp64_u).max())
    else:
        far_err = None

    # the unit sphere's far field against the Mie series (discretisation + FMM + solver error)
    mie_err = None
    if wl["geometry"] == "sphere" and not wl["bc"] and len(dirs) == 1:
        ref = mie_soft_far_field(wl["kappa"], xhat, dirs[0])
        mie_err = float(np.abs(main_form["u"][:, 0] - ref).max() / np.abs(ref).max())

    # ---- end to end through the public API with host buffers ----
    opt = options(args.precision)
    ke = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = []
    for _ in range(ke):
        s0 = time.perf_counter()
        g2 = B.igabem_geometry_create(ctx, patches)
        p2 = B.igabem_problem_create(g2, opt)
        N = B.igabem_problem_info(p2)["n_dofs"]
        d_h, _ = B.igabem_solve(p2, dirs, N)
        u_h = B.igabem_farfield(p2, d_h, xhat)
        B.igabem_problem_destroy(p2)
        B.igabem_geometry_destroy(g2)
        e2e_steps.append(time.perf_counter() - s0)
    e2e_value = ke / (time.perf_counter() - t0) * world
    _, _, knots, ctrl, w = inputs.patches_to_arrays(patches)
    info = main_form["info"]
    h2d = int(knots.nbytes + ctrl.nbytes + w.nbytes + 8 * 2 * 2 * len(patches) + dirs.nbytes + xhat.nbytes)
    d2h = int(info["n_dofs"] * 16 * len(dirs) + len(xhat) * 16 * len(dirs))

    # ---- roofline of the dominant kernel of a solve step from the timed region's CUDA events: the FP64
    # singular quadrature of the touching element pairs (k_near_singular); the M2L beside it ----
    far = info["n_far_pairs"]
    Q = wl["cheb_q"] ** 2
    hard = bool(wl["bc"])
    fp64 = args.precision == "fp64"
    sing = main_form["prof"].get("setup_singular", {"ms": 0.0, "calls": 0})
    sing_ms = sing["ms"] / max(1, sing["calls"])
    sing_flops = singular_flops(info, wl["degree_p"], hard)
    sing_achieved = sing_flops / (sing_ms / 1e3) / 1e12 if sing_ms > 0 else 0.0
    m2l = main_form["prof"].get("m2l", {"ms": 0.0, "calls": 0})
    m2l_ms = m2l["ms"] / max(1, m2l["calls"])
    roofline = {"bound": "alu", "kernel": "k_near_singular (FP64)", "achieved": sing_achieved,
                "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": sing_achieved / peaks["fp64_tflops"],
                "traffic": None,
                "peak_source": "measured FP64 FMA rate (igabem_measure_peaks, this run; 2 flops per FMA)",
                "algorithmic_flops_per_setup": sing_flops, "avg_ms_per_setup": sing_ms,
                "singular_points": info["n_singular_points"],
                "singular_geometry_points": info["n_singular_geo_points"],
                "singular_geometry_columns": info["n_singular_geo_columns"],
                "singular_groups": info["n_singular_groups"],
                "singular_factored_points": info["n_singular_factored_points"],
                "m2l": m2l_alu_roofline("k_m2l_rows<double>" if fp64 else "k_m2l_rows<float>", far, Q, hard,
                                        len(dirs), m2l_ms, peaks, fp64)}

    def summary(f):
        return {"precision": f["precision"], "precond": wl["precond"][f["precision"]], "solves_per_s": f["solves_per_s"], "matvecs_per_s": f["matvecs_per_s"],
                "matvec_ms": f["matvec_ms"], "ms_per_step": f["ms_per_step"], "leaf_offset": f["leaf_offset"],
                "gmres_tol": f["tol"], "gmres_iterations": f["iters"], "matvecs_per_solve": f["mvs"],
                "solve_latency_ms": {"p50": f["p50"], "p99": f["p99"]}, "phase_ms_per_step": f["phases"],
                "setup_ms": f["info"]["setup_ms"]}

    out = {
        "metric": METRIC, "value": main_form["solves_per_s"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_form["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32+f64",
        "data": "synthetic (seeded geometry, plane wave)",
        "config": {"workload": args.workload, "n_dofs": info["n_dofs"], "n_elements": info["n_elements"],
                   "n_rhs": len(dirs), "kappa_cap": wl["kappa_cap"],
                   "precision": args.precision, "leaf_offset": main_form["leaf_offset"], "cheb_q": wl["cheb_q"],
                   "eta_adm": wl["eta_adm"], "kappa": wl["kappa"], "tol": main_form["tol"],
                   "gmres_restart": wl["restart"], "precond": wl["precond"][args.precision],
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before each step"},
        "matvecs_per_s": main_form["matvecs_per_s"],
        "matvec_ms": main_form["matvec_ms"],
        "solve_latency_ms": {"p50": main_form["p50"], "p99": main_form["p99"]},
        "gmres_iterations": main_form["iters"], "matvecs_per_solve": main_form["mvs"],
        "phase_ms_per_step": main_form["phases"],
        "other_form": summary(other_form) if other_form is not None else None,
        "farfield_rel_err_mixed_vs_fp64": far_err,
        "farfield_rel_err_vs_mie": mie_err,
        "measured_peaks": peaks,
        "gpu_launches": main_form["launches"],
        "clocks": main_form["clocks"],
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * statistics.mean(e2e_steps)},
        "roofline": roofline,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(wl)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
