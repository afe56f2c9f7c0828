"""ctypes binding of libigabem.so (include/igabem.h): the same entry points, argument marshalling only.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA memory of the context's
device); complex arrays are complex128 in the [N][R] layout of the C ABI.  Every computation runs in
the CUDA library: if it is not built this module raises on import of the library, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c_int, c_long, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_long, ctypes.c_double,
                                                ctypes.c_void_p, ctypes.c_size_t)

IGABEM_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOT_CONVERGED", -5: "ENUMERIC", -6: "ETIMEOUT"}
SOUND_SOFT, SOUND_HARD = 0, 1
FP64, MIXED_FP32, MIXED_TC = 0, 1, 2


class igabem_options(ctypes.Structure):
    _fields_ = [("degree_p", c_int), ("level_m", c_int), ("kappa", c_double), ("eta_cfie", c_double),
                ("bc", c_int), ("cheb_q", c_int), ("leaf_offset", c_int), ("eta_adm", c_double),
                ("kappa_cap", c_double), ("gauss_regular", c_int), ("gauss_singular", c_int),
                ("precision", c_int), ("gmres_restart", c_int), ("max_iter", c_int), ("tol", c_double),
                ("no_fmm", c_int), ("profile", c_int), ("precond", c_int), ("q_max", c_int),
                ("m2l_stored", c_int), ("no_graph", c_int)]


class igabem_info(ctypes.Structure):
    _fields_ = [("n_dofs", c_long), ("n_patch_dofs", c_long), ("n_elements", c_long),
                ("n_clusters", c_long), ("n_near_pairs", c_long), ("n_near_element_pairs", c_long),
                ("n_touching_pairs", c_long), ("n_far_pairs", c_long), ("device_bytes", c_size_t),
                ("setup_ms", c_double), ("host_setup_ms", c_double), ("n_singular_points", c_long),
                ("n_levels", c_int), ("level_q", c_int * 24), ("level_far", c_long * 24),
                ("n_singular_geo_points", c_long), ("n_singular_geo_columns", c_long),
                ("n_singular_groups", c_long), ("n_singular_factored_points", c_long)]


class igabem_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("rel_residual", c_double), ("n_matvecs", c_int),
                ("solve_ms", c_double)]


PHASES = ["setup_tables", "setup_near", "gather", "near", "p2m", "m2m", "m2l", "l2l", "l2p", "krylov",
          "rhs", "farfield", "setup_singular"]


class igabem_profile(ctypes.Structure):
    _fields_ = [("launches", c_long), ("ms", c_double * len(PHASES)), ("calls", c_long * len(PHASES)),
                ("phase_launches", c_long * len(PHASES))]


class igabem_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_long), ("completed", c_long), ("failed", c_long), ("p50_ms", c_double),
                ("p99_ms", c_double), ("mean_ms", c_double), ("solves_per_s", c_double),
                ("peak_bytes", c_size_t), ("budget_bytes", c_size_t), ("peak_active", c_int),
                ("merged", c_long), ("cache_hits", c_long), ("resident", c_long)]


class igabem_peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", c_double), ("fp64_tflops", c_double), ("sincosf_gops", c_double),
                ("rsqrtf_gops", c_double), ("sincos_fp64_gops", c_double), ("sm_count", c_int),
                ("sm_clock_mhz_attr", c_double)]


class igabem_tune_info(ctypes.Structure):
    _fields_ = [("leaf_offset", c_int), ("m2l_stored", c_int), ("setup_ms", c_double), ("matvec_ms", c_double),
                ("score_ms", c_double), ("candidates", c_int), ("from_cache", c_int)]


class IgabemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_LIB = None

# name -> (restype, argtypes); the complete list of entry points declared in include/igabem.h
SIGNATURES = {
    "igabem_last_error": (ctypes.c_char_p, []),
    "igabem_default_options": (None, [ctypes.POINTER(igabem_options)]),
    "igabem_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p]),
    "igabem_destroy": (None, [c_void_p]),
    "igabem_geometry_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, ctypes.POINTER(c_void_p)]),
    "igabem_geometry_destroy": (None, [c_void_p]),
    "igabem_problem_create": (c_int, [c_void_p, ctypes.POINTER(igabem_options), ctypes.POINTER(c_void_p)]),
    "igabem_problem_info": (c_int, [c_void_p, ctypes.POINTER(igabem_info)]),
    "igabem_problem_destroy": (None, [c_void_p]),
    "igabem_rhs": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_matvec": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(igabem_solve_info)]),
    "igabem_farfield": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_profile_enable": (c_int, [c_void_p, c_int]),
    "igabem_profile_get": (c_int, [c_void_p, ctypes.POINTER(igabem_profile), c_int]),
    "igabem_farfield_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_wait_selftest": (c_int, [c_void_p, ctypes.c_double]),
    "igabem_measure_peaks": (c_int, [c_void_p, ctypes.POINTER(igabem_peaks)]),
    "igabem_potential": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_autotune": (c_int, [c_void_p, ctypes.POINTER(igabem_options), c_int, c_int, ctypes.c_char_p,
                                ctypes.POINTER(igabem_options), ctypes.POINTER(igabem_tune_info)]),
    "igabem_solve_sources": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(igabem_solve_info)]),
    "igabem_rhs_sources": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "igabem_server_create": (c_int, [c_void_p, c_size_t, c_int, ctypes.POINTER(c_void_p)]),
    "igabem_server_destroy": (c_int, [c_void_p]),
    "igabem_submit": (c_int, [c_void_p, c_void_p, ctypes.POINTER(igabem_options), c_int, c_void_p, c_int,
                              c_void_p, ctypes.POINTER(c_void_p)]),
    "igabem_poll": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "igabem_wait": (c_int, [c_void_p, c_double]),
    "igabem_result": (c_int, [c_void_p, c_void_p, ctypes.POINTER(igabem_solve_info)]),
    "igabem_request_destroy": (None, [c_void_p]),
    "igabem_server_get_stats": (c_int, [c_void_p, ctypes.POINTER(igabem_server_stats)]),
}


def lib(path: str | None = None):
    """Load libigabem.so (building it in-tree if the sources changed) and declare its symbols."""
    global _LIB
    if _LIB is None:
        path = path or _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _LIB = L
    return _LIB


def _check(rc):
    if rc != IGABEM_OK:
        raise IgabemError(rc, lib().igabem_last_error().decode())


def _ptr(a):
    """Device or host address of a numpy array or torch tensor (kept alive by the caller)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _is_torch(a):
    return hasattr(a, "data_ptr")


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _like(ref, shape):
    """complex128 output in the memory of `ref` (numpy or torch, same device)."""
    if _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=torch.complex128, device=ref.device)
    return np.empty(shape, dtype=np.complex128)


def igabem_last_error() -> str:
    return lib().igabem_last_error().decode()


def igabem_default_options(**kw) -> igabem_options:
    o = igabem_options()
    lib().igabem_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def igabem_create(device: int = 0, stream: int | None = None):
    h = c_void_p()
    _check(lib().igabem_create(ctypes.byref(h), device, c_void_p(stream) if stream else None))
    return h


def igabem_destroy(ctx):
    lib().igabem_destroy(ctx)


def igabem_geometry_create(ctx, patches):
    """patches: objects with p1, p2, knots1, knots2, ctrl (k1,k2,3), weights (k1,k2)."""
    deg = _host([[p.p1, p.p2] for p in patches], np.int32)
    cnt = _host([[p.ctrl.shape[0], p.ctrl.shape[1]] for p in patches], np.int32)
    knots = _host(np.concatenate([np.concatenate([p.knots1, p.knots2]) for p in patches]), np.float64)
    ctrl = _host(np.concatenate([np.asarray(p.ctrl).reshape(-1, 3) for p in patches]), np.float64)
    w = _host(np.concatenate([np.asarray(p.weights).reshape(-1) for p in patches]), np.float64)
    h = c_void_p()
    _check(lib().igabem_geometry_create(ctx, len(patches), _ptr(deg), _ptr(cnt), _ptr(knots),
                                        _ptr(ctrl), _ptr(w), ctypes.byref(h)))
    return h


def igabem_geometry_destroy(geom):
    lib().igabem_geometry_destroy(geom)


def igabem_problem_create(geom, opt: igabem_options):
    h = c_void_p()
    _check(lib().igabem_problem_create(geom, ctypes.byref(opt), ctypes.byref(h)))
    return h


def igabem_problem_info(prob) -> dict:
    i = igabem_info()
    _check(lib().igabem_problem_info(prob, ctypes.byref(i)))
    out = {k: getattr(i, k) for k, _ in igabem_info._fields_}
    n = min(i.n_levels, 24)
    out["level_q"] = list(i.level_q[:n])
    out["level_far"] = list(i.level_far[:n])
    return out


def igabem_problem_destroy(prob):
    lib().igabem_problem_destroy(prob)


def _ncols(a):
    return 1 if len(a.shape) == 1 else int(a.shape[1])


def igabem_rhs(prob, dirs, n_dofs: int, out=None):
    d = _host(dirs, np.float64).reshape(-1, 3)
    R = d.shape[0]
    out = np.empty((n_dofs, R), np.complex128) if out is None else out
    _check(lib().igabem_rhs(prob, R, _ptr(d), _ptr(out)))
    return out


def igabem_matvec(prob, x, y=None):
    R = _ncols(x)
    y = _like(x, tuple(x.shape)) if y is None else y
    _check(lib().igabem_matvec(prob, R, _ptr(x), _ptr(y)))
    return y


def igabem_solve(prob, dirs, n_dofs: int, density=None, raise_on_not_converged=True):
    d = _host(dirs, np.float64).reshape(-1, 3)
    R = d.shape[0]
    density = np.empty((n_dofs, R), np.complex128) if density is None else density
    info = igabem_solve_info()
    rc = lib().igabem_solve(prob, R, _ptr(d), _ptr(density), ctypes.byref(info))
    if rc != IGABEM_OK and (raise_on_not_converged or rc != -4):
        _check(rc)
    return density, {k: getattr(info, k) for k, _ in igabem_solve_info._fields_}


def igabem_solve_sources(prob, z, n_dofs: int, density=None, raise_on_not_converged=True):
    """Solve for incident point sources G(x, z_r) at the points z [n][3]."""
    zz = _host(z, np.float64).reshape(-1, 3)
    R = zz.shape[0]
    density = np.empty((n_dofs, R), np.complex128) if density is None else density
    info = igabem_solve_info()
    rc = lib().igabem_solve_sources(prob, R, _ptr(zz), _ptr(density), ctypes.byref(info))
    if rc != IGABEM_OK and (raise_on_not_converged or rc != -4):
        _check(rc)
    return density, {k: getattr(info, k) for k, _ in igabem_solve_info._fields_}


def igabem_rhs_sources(prob, z, n_dofs: int, out=None):
    zz = _host(z, np.float64).reshape(-1, 3)
    R = zz.shape[0]
    out = np.empty((n_dofs, R), np.complex128) if out is None else out
    _check(lib().igabem_rhs_sources(prob, R, _ptr(zz), _ptr(out)))
    return out


def igabem_potential(prob, density, points, out=None):
    """Scattered field [n_pts][R] at points [n_pts][3] (numpy or torch, host or CUDA)."""
    R = _ncols(density)
    pts = points if _is_torch(points) else _host(points, np.float64).reshape(-1, 3)
    n = int(pts.shape[0])
    if out is None:
        out = np.empty((n, R), np.complex128)
    dens = density if _is_torch(density) else _host(density, np.complex128)
    _check(lib().igabem_potential(prob, R, _ptr(dens), n, _ptr(pts), _ptr(out)))
    return out


def igabem_farfield(prob, density, xhat, out=None):
    R = _ncols(density)
    xh = _host(xhat, np.float64).reshape(-1, 3)
    out = _like(density, (xh.shape[0], R)) if out is None else out
    _check(lib().igabem_farfield(prob, R, _ptr(density), xh.shape[0], _ptr(xh), _ptr(out)))
    return out


def igabem_server_create(ctx, memory_budget: int = 0, max_active: int = 4):
    h = c_void_p()
    _check(lib().igabem_server_create(ctx, memory_budget, max_active, ctypes.byref(h)))
    return h


def igabem_server_destroy(srv):
    _check(lib().igabem_server_destroy(srv))


class Request:
    """A submitted request and the host arrays it was given (kept alive until it is destroyed)."""

    def __init__(self, handle, n_rhs, n_dir, keep):
        self.handle, self.n_rhs, self.n_dir, self._keep = handle, n_rhs, n_dir, keep


def igabem_submit(srv, geom, opt: igabem_options, dirs, xhat) -> Request:
    d = _host(dirs, np.float64).reshape(-1, 3)
    xh = _host(xhat, np.float64).reshape(-1, 3)
    h = c_void_p()
    _check(lib().igabem_submit(srv, geom, ctypes.byref(opt), d.shape[0], _ptr(d), xh.shape[0], _ptr(xh),
                               ctypes.byref(h)))
    return Request(h, d.shape[0], xh.shape[0], (d, xh, opt))


def igabem_poll(req: Request) -> bool:
    done = c_int(0)
    _check(lib().igabem_poll(req.handle, ctypes.byref(done)))
    return bool(done.value)


def igabem_wait(req: Request, timeout_s: float = -1.0):
    _check(lib().igabem_wait(req.handle, timeout_s))


def igabem_result(req: Request, raise_errors: bool = True):
    """(far field [n_dir][n_rhs], solve info dict, status code)."""
    u = np.zeros((req.n_dir, req.n_rhs), np.complex128)
    info = igabem_solve_info()
    rc = lib().igabem_result(req.handle, _ptr(u), ctypes.byref(info))
    if rc != IGABEM_OK and raise_errors:
        _check(rc)
    return u, {k: getattr(info, k) for k, _ in igabem_solve_info._fields_}, rc


def igabem_request_destroy(req: Request):
    lib().igabem_request_destroy(req.handle)


def igabem_server_get_stats(srv) -> dict:
    st = igabem_server_stats()
    _check(lib().igabem_server_get_stats(srv, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in igabem_server_stats._fields_}


def igabem_wait_selftest(ctx, limit_s: float) -> int:
    """Runs the bounded device wait on a barrier nothing arrives at; returns the status code
    (IGABEM_ETIMEOUT = -6 expected)."""
    return lib().igabem_wait_selftest(ctx, float(limit_s))


def igabem_farfield_noalloc(prob, density, xhat, uinf):
    """Far field with no device allocation: density [N][R], xhat [n_dir][3] (float64) and uinf
    [n_dir][R] must be CUDA tensors of the context's device (see include/igabem.h)."""
    R = _ncols(density)
    _check(lib().igabem_farfield_noalloc(prob, R, _ptr(density), int(xhat.shape[0]), _ptr(xhat), _ptr(uinf)))
    return uinf


def igabem_autotune(geom, opt: igabem_options, n_rhs: int, matvecs_per_setup: int = 30, cache_path=None):
    """(tuned options, info dict): the fastest leaf size / M2L storage for this geometry and options."""
    out = igabem_options()
    info = igabem_tune_info()
    path = cache_path.encode() if cache_path else None
    _check(lib().igabem_autotune(geom, ctypes.byref(opt), int(n_rhs), int(matvecs_per_setup), path,
                                 ctypes.byref(out), ctypes.byref(info)))
    return out, {k: getattr(info, k) for k, _ in igabem_tune_info._fields_}


def igabem_measure_peaks(ctx) -> dict:
    """Measured FP32 / FP64 FMA, sincosf, rsqrtf and FP64 sincos rates of the context's device."""
    p = igabem_peaks()
    _check(lib().igabem_measure_peaks(ctx, ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in igabem_peaks._fields_}


def igabem_profile_enable(prob, on: bool = True):
    _check(lib().igabem_profile_enable(prob, 1 if on else 0))


def igabem_profile_get(prob, reset: bool = False) -> dict:
    p = igabem_profile()
    _check(lib().igabem_profile_get(prob, ctypes.byref(p), 1 if reset else 0))
    return {"launches": p.launches,
            "phases": {name: {"ms": p.ms[i], "calls": p.calls[i], "launches": p.phase_launches[i]}
                       for i, name in enumerate(PHASES)}}


def header_symbols() -> list[str]:
    """Entry points declared in include/igabem.h (for the export check)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "igabem.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"\b(igabem_[a-z_]+)\s*\(", src)))
