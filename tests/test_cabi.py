"""The C-ABI library builds, loads and exports every entry point of include/igabem.h (CPU only:
no compute calls)."""
import ctypes
import subprocess

from paper_2306_11324_gb300 import binding


def test_library_exports_every_header_symbol():
    L = binding.lib()
    declared = binding.header_symbols()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared) <= exported
    assert set(binding.SIGNATURES) == set(declared)


def test_default_options_and_error_path_without_a_gpu():
    o = binding.igabem_default_options()
    assert (o.degree_p, o.cheb_q, o.gauss_regular, o.gauss_singular, o.gmres_restart) == (2, 7, 4, 5, 30)
    assert o.eta_adm == 0.5 and o.precision == binding.FP64
    # invalid arguments are refused with a message before any device work
    rc = binding.lib().igabem_problem_create(None, ctypes.byref(o), ctypes.byref(ctypes.c_void_p()))
    assert rc == -1 and "invalid" in binding.igabem_last_error()
