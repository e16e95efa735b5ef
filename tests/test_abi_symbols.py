"""The C-ABI library loads and exports every symbol include/gw.h declares (no GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|size_t|char\s*\*|void)\s*\*?\s*(gw_\w+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def _lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gw_build", os.path.join(ROOT, "paper_1003_0316_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return ctypes.CDLL(mod.build())


def test_header_declares_entry_points():
    names = _declared()
    for need in ("gw_polarization", "gw_screened_w", "gw_sigma_c", "gw_continue",
                 "gw_transition_weights", "gw_sigma_pair_coeffs", "gw_sigma_convolve",
                 "gw_check", "gw_last_error", "gw_version"):
        assert need in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_errors_without_gpu():
    """Argument validation returns before any device call."""
    lib = _lib()
    lib.gw_transition_weights.restype = ctypes.c_int
    lib.gw_last_error.restype = ctypes.c_char_p
    rc = lib.gw_transition_weights(ctypes.c_int64(-1), None, None, ctypes.c_double(1.0),
                                   ctypes.c_int(4), None, None, None)
    assert rc == 1 and b"K" in lib.gw_last_error()
    om = (ctypes.c_double * 2)(0.5, 1.0)
    rc = lib.gw_transition_weights(ctypes.c_int64(10), None, None, ctypes.c_double(1.0),
                                   ctypes.c_int(0), om, None, None)
    assert rc == 1
    lib.gw_version.restype = ctypes.c_int
    assert lib.gw_version() >= 10000
