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


def test_extrapolar_and_real_entry_points_reject_bad_arguments_without_gpu():
    """The extrapolar, real-dielectric and convolution entry points validate their host
    arguments before any device call (GW_EINVAL = 1)."""
    lib = _lib()
    lib.gw_polarization_extrapolar.restype = ctypes.c_int
    K = (ctypes.c_int64 * 1)(10)
    nb = (ctypes.c_int * 1)(8)
    om = (ctypes.c_double * 2)(0.5, 1.0)
    # no Delta_bar / completeness arrays
    rc = lib.gw_polarization_extrapolar(1, K, nb, None, 1, None, None, None, None, None, None,
                                        None, ctypes.c_double(0.5), 2, om, None, 1, None,
                                        ctypes.c_size_t(0), None)
    assert rc == 1
    lib.gw_sigma_extrapolar.restype = ctypes.c_int
    rc = lib.gw_sigma_extrapolar(0, None, None, 4, None, 8, None, None, None, None, None, None,
                                 8, None, None, None, None, ctypes.c_size_t(0), None)
    assert rc == 1
    lib.gw_screened_w_real.restype = ctypes.c_int
    rc = lib.gw_screened_w_real(0, None, 4, None, None, None, None, ctypes.c_size_t(0), None)
    assert rc == 1
    lib.gw_sigma_convolve.restype = ctypes.c_int
    wq = (ctypes.c_double * 1)(1.0)
    npair = (ctypes.c_int64 * 1)(3)
    rc = lib.gw_sigma_convolve(1, wq, npair, 3, om, None, None, None, 2, om, 1, None, None,
                               ctypes.c_size_t(0), None)
    assert rc == 1                       # fewer than 4 frequency nodes


class _PolOpt(ctypes.Structure):
    _fields_ = [("accumulate", ctypes.c_int), ("group_items_per_sm", ctypes.c_int),
                ("b_stages", ctypes.c_int), ("fp64_waves", ctypes.c_int),
                ("herk_events", ctypes.c_void_p), ("n_herk_events", ctypes.c_int),
                ("herk_launches_out", ctypes.c_void_p), ("serial_prep", ctypes.c_int)]


def test_polarization_workspace_holds_one_group_of_large_q():
    """The tensor-core polarization prepares and launches q points group by group: eight q
    that each fill the GPU need two groups' slots of workspace (the next group is prepared
    while the HERK of the current one runs), one with serial_prep; small q share a group."""
    lib = _lib()
    lib.gw_polarization_workspace.restype = ctypes.c_size_t
    lib.gw_polarization_workspace_ex.restype = ctypes.c_size_t
    GW_BF16X3 = 2
    big = lambda n: ((ctypes.c_int64 * n)(*([409600] * n)), (ctypes.c_int * n)(*([600] * n)))
    K0, nb0 = (ctypes.c_int64 * 1)(0), (ctypes.c_int * 1)(1)
    K1, nb1 = big(1)
    K8, nb8 = big(8)
    w0 = lib.gw_polarization_workspace(1, K0, nb0, 16, GW_BF16X3)     # the per-SM scratch
    w1 = lib.gw_polarization_workspace(1, K1, nb1, 16, GW_BF16X3)
    w8 = lib.gw_polarization_workspace(8, K8, nb8, 16, GW_BF16X3)
    assert w1 > w0 > 0 and w8 == w0 + 2 * (w1 - w0)
    serial = _PolOpt(serial_prep=1)
    assert lib.gw_polarization_workspace_ex(8, K8, nb8, 16, GW_BF16X3, ctypes.byref(serial)) == w1
    assert lib.gw_polarization_workspace_ex(1, K1, nb1, 16, GW_BF16X3, ctypes.byref(_PolOpt())) == w1
    # small q: 2 x 2 upper tiles x 16 frequencies = 48 items each, so many share a group
    Ks = (ctypes.c_int64 * 8)(*([1000] * 8))
    nbs = (ctypes.c_int * 8)(*([100] * 8))
    Ks1 = (ctypes.c_int64 * 1)(1000)
    nbs1 = (ctypes.c_int * 1)(100)
    ws8 = lib.gw_polarization_workspace(8, Ks, nbs, 16, GW_BF16X3)
    ws1 = lib.gw_polarization_workspace(1, Ks1, nbs1, 16, GW_BF16X3)
    assert ws8 > ws1


def test_polarization_options_rejected_without_gpu():
    """gw_polarization_ex checks its options before any device call: b_stages must be 0, 4 or
    6, counts must not be negative, event pairs need an array (GW_EINVAL = 1)."""
    lib = _lib()
    lib.gw_last_error.restype = ctypes.c_char_p

    Opt = _PolOpt

    K = (ctypes.c_int64 * 1)(64)
    nb = (ctypes.c_int * 1)(8)
    om = (ctypes.c_double * 2)(0.5, 1.0)
    for fields, word in (({"b_stages": 5}, b"b_stages"), ({"group_items_per_sm": -1}, b"negative"),
                         ({"n_herk_events": 2}, b"herk_events")):
        o = Opt(**fields)
        lib.gw_polarization_ex.restype = ctypes.c_int
        rc = lib.gw_polarization_ex(1, K, nb, None, 1, None, None, ctypes.c_double(1.0), 2, om,
                                    None, 2, ctypes.byref(o), None, ctypes.c_size_t(0), None)
        assert rc == 1 and word in lib.gw_last_error(), (fields, lib.gw_last_error())
    lib.gw_polarization_workspace_ex.restype = ctypes.c_size_t
    assert lib.gw_polarization_workspace_ex(1, K, nb, 2, 2, ctypes.byref(Opt(b_stages=5))) == 0
    assert lib.gw_polarization_workspace_ex(1, K, nb, 2, 2, ctypes.byref(Opt(b_stages=6))) > 0
