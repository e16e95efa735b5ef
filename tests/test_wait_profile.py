"""The HERK wait counters (gw_herk_wait_profile): the normal library refuses them without a GPU
call, the counter list of the binding is the header's, and on a GPU the profiling build counts
every role of a small split-precision polarization while still computing it correctly. The MMA
issue probe (gw_probe_mma_issue) checks its arguments before any device call and, on a GPU,
reports rates no faster than the tensor pipe."""
import ctypes
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _builder():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gw_build", os.path.join(ROOT, "paper_1003_0316_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_counter_list_matches_header():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    n = int(re.search(r"#define GW_HERK_WAIT_COUNTERS (\d+)", src).group(1))
    binding = open(os.path.join(ROOT, "paper_1003_0316_gb300", "__init__.py")).read()
    names = re.search(r"HERK_WAIT_COUNTERS = \((.*?)\)\n", binding, flags=re.S).group(1)
    assert len(re.findall(r'"(\w+)"', names)) == n
    # the header numbers the counters 0 .. n - 1 in its comment
    block = src[src.index("in this order:"):src.index("gw_herk_wait_profile synchronises")]
    assert sorted(int(k) for k in re.findall(r"(?<![\w.])(\d+) [A-Za-z]", block)) == list(range(n))


def test_normal_build_refuses_without_device_call():
    lib = ctypes.CDLL(_builder().build())
    lib.gw_herk_wait_profile.restype = ctypes.c_int
    lib.gw_last_error.restype = ctypes.c_char_p
    c = (ctypes.c_ulonglong * 18)()
    assert lib.gw_herk_wait_profile(c, 18, 1) == 8          # GW_EUNSUPPORTED
    assert b"GW_HERK_WAIT_PROFILE" in lib.gw_last_error()


def test_mma_probe_rejects_bad_arguments_without_gpu():
    lib = ctypes.CDLL(_builder().build())
    lib.gw_probe_mma_issue.restype = ctypes.c_int
    out = ctypes.c_double(0.0)
    assert lib.gw_probe_mma_issue(6, 100, ctypes.byref(out), None) == 1
    assert lib.gw_probe_mma_issue(0, 1, ctypes.byref(out), None) == 1
    assert lib.gw_probe_mma_issue(0, 100, None, None) == 1


@pytest.mark.gpu
def test_mma_probe_rates():
    import paper_1003_0316_gb300 as gw
    alone = gw.probe_mma_issue(0, 200)
    rates = [gw.probe_mma_issue(v, 200) for v in range(len(gw.MMA_ISSUE_VARIANTS))]
    gw.check()
    # 64 cycles per MMA is the pipe's rate (8192 flop per cycle and SM); nothing runs faster
    assert 58.0 <= alone <= 80.0, alone
    assert all(58.0 <= r < 5000.0 for r in rates), rates


_CHILD = r"""
import json, numpy as np, torch
import paper_1003_0316_gb300 as gw
import synth_inputs as S
from oracle import polarization as OP
assert gw.lib_path().endswith("libgw_prof.so")
wl = S.tiny(nb=150, nocc=4, nunocc=40, mesh=(2, 2, 2), nw=8)
M = wl.m_full(0).astype(np.complex64)
d = wl.delta(0)
om = wl.omega()
dev = torch.device("cuda:0")
gw.herk_wait_profile(reset=True)
P = gw.polarization([torch.as_tensor(M, device=dev)], [torch.as_tensor(d, device=dev)], om,
                    wl.prefactor, "bf16x3")[0]
gw.check()
prof = gw.herk_wait_profile(reset=True)
again = gw.herk_wait_profile(reset=False)
ref = OP.polarization(M.astype(np.complex128), d, om, wl.prefactor)
err = float(np.linalg.norm(P.cpu().numpy() - ref) / np.linalg.norm(ref))
print(json.dumps({"prof": prof, "again": again, "err": err, "K": int(M.shape[0])}))
"""


@pytest.mark.gpu
def test_profiling_build_counts_every_role():
    _builder().build(variant="prof")
    env = dict(os.environ, GW_LIBRARY="prof", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    p = out["prof"]
    assert out["err"] < 1e-6
    # the reset zeroed the counters
    assert all(v == 0 for k, v in out["again"].items() if isinstance(v, int))
    for role in ("a", "mma", "epi", "bprod", "wprod"):
        assert p[f"{role}_total"] > 0, role
    # rounds: every A set and MMA issuer round of every item; one drain period per round
    assert p["a_rounds"] == 4 * p["mma_rounds"] and p["mma_rounds"] > 0
    assert p["epi_periods"] == 4 * p["mma_rounds"]
    for k, f in p["fractions"].items():
        assert f is not None and 0.0 <= f <= 1.0, (k, f)
