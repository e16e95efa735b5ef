"""The no-allocation variant of the screened-interaction step.

gw_screened_w_noalloc serves callers that cannot allocate device memory at call time
(a host application that owns all device memory through its own pool, or a loop where
cudaMalloc's possible device synchronisation is unacceptable): its scratch is a static
device array inside the library. This test calls it through the C ABI twice in a row and
checks both results against gw_screened_w (the entry point that takes caller workspace),
with the FP64-path tolerance of the other tests, and checks that a basis too large for the
static scratch is rejected before any work. It lives in its own file, collected last, so a
failure here cannot hide the results of the other tests.
"""
import numpy as np
import pytest

import synth_inputs as S
from oracle import polarization as OP
from oracle import screening as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nb,nw", [(48, 5), (600, 5)])
def test_noalloc_matches_workspace_entry_point(gw, nb, nw):
    wl = S.tiny(nb=nb, nocc=4, nunocc=25, mesh=(2, 2, 2), nw=nw, seed=31 + nb)
    dev = torch.device("cuda:0")
    M = torch.as_tensor(wl.m_full(0), device=dev)
    d = torch.as_tensor(wl.delta(0), device=dev)
    v = torch.as_tensor(wl.v(0), device=dev)
    P = gw.polarization([M], [d], wl.omega(), wl.prefactor, "fp64")[0]
    ref = gw.screened_w([P], [v])[0]
    gw.check()
    ref = ref.cpu().numpy()
    for _ in range(2):                      # two calls in a row share the static scratch
        out = gw.screened_w_noalloc(P, v)
        gw.check()
        got = out.cpu().numpy()
        assert rel_fro(got, ref) <= 1e-12
        assert max_rel(got, ref) <= 1e-12


@pytest.mark.parametrize("nb", [97, 600])
def test_noalloc_against_oracle(gw, nb):
    """The no-allocation entry point (whose inverse runs inside one CTA per system) directly
    against the FP64 oracle, on a polarization the oracle computed itself."""
    wl = S.tiny(nb=nb, nocc=4, nunocc=30, mesh=(2, 2, 2), nw=3, seed=nb + 17)
    om = wl.omega()
    Po = OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor)
    v = wl.v(0)
    dev = torch.device("cuda:0")
    out = gw.screened_w_noalloc(torch.as_tensor(Po, device=dev), torch.as_tensor(v, device=dev))
    gw.check()
    got = out.cpu().numpy()
    ref = OS.screened_wc_all(Po, v)
    assert rel_fro(got, ref) <= 1e-12
    assert max_rel(got, ref) <= 1e-12


def test_noalloc_rejects_basis_beyond_static_scratch(gw):
    nb = 1100
    dev = torch.device("cuda:0")
    P = torch.zeros((1, nb, nb), dtype=torch.complex128, device=dev)
    v = torch.ones(nb, dtype=torch.float64, device=dev)
    with pytest.raises(gw.GWError) as e:
        gw.screened_w_noalloc(P, v)
    assert e.value.code == gw.GW_EINVAL
    assert "static scratch" in str(e.value)
