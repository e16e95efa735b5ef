"""Failure paths on the GPU without faulting it: a bounded device wait that runs out reports
GW_ETIMEOUT and leaves the context usable; non-finite and out-of-range inputs found on the
device are reported by gw_check."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import polarization as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def dev(a, dt=None):
    return torch.as_tensor(np.asarray(a), device="cuda:0", dtype=dt)


def test_bounded_wait_timeout_then_recovery(gw):
    gw.check()                                       # clean status word
    gw.selftest_bounded_wait(5.0)
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_ETIMEOUT
    gw.check()                                       # the word was cleared
    # the context still computes correctly
    wl = S.tiny(nb=16, nocc=2, nunocc=5, mesh=(2, 1, 1), nw=4, seed=3)
    P = gw.polarization([dev(wl.m_full(0))], [dev(wl.delta(0))], wl.omega(), wl.prefactor, "fp64")[0]
    gw.check()
    ref = OP.polarization(wl.m_full(0), wl.delta(0), wl.omega(), wl.prefactor)
    assert np.allclose(P.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_nonfinite_and_nonpositive_delta_reported(gw):
    wl = S.tiny(nb=16, nocc=2, nunocc=5, mesh=(2, 1, 1), nw=4, seed=4)
    for bad in (np.nan, -0.1, 0.0):
        d = wl.delta(0).copy()
        d[3] = bad
        gw.polarization([dev(wl.m_full(0))], [dev(d)], wl.omega(), wl.prefactor, "fp64")
        with pytest.raises(gw.GWError) as e:
            gw.check()
        assert e.value.code == gw.GW_EINVAL
    gw.check()
