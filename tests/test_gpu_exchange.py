"""Exchange self-energy on the GPU against the oracle (FP64 and complex64 projections)."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import exchange as OX
from oracle import gamma as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def dev(a, dt=None):
    return torch.as_tensor(np.asarray(a), device="cuda:0", dtype=dt)


@pytest.mark.parametrize("cdt", [np.complex128, np.complex64])
def test_sigma_x_against_oracle(gw, cdt):
    wl = S.tiny(nb=37, nocc=4, nunocc=11, mesh=(2, 2, 1), nw=4, seed=55, qs=(0, 1, 3))
    Ms = [wl.msig_rows(i).astype(cdt) for i in range(wl.nq)]
    ps, es = zip(*[wl.sigma_pairs(i) for i in range(wl.nq)])
    vs = [wl.v(i) for i in range(wl.nq)]
    est = wl.state_energies()
    nsig = len(wl.sigma_states())
    cbz, vol = OG.bz_constant_sc(10.26, 2), (2 * 10.26) ** 3
    got = gw.sigma_x(list(wl.wq), [dev(m) for m in Ms], [dev(p, torch.int32) for p in ps],
                     [dev(e) for e in es], [dev(v) for v in vs], nsig, dev(est), cbz, vol)
    gw.check()
    ref = OX.sigma_x(list(wl.wq), [m.astype(np.complex128) for m in Ms], ps, es, vs, nsig, est,
                     cbz, vol)
    assert np.allclose(got.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert np.all(got.cpu().numpy() <= 0)
