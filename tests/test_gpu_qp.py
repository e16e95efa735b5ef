"""Quasiparticle energies on the GPU against the oracle, from fitted self-energy curves."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import qp as OQ

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def test_qp_against_oracle(gw):
    om = S.omega_mesh(24)
    y, sg = S.model_sigma_curves(S.SEED_BASE + 106, 300, om)
    Y = torch.as_tensor(y, device="cuda")
    prm, cost, it, st = gw.continue_fit(Y, om, npole=2, sign=torch.as_tensor(sg, device="cuda"))
    gw.check()
    rng = np.random.default_rng(6)
    eps = np.where(sg < 0, -rng.uniform(0.0, 0.5, 300), rng.uniform(0.05, 2.0, 300))
    sigx = np.where(sg < 0, -rng.uniform(0.3, 1.0, 300), -rng.uniform(0.0, 0.2, 300))
    vxc = -rng.uniform(0.2, 0.8, 300)
    T = lambda a: torch.as_tensor(a, device="cuda")
    E, Z, qst = gw.qp_solve(prm, T(eps), T(sigx), T(vxc))
    gw.check()
    Er, Zr, str_ = OQ.qp_solve(prm.cpu().numpy(), eps, sigx, vxc)
    ok = str_ == 0
    assert ok.mean() > 0.9
    assert np.array_equal(qst.cpu().numpy()[ok], str_[ok])
    assert np.allclose(E.cpu().numpy()[ok], Er[ok], rtol=1e-12, atol=1e-13)
    assert np.allclose(Z.cpu().numpy()[ok], Zr[ok], rtol=1e-10, atol=1e-12)
