"""q = Gamma head and wings on the GPU against the oracle: the augmented polarization
(three k.p columns), the body with its l = 0 rank-one average, the head coefficient
K^c_00, L and u; the BZ constant's lattice sum; and the divergent Sigma^c term."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import gamma as OG
from oracle import polarization as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def dev(a, dt=None):
    return torch.as_tensor(np.asarray(a), device="cuda:0", dtype=dt)


def augmented_case(nb=40, nocc=3, nunocc=20, nw=6, seed=21):
    """Projections of a small mesh workload plus three seeded k.p columns per transition
    (complex normals scaled by 0.3, drawn like the projections)."""
    wl = S.tiny(nb=nb, nocc=nocc, nunocc=nunocc, mesh=(2, 2, 1), nw=nw, seed=seed)
    M = wl.m_full(0)
    K = M.shape[0]
    p = 0.3 * S.complex_normals(seed, S.TID_KP, np.arange(3 * K), 0).reshape(K, 3)
    return wl, np.concatenate([p, M], axis=1)


@pytest.mark.parametrize("nb", [40, 37])
def test_gamma_head_wings_body(gw, nb):
    wl, Ma = augmented_case(nb=nb)
    om = wl.omega()
    v = S.coulomb_eigenvalues(nb)
    Paug = gw.polarization([dev(Ma)], [dev(wl.delta(0))], om, wl.prefactor, "fp64")[0]
    Wc, head, L, u = gw.gamma_screened_w(Paug, dev(v))
    gw.check()
    Pa = OP.polarization(Ma, wl.delta(0), om, wl.prefactor)
    K00c, Lr, ur, body = OG.gamma_all(Pa, v)
    assert np.allclose(L.cpu().numpy(), Lr, rtol=1e-11, atol=1e-11 * np.abs(Lr).max())
    assert np.allclose(u.cpu().numpy(), ur, rtol=1e-10, atol=1e-11 * np.abs(ur).max())
    # the sphere rule (64 x 128 nodes) against adaptive quadrature
    assert np.allclose(head.cpu().numpy(), K00c, rtol=1e-10, atol=1e-10 * np.abs(K00c).max())
    b = Wc.cpu().numpy()
    assert np.linalg.norm(b - body) <= 1e-10 * np.linalg.norm(body)
    assert np.allclose(b, np.conj(np.transpose(b, (0, 2, 1))), atol=1e-10 * np.abs(b).max())


@pytest.mark.parametrize("n", [2, 3])
def test_bz_constant_lattice_sum(gw, n):
    a = 10.26
    c = gw.bz_constant_sc(a, n, beta=0.005)
    ref = OG.bz_constant_sc(a, n, beta=0.005)
    assert abs(c - ref) <= 1e-9 * abs(ref), (c, ref)


def test_sigma_div_against_oracle(gw):
    om = S.omega_mesh(16)
    rng = np.random.default_rng(2)
    K = -2.0 * 0.9 * 0.5 / (om ** 2 + 0.81) * (1 + 0.1 * rng.uniform(size=len(om)))
    eps = np.array([-0.4, -0.1, 0.2, 0.9])
    cbz, vol = 95.06, 8640.0
    base = rng.normal(size=(len(eps), len(om))) + 1j * rng.normal(size=(len(eps), len(om)))
    sig = dev(base.copy())
    gw.sigma_div(om, dev(K), cbz, vol, dev(eps), om, sig)
    gw.check()
    ref = base + OG.sigma_div(om, om, K, cbz, vol, eps)
    assert np.abs(sig.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref - base).max()
