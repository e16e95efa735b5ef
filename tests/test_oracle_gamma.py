"""Pins of the q = Gamma oracle (Sec. III.D): the head/wing/body formulas against a
brute-force inverse of the full (N_b+1)-dimensional dielectric problem at finite k, the
angular averages against closed forms and identities, the BZ constant's erf form
against its definition, and the divergent Sigma^c term against the single-pole closed
form of the frequency integral."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import gamma as OG
from oracle import polarization as OP

FOUR_PI = 4.0 * np.pi


def _case(nb=6, K=24, nw=3, seed=5):
    rng = np.random.default_rng(seed)
    M = (rng.normal(size=(K, nb)) + 1j * rng.normal(size=(K, nb))) / (1 + np.arange(nb) / 4)
    p = 0.3 * (rng.normal(size=(K, 3)) + 1j * rng.normal(size=(K, 3)))
    delta = rng.uniform(0.1, 1.5, size=K)
    om = S.omega_mesh(nw)
    v = S.coulomb_eigenvalues(nb)
    return M, p, delta, om, v


def test_head_wing_body_match_brute_force_inverse():
    M, p, delta, om, v = _case()
    pref = 0.25
    Paug = OP.polarization(np.concatenate([p, M], axis=1), delta, om, pref)
    H, Sv, Pt = OG.split_augmented(Paug)
    from oracle import screening as OS
    Wtc = OS.screened_wc_all(Pt, v)
    rng = np.random.default_rng(1)
    for j in range(len(om)):
        u, L = OG.head_wing_terms(H[j], Sv[j], Wtc[j], v)
        assert np.allclose(L, L.conj().T, atol=1e-13)
        Wt = Wtc[j] + np.diag(v)
        for k in (0.4, 1e-3):
            e = rng.normal(size=3)
            e /= np.linalg.norm(e)
            # the full problem from the transitions themselves: m_t(k) = [k e.p_t, M_t]
            Mk = np.concatenate([(k * (p @ e))[:, None], M], axis=1)
            Pfull = OP.polarization(Mk, delta, om[j:j + 1], pref)[0]
            W = OG.full_w_at_k(Pfull, v, k)
            sig = float(np.real(e @ L @ e))
            assert sig > 0
            assert np.isclose(W[0, 0] * k * k / FOUR_PI, 1.0 / sig, rtol=1e-10)
            eu = u @ e
            assert np.allclose(W[0, 1:] * k, FOUR_PI * eu / sig, rtol=1e-9, atol=1e-12)
            assert np.allclose(W[1:, 0] * k, FOUR_PI * eu.conj() / sig, rtol=1e-9, atol=1e-12)
            body = Wt + FOUR_PI * np.outer(eu.conj(), eu) / sig
            assert np.allclose(W[1:, 1:], body, rtol=1e-9, atol=1e-10 * np.abs(body).max())


def test_angular_moments_closed_forms_and_identities():
    lam = 2.5
    inv, A = OG.angular_moments(lam * np.eye(3))
    assert np.isclose(inv, 1.0 / lam, rtol=1e-12)
    assert np.allclose(A, np.eye(3) / (3 * lam), atol=1e-13)
    a, b = 3.0, 1.2                        # spheroid: L = diag(b, b, a)
    inv, A = OG.angular_moments(np.diag([b, b, a]))
    ref = np.arctan(np.sqrt((a - b) / b)) / np.sqrt(b * (a - b))
    assert np.isclose(inv, ref, rtol=1e-12)
    assert np.isclose(A[2, 2], (1.0 - b * ref) / (a - b), rtol=1e-11)
    # any Hermitian positive definite L: trace A = <1/e^T L e>, sum_ab L_ab A_ab = 1
    rng = np.random.default_rng(3)
    X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    L = np.eye(3) * 2 + 0.3 * (X @ X.conj().T)
    inv, A = OG.angular_moments(L)
    assert np.isclose(np.trace(A), inv, rtol=1e-11)
    assert np.isclose(np.sum(np.real(L) * A), 1.0, rtol=1e-11)


@pytest.mark.parametrize("n", [2, 3])
def test_bz_constant_erf_form(n):
    """The erf form with the cutoff exp(-beta q0^2) = beta against the cutoff-free
    Gaussian form (closed-form integral over all reciprocal space minus the lattice sum
    to e^-16), its independence of beta (the terms it neglects are of order beta), and
    the exact homogeneity C(lambda a, lambda^2 beta) = lambda^2 C(a, beta) of the Gaussian
    form, for a simple-cubic lattice."""
    a = 10.26
    c = OG.bz_constant_sc(a, n, beta=0.005)
    c_gauss = OG.bz_constant_sc_gauss(a, n, beta=0.005)
    c_beta = OG.bz_constant_sc(a, n, beta=0.002)
    assert abs(c - c_gauss) <= 1e-4 * abs(c), (c, c_gauss)
    assert abs(c - c_beta) <= 2e-4 * abs(c), (c, c_beta)
    c2 = OG.bz_constant_sc_gauss(2 * a, n, beta=0.005 * 4)
    assert np.isclose(c2, 4 * c_gauss, rtol=1e-10)


def test_sigma_div_single_pole_closed_form():
    """K^c_00(w') = -2 W c0 / (w'^2 + W^2) has int dw' K / (i w + i w' - e) =
    -2 pi c0 / (i w - e - W sgn e) (residues), so the divergent term is
    C c0 / (2 sqrt(pi) V (i w - e - W sgn e)); the spline-and-tail integral approaches it as
    the mesh is refined."""
    Om, c0, cbz, vol = 0.8, 0.7, 13.0, 1000.0
    eps = np.array([-0.3, 0.4])
    errs = []
    for nw in (16, 48):
        om = S.omega_mesh(nw)
        K = -2.0 * Om * c0 / (om ** 2 + Om ** 2)
        got = OG.sigma_div(om, om, K, cbz, vol, eps)
        ref = cbz * c0 / (2 * np.sqrt(np.pi) * vol) / (
            1j * om[None, :] - eps[:, None] - Om * np.sign(eps)[:, None])
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    assert errs[1] < errs[0] and errs[1] < 2e-3, errs


def test_exchange_oracle_pins():
    """Eq. HFterm_MB in the eigenbasis: a pair with one nonzero projection component gives
    -w v_mu |m_mu|^2; unoccupied n' and the divergent term of an unoccupied state vanish;
    the divergent term of an occupied state is -(4 pi / V) C; scaling M by c scales the
    regular part by |c|^2."""
    from oracle import exchange as OX
    v = np.array([3.0, 2.0, 0.5])
    M = np.zeros((3, 3), dtype=np.complex128)
    M[0, 1] = 0.3 - 0.4j                     # |m|^2 = 0.25 on mu = 1
    M[1, 2] = 2.0j                           # unoccupied partner: excluded
    M[2, 0] = 1.0                            # state 1, occupied partner
    eps = np.array([-0.2, 0.7, -1.0])
    st = np.array([0, 0, 1])
    got = OX.sigma_x([0.5], [M], [st], [eps], [v], 2, np.array([0.3, 0.4]), 10.0, 100.0)
    assert np.allclose(got, [-0.5 * 2.0 * 0.25, -0.5 * 3.0 * 1.0], rtol=1e-15)
    div = OX.sigma_x([0.5], [np.zeros((3, 3))], [st], [eps], [v], 2, np.array([-0.3, 0.4]), 10.0, 100.0)
    assert np.allclose(div, [-FOUR_PI / 100.0 * 10.0, 0.0], rtol=1e-15)
    s2 = OX.sigma_x([0.5], [(1 - 2j) * M], [st], [eps], [v], 2, np.array([0.3, 0.4]), 10.0, 100.0)
    assert np.allclose(s2, 5.0 * got, rtol=1e-14)
