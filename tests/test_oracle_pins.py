"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms derived by hand (residue calculus, Sherman-Morrison),
invariants stated in the paper (Hermiticity on the imaginary axis, negative
semidefinite P), limits, and an independent imaginary-time route.
"""
import os

import numpy as np
import pytest
from scipy.integrate import quad

import synth_inputs as S
from synth_inputs.philox import philox4x32_10
from oracle import polarization as OP
from oracle import screening as OS
from oracle import selfenergy as OE
from oracle import continuation as OC
from oracle import mlp as OM

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- inputs ----
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_inputs_shapes_and_ranges():
    wl = S.small_fp64()
    assert wl.K(0) == 8 * 4 * 28
    d = wl.delta(0)
    assert d.shape == (896,) and d.min() >= 0.05 and d.max() <= 2.5
    om = wl.omega()
    assert np.all(np.diff(om) > 0) and om[0] > 0 and om[-1] < 50
    M = wl.m_full(0)
    sub = wl.m_rows(0, rows=[3, 700], cols=[5, 63])
    assert np.array_equal(sub, M[[3, 700]][:, [5, 63]])
    # column scale 1/(1+I/16): second moment of |M| is 2/(1+I/16)^2
    big = S.tiny(nb=40, nocc=4, nunocc=50, mesh=(2, 2, 2))
    Mb = big.m_full(0)
    m2 = np.mean(np.abs(Mb) ** 2, axis=0) * (1 + np.arange(40) / 16) ** 2
    assert np.all(np.abs(m2 - 2.0) < 0.25)


def test_workload_sizes():
    wl = S.medium_mixed()
    assert wl.K(0) == 409600 and wl.nq == 8 and abs(sum(wl.wq) - 1) < 1e-15
    assert len(wl.sigma_states()) == 16
    b = S.batched_uneven()
    assert all(300 <= n <= 1500 for n in b.nb) and all(200 <= n <= 800 for n in b.nunocc)


# ------------------------------------------------------------ polarization --
def test_bracket_imaginary_time_route():
    """One transition in imaginary time: P(tau) = -exp(-Delta |tau|) per unit weight
    (product of the occupied and unoccupied free propagators); its Fourier transform
    to i omega must equal the bracket of Eq. polar_MB at i omega."""
    for delta in (0.05, 0.7, 2.3):
        for w in (0.0, 0.3, 4.0):
            if w == 0.0:
                ft = 2.0 * quad(lambda t: -np.exp(-delta * t), 0, np.inf,
                                epsabs=1e-14, epsrel=1e-12)[0]
            else:
                ft = 2.0 * quad(lambda t: -np.exp(-delta * t), 0, np.inf, weight="cos",
                                wvar=w, limlst=200)[0]
            b = OP.bracket(np.array([delta]), np.array([w]))[0, 0]
            assert abs(ft - b) <= 1e-9 * abs(b)


def _small_p():
    wl = S.tiny(nb=12, nocc=3, nunocc=5, mesh=(2, 1, 2), nw=5)
    M = wl.m_full(0)
    d = wl.delta(0)
    om = wl.omega()
    return wl, M, d, om, OP.polarization(M, d, om, wl.prefactor)


def test_single_transition_rank_one():
    m = np.array([[0.3 - 1.1j, 2.0 + 0.5j, -0.7j]])
    om = np.array([0.0, 0.5, 9.0])
    P = OP.polarization(m, np.array([0.4]), om, 0.25)
    for j, w in enumerate(om):
        expect = -0.25 * 2 * 0.4 / (0.4 ** 2 + w ** 2) * np.outer(m[0], m[0].conj())
        assert np.allclose(P[j], expect, rtol=1e-14, atol=0)
    # index order of the paper: P_IJ = sum_t w_t M_tI conj(M_tJ)
    assert np.isclose(P[1][0, 1], P[1][0, 0] / abs(m[0, 0]) ** 2 * m[0, 0] * np.conj(m[0, 1]))


def test_p_hermitian_and_negative_semidefinite():
    _, _, _, _, P = _small_p()
    for Pj in P:
        assert np.allclose(Pj, Pj.conj().T, rtol=0, atol=1e-15 * np.abs(Pj).max())
        assert np.all(np.abs(np.diag(Pj).imag) <= 1e-15 * np.abs(Pj).max())
        ev = np.linalg.eigvalsh(Pj)
        assert ev.max() <= 1e-13 * abs(ev).max()


def test_p_high_and_zero_frequency_limits():
    wl, M, d, _, _ = _small_p()
    pref = wl.prefactor
    big = np.array([1e5])
    P = OP.polarization(M, d, big, pref)[0] * big[0] ** 2
    lim = -pref * 2 * (M.T * d[None, :]) @ M.conj()
    assert np.abs(P - lim).max() <= 1e-8 * np.abs(lim).max()
    P0 = OP.polarization(M, d, np.array([0.0]), pref)[0]
    lim0 = -pref * 2 * (M.T / d[None, :]) @ M.conj()
    assert np.abs(P0 - lim0).max() <= 1e-13 * np.abs(lim0).max()


def test_p_time_reversal_additivity_scaling():
    wl, M, d, om, P = _small_p()
    pref = wl.prefactor
    Pc = OP.polarization(M.conj(), d, om, pref)
    assert np.allclose(Pc, P.conj(), rtol=1e-14, atol=0)
    assert np.allclose(Pc, np.transpose(P, (0, 2, 1)), rtol=1e-13, atol=1e-15)
    h = M.shape[0] // 2
    Pa = OP.polarization(M[:h], d[:h], om, pref) + OP.polarization(M[h:], d[h:], om, pref)
    assert np.abs(Pa - P).max() <= 1e-14 * np.abs(P).max()
    c = 0.3 - 1.7j
    assert np.allclose(OP.polarization(c * M, d, om, pref), abs(c) ** 2 * P, rtol=1e-13)


# -------------------------------------------------------------- screening ---
def test_w_single_basis_function():
    P = np.array([[[-0.8 + 0j]], [[-0.01 + 0j]]])
    v = np.array([3.0])
    Wc = OS.screened_wc_all(P, v)
    for j in range(2):
        p = P[j, 0, 0].real
        assert abs(Wc[j, 0, 0] - v[0] ** 2 * p / (1 - v[0] * p)) <= 1e-14 * abs(Wc[j, 0, 0])


def test_w_rank_one_sherman_morrison():
    rng = np.random.default_rng(1)
    n = 9
    m = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = S.coulomb_eigenvalues(n)
    alpha = 0.37
    P = -alpha * np.outer(m, m.conj())
    Wc = OS.screened_wc(P, v)
    vm = v * m
    expect = -alpha * np.outer(vm, vm.conj()) / (1 + alpha * np.real(m.conj() @ (v * m)))
    assert np.abs(Wc - expect).max() <= 1e-13 * np.abs(expect).max()


def test_w_zero_p_and_invariants_and_neumann():
    _, _, _, _, P = _small_p()
    v = S.coulomb_eigenvalues(P.shape[1])
    assert np.all(OS.screened_wc(0 * P[0], v) == 0)
    for Pj in P:
        eps, X = OS.dielectric(Pj, v)
        assert np.linalg.eigvalsh(eps).min() >= 1 - 1e-12
        Wc = OS.screened_wc(Pj, v)
        assert np.allclose(Wc, Wc.conj().T, atol=1e-14 * np.abs(Wc).max())
        assert np.linalg.eigvalsh(Wc).max() <= 1e-12 * np.abs(Wc).max()
    Ps = P[-1] * 1e-6
    V = np.diag(v)
    neu = V @ Ps @ V + V @ Ps @ V @ Ps @ V
    third = V @ Ps @ V @ Ps @ V @ Ps @ V
    Wc = OS.screened_wc(Ps, v)
    assert np.abs(Wc - neu).max() <= 2 * np.abs(third).max() + 1e-15 * np.abs(neu).max()
    assert np.abs(Wc - neu - third).max() <= 0.1 * np.abs(third).max() + 1e-15 * np.abs(neu).max()


# ------------------------------------------------------------ self-energy ---
def _single_pole_closed_form(w, wq, gamma, v, beta, delta, eps_np):
    """Residue calculus on Eq. SEc_AC for N_b = 1, one transition and one pair:
    W^c(i w') = -2 Omega c0 / (w'^2 + Omega^2), Omega^2 = Delta^2 + 2 v beta Delta,
    c0 = v^2 beta Delta / Omega; closing the w' contour away from the pole of the
    Green function gives Sigma(i w) = w_q gamma c0 / (i w - e' - Omega sgn e')."""
    Om = np.sqrt(delta ** 2 + 2.0 * v * beta * delta)
    c0 = v ** 2 * beta * delta / Om
    return wq * gamma * c0 / (1j * np.asarray(w) - eps_np - Om * np.sign(eps_np))


@pytest.mark.parametrize("eps_np", [-0.3, 0.9])
def test_sigma_single_pole_closed_form(eps_np):
    delta, m, pref, v, msig = 0.7, 1.3 - 0.4j, 0.25, 2.0, 0.8 + 0.3j
    wout = np.array([0.05, 1.0, 3.0, 30.0])
    exact = _single_pole_closed_form(wout, 1.0, abs(msig) ** 2, v, pref * abs(m) ** 2,
                                     delta, eps_np)
    errs = []
    for nw in (8, 16, 32, 64):
        om = S.omega_mesh(nw)
        P = OP.polarization(np.array([[m]]), np.array([delta]), om, pref)
        Wc = OS.screened_wc_all(P, np.array([v]))
        c = OE.pair_coefficients(np.array([[msig]]), Wc)
        assert np.all(c <= 0)
        sig = OE.sigma_c(om, wout, [1.0], [c], [np.array([0])], [np.array([eps_np])], 1)[0]
        errs.append(np.abs(sig - exact).max() / np.abs(exact).max())
    assert errs[1] < 1e-4 and errs[3] < 1e-6
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_sigma_conjugation_symmetry_and_linearity():
    om = S.omega_mesh(8)
    wout = np.array([0.2, 1.5, 7.0])
    c = -np.exp(-om / 3.0)
    for e in (-0.2, 0.4):
        Tp = OE.convolution_weights(om, wout, e)
        Tm = OE.convolution_weights(om, -wout, e)
        assert np.allclose(Tm @ c, np.conj(Tp @ c), rtol=1e-11, atol=1e-14)


def test_spline_reproduces_tail_consistent_cubic():
    """A function that is a cubic in lambda with the tail slope at the last node is
    reproduced exactly by the interpolant (not-a-knot + clamped end)."""
    om = S.omega_mesh(10)
    lam = om / (1 + om)
    wn, ln = om[-1], lam[-1]
    # c(l) = a0 + a1 l + a2 l^2 + a3 l^3 with c'(l_N) = -2 c(l_N)/w_N (1+w_N)^2
    a1, a2, a3 = 0.4, -1.1, 0.6
    k = -2.0 / wn * (1 + wn) ** 2
    # solve for a0: a1 + 2 a2 ln + 3 a3 ln^2 = k (a0 + a1 ln + a2 ln^2 + a3 ln^3)
    a0 = (a1 + 2 * a2 * ln + 3 * a3 * ln ** 2) / k - (a1 * ln + a2 * ln ** 2 + a3 * ln ** 3)
    f = lambda l: a0 + a1 * l + a2 * l ** 2 + a3 * l ** 3
    sp = OE.LambdaSpline(om, f(lam))
    x = np.linspace(0, wn, 37)
    assert np.allclose(sp(x), f(x / (1 + x)), rtol=0, atol=1e-12)


# ---------------------------------------------------------- continuation ----
def test_lm_recovers_exact_poles():
    om = S.omega_mesh(24)
    a = np.array([0.31 - 0.05j, 0.12 + 0.02j])
    wp = np.array([-0.9 + 0.15j, -3.2 + 0.4j])
    y = OC.model(a, wp, 1j * om)
    theta0 = OC.pack(a * (1 + 0.05), wp * (1 - 0.04 + 0.02j))
    th, C, it, st = OC.lm_fit(om, y, theta0)
    a2, w2 = OC.unpack(th)
    order = np.argsort(w2.real)[::-1]
    assert st == 0
    assert np.allclose(w2[order], wp, rtol=1e-9, atol=1e-10)
    assert np.allclose(a2[order], a, rtol=1e-9, atol=1e-10)


def test_lm_single_pole_from_default_start():
    om = S.omega_mesh(24)
    a, wp = np.array([0.2 + 0j]), np.array([1.7 - 0.3j])
    y = OC.model(a, wp, 1j * om)
    th, C, it, st = OC.plain_fit(om, y, 1, +1)
    a2, w2 = OC.unpack(th)
    assert np.allclose(w2, wp, rtol=1e-9) and np.allclose(a2, a, rtol=1e-9)


# ------------------------------------------------------------------- MLP ----
def test_mlp_gradients_against_finite_differences():
    rng = np.random.default_rng(0)
    p = OM.init_params(3)
    om = S.omega_mesh(24)
    a = 0.2 * (rng.normal(size=(4, 2)) + 1j * rng.normal(size=(4, 2)))
    wp = rng.normal(size=(4, 2)) * 2 - 0.3j
    y = np.stack([OC.model(a[b], wp[b], 1j * om) for b in range(4)])
    L, g = OM.loss_and_grads(p, om, y)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=4, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = OM.loss_and_grads(p, om, y)
            flat[idx] = old - h
            Lm, _ = OM.loss_and_grads(p, om, y)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * abs(L)) + 1e-11, (name, idx, fd, an)


def test_bf16_rounding_matches_torch_and_packing_round_trips():
    """The BF16 emulation of the inference reference agrees with torch's own BF16
    conversion (round to nearest, ties to even), including exact ties; the packed layout
    round-trips."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    a = (rng.normal(size=4000) * 10.0 ** rng.uniform(-3, 3, size=4000)).astype(np.float32)
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)   # exact ties
    a = np.concatenate([a, ties, -ties])
    got = OM.bf16_round(a)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, ref)
    p = OM.init_params(3)
    q = OM.unpack(OM.pack(p))
    assert all(np.array_equal(p[k], q[k]) for k in OM.ORDER)
    assert OM.pack(p).size == 128 * 48 + 128 + 128 * 128 + 128 + 8 * 128 + 8


def test_tf32_rounding_rule_by_bits_matches_definition():
    """The split-precision kernel rounds FP32 to TF32 by (bits + 0x1000) & 0xFFFFE000. Checked
    here against the definition (nearest TF32 value, ties away from zero), computed exactly
    with rationals, on random values, exact ties and values next to powers of two."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    x = (rng.normal(size=2000) * 10.0 ** rng.uniform(-20, 20, size=2000)).astype(np.float32)
    b = x.view(np.uint32)
    ties = ((b & np.uint32(0xFFFFE000)) | np.uint32(0x1000)).view(np.float32)
    below2 = np.nextafter(np.float32(2.0) ** np.arange(-10, 10, dtype=np.float32), np.float32(0))
    vals = np.concatenate([x, ties, below2, -ties])
    got = ((vals.view(np.uint32).astype(np.uint64) + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)
    for v, g in zip(vals, got):
        f = Fraction(float(v))
        e = np.frexp(np.float32(abs(v)))[1]          # |v| in [2^(e-1), 2^e)
        ulp = Fraction(2) ** (int(e) - 1 - 10)       # TF32 spacing there
        q = abs(f) / ulp
        n = int(q)
        if q - n >= Fraction(1, 2):
            n += 1
        ref = n * ulp * (1 if f >= 0 else -1)
        assert Fraction(float(g)) == ref, (v, g, float(ref))


def test_qp_newton_single_real_pole_closed_form():
    """One pole with real residue a and real position w: E - c - a/(E - w) = 0 is the quadratic
    (E - c)(E - w) = a, roots (c + w +- sqrt((c - w)^2 + 4a)) / 2; Newton from eps lands on the
    root on eps's side of the pole; Z = 1 / (1 + a/(E - w)^2)."""
    from oracle import qp as OQ
    cases = [(-0.3, 0.1, 0.05, -1.2, 0.02), (0.4, -0.2, 0.1, 1.5, -0.03), (0.2, 0.0, 0.0, 2.0, 0.3)]
    for eps, sx, vxc, w, a in cases:
        c = eps + sx - vxc
        disc = np.sqrt((c - w) ** 2 + 4 * a)
        roots = np.array([(c + w + disc) / 2, (c + w - disc) / 2])
        want = roots[np.argmin(np.abs(roots - eps))]
        prm = np.array([[[a, 0.0, w, 0.0]]])
        E, Z, st = OQ.qp_solve(prm, [eps], [sx], [vxc])
        assert st[0] == 0
        assert abs(E[0] - want) <= 1e-13 * max(1, abs(want))
        assert np.isclose(Z[0], 1.0 / (1.0 + a / (want - w) ** 2), rtol=1e-12)
    # no self-energy: E = eps + Sigma_x - v_xc, Z = 1
    E, Z, _ = OQ.qp_solve(np.zeros((1, 2, 4)) + np.array([0, 0, 3.0, -1.0]), [0.3], [-0.5], [-0.4])
    assert abs(E[0] - 0.2) <= 1e-15 and abs(Z[0] - 1.0) <= 1e-15


def test_adam_two_steps_by_hand():
    """Adam (Kingma & Ba 2015, Algorithm 1) worked by hand on two parameters. With
    m_0 = v_0 = 0 the bias corrections give, after step 1, m^ = g_1 and v^ = g_1^2, so the
    update is lr g_1 / (|g_1| + eps); after step 2,
    m^ = (b1 (1 - b1) g_1 + (1 - b1) g_2) / (1 - b1^2) = (b1 g_1 + g_2) / (1 + b1) and
    v^ = (b2 g_1^2 + g_2^2) / (1 + b2). With g_1 = (0.5, -2), g_2 = (1, 4), lr = 0.1,
    b1 = 0.9, b2 = 0.999, eps = 1e-8 the second update of the first parameter is
    0.1 * (1.45 / 1.9) / (sqrt(1.249750 / 1.999) + 1e-8)."""
    lr, eps = 0.1, 1e-8
    p = {"w": np.array([1.0, -3.0])}
    st = {}
    g1 = {"w": np.array([0.5, -2.0])}
    g2 = {"w": np.array([1.0, 4.0])}
    p = OM.adam_step(p, g1, st, lr, 1)
    step1 = lr * g1["w"] / (np.abs(g1["w"]) + eps)
    assert np.allclose(p["w"], np.array([1.0, -3.0]) - step1, rtol=0, atol=1e-15)
    p = OM.adam_step(p, g2, st, lr, 2)
    mh = (0.9 * g1["w"] + g2["w"]) / 1.9
    vh = (0.999 * g1["w"] ** 2 + g2["w"] ** 2) / 1.999
    step2 = lr * mh / (np.sqrt(vh) + eps)
    assert np.allclose(p["w"], np.array([1.0, -3.0]) - step1 - step2, rtol=0, atol=1e-15)
    # the first parameter by hand: 1 - 0.0999999980 - 0.0965184...
    assert abs(p["w"][0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8)
                            - 0.1 * (1.45 / 1.9) / (np.sqrt(1.24975 / 1.999) + 1e-8))) <= 1e-15
    # a constant gradient: every bias-corrected step is exactly lr g / (|g| + eps)
    q, st2 = {"w": np.array([0.0])}, {}
    for t in range(1, 6):
        q = OM.adam_step(q, {"w": np.array([0.25])}, st2, lr, t)
    assert abs(q["w"][0] + 5 * lr * 0.25 / (0.25 + eps)) <= 1e-14


def test_mlp_loss_reading_by_construction():
    """The loss of the learned start against curves built from known parameters: a network
    whose last layer is zero outputs its bias o, read as a_p = s (o_4p + i o_4p+1),
    w_p = o_4p+2 + i o_4p+3 with s = max_j |y_j|. A curve that is exactly that two-pole
    function has loss 0; the same curve shifted by a constant c has loss |c|^2 / s^2 (the
    residual is -c at each of the 24 nodes, averaged over the nodes)."""
    om = S.omega_mesh(24)
    a = np.array([0.3 - 0.05j, 0.12 + 0.02j])
    wp = np.array([0.8 - 0.1j, 3.1 - 0.4j])
    y = OC.model(a, wp, 1j * om)
    s = np.abs(y).max()
    o = np.array([a[0].real / s, a[0].imag / s, wp[0].real, wp[0].imag,
                  a[1].real / s, a[1].imag / s, wp[1].real, wp[1].imag])
    p = OM.init_params(1)
    p["W3"][:] = 0.0
    p["b3"][:] = o
    L0, _ = OM.loss_and_grads(p, om, y[None, :])
    assert L0 <= 1e-30
    c = 0.02 + 0.01j
    yc = y + c
    sc = np.abs(yc).max()
    p["b3"][:] = o * np.array([s / sc, s / sc, 1, 1, s / sc, s / sc, 1, 1])
    L1, _ = OM.loss_and_grads(p, om, yc[None, :])
    assert abs(L1 - abs(c) ** 2 / sc ** 2) <= 1e-15
    # the features are the curve over s, interleaved (Re y_0, Im y_0, Re y_1, ...)
    x, s2 = OM.features(yc[None, :])
    assert s2[0] == sc and x[0, 0] == yc[0].real / sc and x[0, 3] == yc[1].imag / sc
