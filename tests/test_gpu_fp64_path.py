"""GPU parity of the FP64 path against the CPU oracle, element by element.

Tolerances (FP64 path): relative Frobenius error <= 1e-12 and max-abs error <= 1e-12 of
the largest entry for P and W^c; Sigma^c within 1e-11 of its largest entry (the oracle
integrates by adaptive quadrature to ~1e-13); the LM fit recovers exact poles to 1e-9.
"""
import numpy as np
import pytest

import synth_inputs as S
from oracle import polarization as OP
from oracle import screening as OS
from oracle import selfenergy as OE
from oracle import continuation as OC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def dev():
    return torch.device("cuda:0")


def T(a, dt=None):
    return torch.as_tensor(np.asarray(a), device=dev(), dtype=dt)


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_device_generator_matches_host_generator(gw):
    wl = S.tiny(nb=37, nocc=3, nunocc=11, mesh=(2, 2, 1))
    host = wl.m_full(0)
    g = gw.synth_projections(wl.seed, S.TID_M, wl.qs[0], 0, wl.K(0), 37, dtype=torch.complex128)
    assert np.allclose(g.cpu().numpy(), host, rtol=4e-16, atol=1e-300)
    rows = [5, 100]
    sub = gw.synth_projections(wl.seed, S.TID_M, wl.qs[0], 5, 96, 37, dtype=torch.complex64)
    assert np.allclose(sub.cpu().numpy()[[0, 95]], host[rows].astype(np.complex64), rtol=1e-7)


def test_weights(gw):
    wl = S.small_fp64()
    d = wl.delta(0)
    om = wl.omega()
    f = np.linspace(0.5, 1.5, len(d))
    w = gw.transition_weights(T(d), om, wl.prefactor, T(f)).cpu().numpy()
    ref = OP.transition_weights(d, om, wl.prefactor, f)
    assert max_rel(w, ref) <= 1e-15


@pytest.mark.parametrize("case", ["small", "ragged_batch"])
def test_polarization_fp64(gw, case):
    if case == "small":
        wls = [S.small_fp64()]
    else:
        wls = [S.tiny(nb=150, nocc=5, nunocc=41, mesh=(2, 2, 3), nw=7, seed=77),
               S.tiny(nb=33, nocc=2, nunocc=9, mesh=(1, 1, 1), nw=7, seed=78)]
    om = wls[0].omega()
    Ms = [w.m_full(0) for w in wls]
    ds = [w.delta(0) for w in wls]
    pref = 2.0 / 12
    P = gw.polarization([T(m) for m in Ms], [T(d) for d in ds], om, pref, "fp64")
    for M, d, Pg in zip(Ms, ds, P):
        ref = OP.polarization(M, d, om, pref)
        Pg = Pg.cpu().numpy()
        assert rel_fro(Pg, ref) <= 1e-12
        assert max_rel(Pg, ref) <= 1e-12
        # exactly Hermitian with a real diagonal
        assert np.array_equal(Pg, np.conj(np.transpose(Pg, (0, 2, 1))))


def test_polarization_empty_and_symmetry_weights(gw):
    wl = S.tiny(nb=20, nocc=2, nunocc=4, mesh=(1, 1, 2), nw=5)
    om = wl.omega()
    M = wl.m_full(0)
    d = wl.delta(0)
    f = np.full(len(d), 0.25)
    P0 = gw.polarization([T(M[:0])], [T(d[:0])], om, 1.0, "fp64")[0]
    assert torch.count_nonzero(P0) == 0
    Pf = gw.polarization([T(M)], [T(d)], om, 1.0, "fp64", fs=[T(f)])[0].cpu().numpy()
    assert max_rel(Pf, OP.polarization(M, d, om, 1.0, f)) <= 1e-12


def test_polarization_rejects_bad_delta(gw):
    wl = S.tiny(nb=8)
    om = wl.omega()
    d = wl.delta(0).copy()
    d[1] = -0.1
    gw.polarization([T(wl.m_full(0))], [T(d)], om, 1.0, "fp64")
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_EINVAL


def test_argument_errors(gw):
    wl = S.tiny(nb=8)
    M = T(wl.m_full(0))
    d = T(wl.delta(0))
    with pytest.raises(gw.GWError) as e:
        gw.polarization([M], [d], wl.omega(), 1.0, "tf32x3")
    assert e.value.code == gw.GW_EUNSUPPORTED
    with pytest.raises(gw.GWError) as e:
        gw.polarization([M], [d], np.zeros(65), 1.0, "fp64")
    assert e.value.code == gw.GW_EINVAL
    with pytest.raises(gw.GWError) as e:
        gw.polarization([M], [d], wl.omega(), 1.0, "fp64", ws=torch.empty(16, dtype=torch.uint8,
                                                                          device=dev()))
    assert e.value.code == gw.GW_EWORKSPACE


@pytest.mark.parametrize("nb", [64, 150])
def test_screened_w_fp64_stagewise(gw, nb):
    wl = S.tiny(nb=nb, nocc=4, nunocc=30, mesh=(2, 2, 2), nw=6, seed=nb)
    om = wl.omega()
    Po = OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor)
    v = wl.v(0)
    Wg = gw.screened_w([T(Po)], [T(v)])[0]
    gw.check()
    Wg = Wg.cpu().numpy()
    ref = OS.screened_wc_all(Po, v)
    assert rel_fro(Wg, ref) <= 1e-12
    assert max_rel(Wg, ref) <= 1e-12
    assert np.array_equal(Wg, np.conj(np.transpose(Wg, (0, 2, 1))))


def test_screened_w_in_place_and_not_hpd(gw):
    wl = S.tiny(nb=40, nocc=3, nunocc=10, mesh=(2, 1, 2), nw=4)
    om = wl.omega()
    Po = OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor)
    v = wl.v(0)
    P = T(Po)
    gw.screened_w([P], [T(v)], out=[P])
    gw.check()
    assert max_rel(P.cpu().numpy(), OS.screened_wc_all(Po, v)) <= 1e-12
    bad = T(-Po)        # positive semidefinite P: eps not positive definite
    gw.screened_w([bad], [T(v)])
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_ENOTHPD


def test_pair_coefficients_fp64(gw):
    wl = S.tiny(nb=70, nocc=3, nunocc=20, mesh=(2, 1, 2), nw=5, seed=5)
    om = wl.omega()
    Wo = OS.screened_wc_all(OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor), wl.v(0))
    Ms = wl.msig_rows(0)
    c = gw.sigma_pair_coeffs([T(Ms)], [T(Wo)])[0].cpu().numpy()
    ref = OE.pair_coefficients(Ms, Wo)
    assert max_rel(c, ref) <= 1e-12
    assert np.all(c <= 0)


@pytest.mark.parametrize("nw", [6, 16])
def test_convolution_stagewise(gw, nw):
    rng = np.random.default_rng(nw)
    om = S.omega_mesh(nw)
    om_out = np.concatenate([S.omega_mesh(5), [-0.7, 80.0]])
    npair, nsig = 40, 3
    c = -np.exp(-om[:, None] / rng.uniform(0.5, 5, size=npair)[None, :]) * rng.uniform(0.1, 2, npair)
    eps = np.concatenate([rng.uniform(-0.5, -1e-3, 20), rng.uniform(1e-3, 2.0, 20)])
    eps[0], eps[-1] = -1e-4, 2e-4
    state = rng.integers(0, nsig, size=npair).astype(np.int32)
    sg = gw.sigma_convolve([0.7], [T(c)], [T(state)], [T(eps)], om, om_out, nsig).cpu().numpy()
    ref = OE.sigma_c(om, om_out, [0.7], [c], [state], [eps], nsig)
    assert max_rel(sg, ref) <= 1e-11


@pytest.mark.parametrize("nw,nwo", [(8, 37), (40, 16)])
def test_convolution_shared_energies(gw, nw, nwo):
    """Pairs that share energies (the weights are computed once per distinct energy of a q
    point) over three q points of different sizes, one of them empty; 37 output frequencies
    span three blocks of 16 (ragged), 40 nodes the larger spline bases."""
    rng = np.random.default_rng(nw + nwo)
    om = S.omega_mesh(nw)
    om_out = np.concatenate([S.omega_mesh(nwo - 2), [-0.3, 120.0]])
    nsig = 5
    cs, sts, es, wq = [], [], [], [0.2, 0.5, 0.3]
    for npair, nlev in ((300, 7), (0, 1), (57, 12)):
        levels = np.concatenate([rng.uniform(-0.6, -0.01, nlev), rng.uniform(0.05, 2.5, nlev)])
        eps = levels[rng.integers(0, len(levels), size=npair)]
        c = -np.exp(-om[:, None] / rng.uniform(0.5, 5, size=npair)[None, :]) * rng.uniform(0.1, 2, npair)
        cs.append(c)
        es.append(eps)
        sts.append(rng.integers(0, nsig, size=npair).astype(np.int32))
    sg = gw.sigma_convolve(wq, [T(c) for c in cs], [T(x) for x in sts], [T(e) for e in es], om,
                           om_out, nsig).cpu().numpy()
    gw.check()
    ref = OE.sigma_c(om, om_out, wq, cs, sts, es, nsig)
    assert max_rel(sg, ref) <= 1e-11


def test_fit_recovers_poles(gw):
    """Exact two-pole curves: the GPU fit and the oracle's run of the same algorithm on the
    same data agree per curve, and both recover the poles and residues (1e-8). The oracle
    recovers every one of these 64 curves (checked here too), so no curve is exempt."""
    om = S.omega_mesh(24)
    rng = np.random.default_rng(3)
    n = 64
    a = 0.3 * (rng.uniform(0.5, 1, (n, 2)) + 0.1j * rng.normal(size=(n, 2)))
    wp = np.stack([rng.uniform(0.3, 1.5, n) - 0.2j, rng.uniform(2.5, 6, n) - 0.5j], axis=1)
    y = np.stack([OC.model(a[i], wp[i], 1j * om) for i in range(n)])
    params, cost, iters, status = gw.continue_fit(T(y), om, npole=2)
    params = params.cpu().numpy()
    status = status.cpu().numpy()
    for i in range(n):
        a2, w2 = OC.unpack(params[i].reshape(-1))
        o = np.argsort(w2.real)
        th_o, C_o, it_o, st_o = OC.plain_fit(om, y[i], 2, +1)
        a_o, w_o = OC.unpack(th_o)
        oo = np.argsort(w_o.real)
        # the oracle recovers the exact parameters ...
        assert np.allclose(w_o[oo], wp[i], rtol=1e-8, atol=1e-9), i
        assert np.allclose(a_o[oo], a[i], rtol=1e-8, atol=1e-9), i
        # ... and so does the GPU, agreeing with the oracle's result
        assert np.allclose(w2[o], w_o[oo], rtol=1e-8, atol=1e-10), i
        assert np.allclose(a2[o], a_o[oo], rtol=1e-8, atol=1e-10), i
        assert status[i] == 0 and st_o == 0, (i, status[i], st_o)


def test_end_to_end_small_fp64(gw):
    wl = S.small_fp64()
    om = wl.omega()
    M, d, v = wl.m_full(0), wl.delta(0), wl.v(0)
    ps, eps = wl.sigma_pairs(0)
    Ms = wl.msig_rows(0)
    nsig = len(wl.sigma_states())
    P = gw.polarization([T(M)], [T(d)], om, wl.prefactor, "fp64")
    W = gw.screened_w(P, [T(v)])
    sig = gw.sigma_c(list(wl.wq), [T(Ms)], [T(ps, torch.int32)], [T(eps)], W, om, om, nsig)
    gw.check()
    Po = OP.polarization(M, d, om, wl.prefactor)
    Wo = OS.screened_wc_all(Po, v)
    co = OE.pair_coefficients(Ms, Wo)
    so = OE.sigma_c(om, om, list(wl.wq), [co], [ps], [eps], nsig)
    assert rel_fro(P[0].cpu().numpy(), Po) <= 1e-12
    assert rel_fro(W[0].cpu().numpy(), Wo) <= 1e-12
    assert max_rel(sig.cpu().numpy(), so) <= 1e-11


@pytest.mark.parametrize("nb", [70, 33])
def test_screened_w_real_symmetric(gw, nb):
    """Inversion-symmetric systems: real projections give a real symmetric P; the real
    dielectric solve (real Cholesky and inverse) matches the oracle and the complex solve."""
    wl = S.tiny(nb=nb, nocc=3, nunocc=20, mesh=(2, 1, 2), nw=6, seed=nb + 3)
    om = wl.omega()
    Mr = wl.m_full(0).real
    P = OP.polarization(Mr, wl.delta(0), om, wl.prefactor)
    assert np.all(P.imag == 0)
    v = wl.v(0)
    Wr = gw.screened_w([T(P)], [T(v)], real=True)[0]
    gw.check()
    Wr = Wr.cpu().numpy()
    ref = OS.screened_wc_all(P, v)
    assert np.all(Wr.imag == 0)
    assert max_rel(Wr, ref) <= 1e-12
    Wc = gw.screened_w([T(P)], [T(v)])[0].cpu().numpy()
    assert max_rel(Wr, Wc) <= 1e-13


def test_screened_w_real_rejects_non_positive_definite(gw):
    wl = S.tiny(nb=40, nocc=2, nunocc=6, mesh=(1, 1, 2), nw=4, seed=2)
    P = np.zeros((4, 40, 40), dtype=np.complex128)
    P[:, 5, 5] = 10.0          # eps_55 = 1 - 10 v_5 < 0: not positive definite
    gw.screened_w([T(P)], [T(wl.v(0))], real=True)
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_ENOTHPD


def test_screened_w_uneven_batch_against_oracle(gw):
    """One call over q points of unequal N_b (odd, not multiples of the 32-row blocks): the
    per-system offsets, the grid over (system, block column) and the early exits of the
    smaller systems, each system against the oracle."""
    nbs = [150, 33, 97]
    wls = [S.tiny(nb=nb, nocc=3, nunocc=24, mesh=(2, 2, 1), nw=3, seed=200 + nb) for nb in nbs]
    om = wls[0].omega()
    Ps = [OP.polarization(w.m_full(0), w.delta(0), om, w.prefactor) for w in wls]
    vs = [w.v(0) for w in wls]
    W = gw.screened_w([T(p) for p in Ps], [T(v) for v in vs])
    gw.check()
    for Pq, v, Wg in zip(Ps, vs, W):
        ref = OS.screened_wc_all(Pq, v)
        Wg = Wg.cpu().numpy()
        assert rel_fro(Wg, ref) <= 1e-12
        assert max_rel(Wg, ref) <= 1e-12


@pytest.mark.slow
def test_screened_w_bench_size_against_oracle(gw):
    """N_b = 600 (the mesh workload's basis) at two frequencies, stagewise against the oracle."""
    wl = S.tiny(nb=600, nocc=4, nunocc=40, mesh=(2, 2, 2), nw=2, seed=600)
    om = wl.omega()
    Po = OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor)
    v = wl.v(0)
    Wg = gw.screened_w([T(Po)], [T(v)])[0]
    gw.check()
    Wg = Wg.cpu().numpy()
    ref = OS.screened_wc_all(Po, v)
    assert rel_fro(Wg, ref) <= 1e-12
    assert max_rel(Wg, ref) <= 1e-12


@pytest.mark.slow
def test_polarization_fp64_full_size_sampled(gw):
    """The FP64 path at the mesh workload's size (one q: K = 409,600, N_b = 600; projections
    generated on the device, split-K over whole waves of CTAs) at 2 frequencies: the full cross
    block of 24 sampled basis indices against the oracle, which draws those columns itself."""
    wl = S.medium_mixed()
    iq = 1
    K, nb = wl.K(iq), wl.nb[iq]
    om = wl.omega()[[0, 9]]
    M = gw.synth_projections(wl.seed, S.TID_M, wl.qs[iq], 0, K, nb, dtype=torch.complex128)
    d = wl.delta(iq)
    P = gw.polarization([M], [T(d)], om, wl.prefactor, "fp64")[0]
    gw.check()
    del M
    rng = np.random.default_rng(24)
    cols = np.sort(rng.choice(nb, size=24, replace=False))
    got = P[:, cols][:, :, cols].cpu().numpy()
    ref = OP.polarization(wl.m_rows(iq, cols=cols), d, om, wl.prefactor)
    assert rel_fro(got, ref) <= 1e-12
    assert max_rel(got, ref) <= 1e-12


@pytest.mark.slow
def test_screened_w_large_basis_against_oracle(gw):
    """N_b = 2048 (the supercell's order of magnitude) at one frequency: the factorisation over
    many CTAs (one launch per panel step), the inverse by block columns and W^c, against the
    oracle on a polarization it computed itself from 4,096 transitions."""
    wl = S.tiny(nb=2048, nocc=8, nunocc=256, mesh=(1, 1, 2), nw=1, seed=2048)
    om = wl.omega()
    Po = OP.polarization(wl.m_full(0), wl.delta(0), om, wl.prefactor)
    v = wl.v(0)
    Wg = gw.screened_w([T(Po)], [T(v)])[0]
    gw.check()
    Wg = Wg.cpu().numpy()
    ref = OS.screened_wc_all(Po, v)
    assert rel_fro(Wg, ref) <= 1e-12
    assert max_rel(Wg, ref) <= 1e-12


def test_make_delta_matches_the_transition_layout(gw):
    """gw_make_delta builds Delta_t from the band energies and the k+q map in the row order of
    the projections, the same numbers as the input module's layout (the 4x4x4 mesh, two q, one
    with fewer unoccupied bands than the energy table holds); a bad k+q index is reported."""
    wl = S.medium_mixed()
    eo = T(wl.eps_occ())
    eu = T(wl.eps_unocc())
    for iq in (0, 5):
        kq = T(wl.kplus(np.arange(wl.nk), wl.qs[iq]).astype(np.int32))
        d = gw.make_delta(eo, eu, kq, nunocc=wl.nunocc[iq])
        gw.check()
        assert np.array_equal(d.cpu().numpy(), wl.delta(iq))
    d = gw.make_delta(eo, eu[:, :300], T(wl.kplus(np.arange(wl.nk), wl.qs[1]).astype(np.int32)))
    gw.check()
    ref = (wl.eps_unocc()[wl.kplus(np.arange(wl.nk), wl.qs[1])][:, None, :300]
           - wl.eps_occ()[:, :, None]).reshape(-1)
    assert np.array_equal(d.cpu().numpy(), ref)
    bad = np.zeros(wl.nk, dtype=np.int32)
    bad[3] = wl.nk
    gw.make_delta(eo, eu, T(bad))
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_EINVAL
