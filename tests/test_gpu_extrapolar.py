"""GPU parity of the extrapolar correction (Sec. V, band convergence) against the oracle:
the polarization with the modified transition weights plus the completeness term (FP64
path to 1e-12; split precisions to the bounds of the tensor-core polarization, the
completeness term in FP32 with a two-float running sum), and the extra Sigma^c pair of each
state (FP64). Inputs from tests/extrapolar_case.py: a workload with more bands than are
kept, whose whole band set is the complete set of the synthetic model."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import extrapolar as OX
from oracle import polarization as OP
from oracle import screening as OS
from oracle import selfenergy as OE
from extrapolar_case import ExtrapolarCase, tiny_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {"tf32x3": 1e-6, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def T(a, dt=None):
    return torch.as_tensor(np.asarray(a), device="cuda:0", dtype=dt)


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_P(c, om, pref, M, C):
    return OX.polarization_extrapolar(M, c.delta, c.dbar_t, C, c.dbar_kn, om, pref)


@pytest.mark.parametrize("nb,mesh,nocc", [(70, (2, 2, 2), 5), (33, (1, 1, 2), 2)])
def test_fp64_polarization_extrapolar(gw, nb, mesh, nocc):
    """Ragged 64-wide HERK tiles and 16-wide completeness tiles; 40 occupied states (one full
    and one ragged chunk of 32) and 4 (one ragged chunk)."""
    c = tiny_case(nb=nb, nocc=nocc, nunocc=12, nkeep=7, mesh=mesh, nw=8, seed=nb)
    om, pref = c.wl.omega(), c.wl.prefactor
    P = gw.polarization_extrapolar([T(c.M)], [T(c.delta)], [T(c.dbar_t)], [T(c.C)],
                                   [T(c.dbar_kn)], om, pref, "fp64")[0]
    gw.check()
    P = P.cpu().numpy()
    ref = _oracle_P(c, om, pref, c.M, c.C)
    assert rel_fro(P, ref) <= 1e-12
    assert np.array_equal(P, np.conj(np.transpose(P, (0, 2, 1))))
    # and the brute-force full-band sum with the dropped bands at e_bar
    assert rel_fro(P, OP.polarization(c.M_full, c.delta_full, om, pref)) <= 1e-12


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_split_polarization_extrapolar(gw, prec):
    c = tiny_case(nb=150, nocc=9, nunocc=60, nkeep=40, mesh=(2, 2, 2), nw=6, seed=11)
    om, pref = c.wl.omega(), c.wl.prefactor
    M32 = c.M.astype(np.complex64)
    C32 = c.C.astype(np.complex64)
    P = gw.polarization_extrapolar([T(M32)], [T(c.delta)], [T(c.dbar_t)], [T(C32)],
                                   [T(c.dbar_kn)], om, pref, prec)[0]
    gw.check()
    P = P.cpu().numpy()
    ref = _oracle_P(c, om, pref, M32.astype(np.complex128), C32.astype(np.complex128))
    assert rel_fro(P, ref) <= BOUND[prec]
    assert np.array_equal(P, np.conj(np.transpose(P, (0, 2, 1))))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_real_polarization_extrapolar(gw, prec):
    """Inversion-symmetric systems: real projections and a real symmetric completeness term."""
    c = tiny_case(nb=37, nocc=3, nunocc=20, nkeep=12, mesh=(2, 2, 2), nw=5, seed=23)
    om, pref = c.wl.omega(), c.wl.prefactor
    Mr = c.M.real.astype(np.float32)
    Mf = c.M_full.real.reshape(c.nkn, c.wl.nunocc[0], -1)
    Cr = np.einsum("kna,knb->kab", Mf, Mf).astype(np.float32)
    P = gw.polarization_extrapolar([T(Mr)], [T(c.delta)], [T(c.dbar_t)], [T(Cr)],
                                   [T(c.dbar_kn)], om, pref, prec)[0]
    gw.check()
    P = P.cpu().numpy()
    ref = _oracle_P(c, om, pref, Mr.astype(np.complex128), Cr.astype(np.complex128))
    assert np.all(P.imag == 0)
    assert rel_fro(P, ref) <= BOUND[prec]


def test_polarization_extrapolar_batched_and_empty(gw):
    """Two q in one call, the second with no occupied states in the completeness term
    (P^EX = P(Delta) - P(Delta_bar) there), and symmetry weights on both terms."""
    c1 = tiny_case(nb=40, nocc=3, nunocc=10, nkeep=6, mesh=(2, 1, 2), nw=6, seed=5)
    c2 = tiny_case(nb=24, nocc=2, nunocc=8, nkeep=5, mesh=(2, 1, 1), nw=6, seed=6)
    om, pref = c1.wl.omega(), 0.3
    rng = np.random.default_rng(1)
    f_kn = rng.uniform(0.5, 2.0, size=c1.nkn)
    f_t = f_kn[c1.kn_of_t[c1.kept]]
    f2 = np.ones(len(c2.delta))
    C2 = np.zeros((0, 24, 24), dtype=np.complex128)
    P = gw.polarization_extrapolar(
        [T(c1.M), T(c2.M)], [T(c1.delta), T(c2.delta)], [T(c1.dbar_t), T(c2.dbar_t)],
        [T(c1.C), T(C2)], [T(c1.dbar_kn), T(c2.dbar_kn[:0])], om, pref, "fp64",
        fs=[T(f_t), T(f2)], f_kns=[T(f_kn), T(np.ones(0))])
    gw.check()
    ref1 = OX.polarization_extrapolar(c1.M, c1.delta, c1.dbar_t, c1.C, c1.dbar_kn, om, pref,
                                      f=f_t, f_kn=f_kn)
    ref2 = OX.polarization_extrapolar(c2.M, c2.delta, c2.dbar_t, C2, c2.dbar_kn[:0], om, pref)
    assert rel_fro(P[0].cpu().numpy(), ref1) <= 1e-12
    assert rel_fro(P[1].cpu().numpy(), ref2) <= 1e-12


def test_polarization_extrapolar_rejects_nonpositive_delta_bar(gw):
    c = tiny_case(nb=16, nocc=2, nunocc=6, nkeep=3, mesh=(1, 1, 2), nw=4, seed=8)
    om = c.wl.omega()
    bad = c.dbar_kn.copy()
    bad[1] = 0.0
    gw.polarization_extrapolar([T(c.M)], [T(c.delta)], [T(c.dbar_t)], [T(c.C)], [T(bad)], om,
                               0.5, "fp64")
    with pytest.raises(gw.GWError) as e:
        gw.check()
    assert e.value.code == gw.GW_EINVAL
    # the context stays usable
    P = gw.polarization_extrapolar([T(c.M)], [T(c.delta)], [T(c.dbar_t)], [T(c.C)],
                                   [T(c.dbar_kn)], om, 0.5, "fp64")[0]
    gw.check()
    assert rel_fro(P.cpu().numpy(), _oracle_P(c, om, 0.5, c.M, c.C)) <= 1e-12


@pytest.mark.parametrize("nw", [6, 20])
def test_sigma_extrapolar_fp64(gw, nw):
    """The extra pair coefficients and the corrected Sigma^c against the oracle and against
    the brute-force sum over all partner bands with the dropped ones at e_bar; nw = 20 spans
    three frequency groups of 8, 4 states one state group."""
    c = tiny_case(nb=40, nocc=3, nunocc=11, nkeep=6, mesh=(2, 1, 2), nw=nw, seed=17,
                  states=(0, 2, 3, 5, 7))
    wl = c.wl
    om, om_out = wl.omega(), wl.omega_out()
    P = OP.polarization(c.M_full, c.delta_full, om, wl.prefactor)
    Wc = OS.screened_wc_all(P, wl.v(0))
    ck = gw.sigma_pair_coeffs([T(c.Ms)], [T(Wc)], precision="fp64")[0]
    sig = gw.sigma_convolve([1.0], [ck], [T(c.ps, torch.int32)], [T(c.eps)], om, om_out, c.nsig)
    sig, cbar = gw.sigma_extrapolar([1.0], [T(c.S)], [T(Wc)], [T(c.ps, torch.int32)], [ck],
                                    [c.ebar], om, om_out, sig)
    gw.check()
    ck_o = OE.pair_coefficients(c.Ms, Wc)
    cbar_o = OX.extrapolar_coefficients(c.S, Wc, ck_o, c.ps, c.nsig)
    assert np.abs(cbar.cpu().numpy()[0] - cbar_o).max() <= 1e-11 * np.abs(cbar_o).max()
    ref = OX.sigma_c_extrapolar(om, om_out, [1.0], [ck_o], [c.ps], [c.eps], c.nsig, [cbar_o],
                                [c.ebar])
    got = sig.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    cf = OE.pair_coefficients(c.Ms_full, Wc)
    full = OE.sigma_c(om, om_out, [1.0], [cf], [c.ps_full], [c.eps_full], c.nsig)
    assert np.abs(got - full).max() <= 1e-10 * np.abs(full).max()


@pytest.mark.slow
def test_split_polarization_extrapolar_full_size_sampled(gw):
    """One q of the 4x4x4-mesh workload (N_b = 600, 16 occupied bands, 400 kept of 600
    unoccupied: K = 409,600 kept transitions, 1,024 occupied states), BF16x3; projections
    generated on the device, the completeness integrals formed from them there (complex64);
    sampled entries against the oracle, which regenerates the needed columns on the host."""
    base = S.medium_mixed()
    wl = S.Workload(name="extrapolar_nk64_nb600", seed=base.seed, mesh=base.mesh,
                    qs=(base.qs[1],), wq=(1.0,), nb=(600,), nocc=16, nunocc=(600,), nw=16)
    nb, nu, nkeep = 600, 600, 400
    nkn = wl.nk * wl.nocc
    om, pref = wl.omega(), wl.prefactor
    Kf = wl.K(0)
    Mf = gw.synth_projections(wl.seed, S.TID_M, wl.qs[0], 0, Kf, nb, dtype=torch.complex64)
    M3 = Mf.view(nkn, nu, nb)
    C = torch.matmul(M3.transpose(1, 2), M3.conj())            # [nkn][nb][nb] complex64
    Mk = M3[:, :nkeep, :].reshape(nkn * nkeep, nb).contiguous()
    del Mf, M3
    eo = wl.eps_occ().reshape(-1)
    ebar = float(wl.eps_unocc()[:, :nkeep].max()) + 8.0
    dbar_kn = ebar - eo
    t = np.arange(Kf)
    kept = t[(t % nu) < nkeep]
    d = wl.delta(0)[kept]
    dbar_t = dbar_kn[kept // nu]
    P = gw.polarization_extrapolar([Mk], [T(d)], [T(dbar_t)], [C], [T(dbar_kn)], om, pref,
                                   "bf16x3")[0]
    gw.check()
    rng = np.random.default_rng(5)
    cols = np.sort(rng.choice(nb, size=16, replace=False))
    Mc = wl.m_rows(0, cols=cols).astype(np.complex64).astype(np.complex128)   # [Kf][16]
    Mc3 = Mc.reshape(nkn, nu, len(cols))
    Cs = np.einsum("kna,knb->kab", Mc3, Mc3.conj())
    ref = OX.polarization_extrapolar(Mc[kept], d, dbar_t, Cs, dbar_kn, om, pref)
    got = P[:, cols][:, :, cols].cpu().numpy()
    assert rel_fro(got, ref) <= 1e-6
