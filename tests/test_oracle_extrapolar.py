"""Pins of the extrapolar-correction oracle (Sec. V, band convergence): when the bands
beyond the cutoff really sit at e_bar, the corrected sums over the kept bands must equal
the brute-force sums over all bands; with no bands beyond the cutoff the correction
vanishes; and when the dropped bands spread around e_bar the error is first order in the
spread."""
import numpy as np

import synth_inputs as S
from oracle import extrapolar as OX
from oracle import polarization as OP
from oracle import screening as OS
from oracle import selfenergy as OE
from extrapolar_case import tiny_case


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_polarization_equals_full_band_sum_with_dropped_bands_at_ebar():
    c = tiny_case()
    om = c.wl.omega()
    pref = c.wl.prefactor
    Pex = OX.polarization_extrapolar(c.M, c.delta, c.dbar_t, c.C, c.dbar_kn, om, pref)
    Pfull = OP.polarization(c.M_full, c.delta_full, om, pref)
    Ptrunc = OP.polarization(c.M, c.delta, om, pref)
    assert _rel(Pex, Pfull) < 1e-13
    assert _rel(Ptrunc, Pfull) > 1e-2            # the correction is not trivial
    assert np.allclose(Pex, np.conj(np.transpose(Pex, (0, 2, 1))), atol=1e-14)
    assert np.all(np.linalg.eigvalsh(Pex) < 1e-12)   # still negative semidefinite


def test_polarization_symmetry_weights_enter_both_terms():
    c = tiny_case(seed=99)
    om = c.wl.omega()
    rng = np.random.default_rng(3)
    f_kn = rng.uniform(0.5, 2.0, size=c.nkn)
    f_full = f_kn[c.kn_of_t]
    Pex = OX.polarization_extrapolar(c.M, c.delta, c.dbar_t, c.C, c.dbar_kn, om, 0.5,
                                     f=f_full[c.kept], f_kn=f_kn)
    Pfull = OP.polarization(c.M_full, c.delta_full, om, 0.5, f=f_full)
    assert _rel(Pex, Pfull) < 1e-13


def test_sigma_equals_full_band_sum_with_dropped_bands_at_ebar():
    c = tiny_case(nw=8)
    wl = c.wl
    om, om_out = wl.omega(), wl.omega_out()
    P = OP.polarization(c.M_full, c.delta_full, om, wl.prefactor)
    Wc = OS.screened_wc_all(P, wl.v(0))
    ck = OE.pair_coefficients(c.Ms, Wc)
    cbar = OX.extrapolar_coefficients(c.S, Wc, ck, c.ps, c.nsig)
    sig_ex = OX.sigma_c_extrapolar(om, om_out, [1.0], [ck], [c.ps], [c.eps], c.nsig, [cbar],
                                   [c.ebar])
    cf = OE.pair_coefficients(c.Ms_full, Wc)
    sig_full = OE.sigma_c(om, om_out, [1.0], [cf], [c.ps_full], [c.eps_full], c.nsig)
    sig_tr = OE.sigma_c(om, om_out, [1.0], [ck], [c.ps], [c.eps], c.nsig)
    assert np.abs(sig_ex - sig_full).max() < 1e-11 * np.abs(sig_full).max()
    assert np.abs(sig_tr - sig_full).max() > 1e-3 * np.abs(sig_full).max()
    # the extra coefficient is the sum of the dropped pairs' coefficients
    drop = np.setdiff1d(np.arange(len(c.ps_full)), c.pkept)
    for s in range(c.nsig):
        ds = drop[c.ps_full[drop] == s]
        assert np.allclose(cbar[:, s], cf[:, ds].sum(axis=1), rtol=1e-11, atol=1e-14)


def test_no_bands_beyond_the_cutoff_gives_no_correction():
    c = tiny_case(nunocc=5, nkeep=5)
    om = c.wl.omega()
    Pex = OX.polarization_extrapolar(c.M, c.delta, c.dbar_t, c.C, c.dbar_kn, om, 0.25)
    assert _rel(Pex, OP.polarization(c.M, c.delta, om, 0.25)) < 1e-13
    P = OP.polarization(c.M, c.delta, om, 0.25)
    Wc = OS.screened_wc_all(P, c.wl.v(0))
    ck = OE.pair_coefficients(c.Ms, Wc)
    cbar = OX.extrapolar_coefficients(c.S, Wc, ck, c.ps, c.nsig)
    assert np.abs(cbar).max() < 1e-12 * np.abs(ck).max()


def test_error_is_first_order_in_the_spread_of_the_dropped_bands():
    om = S.omega_mesh(6)
    errs = []
    for h in (0.4, 0.1):
        c = tiny_case(spread=h)
        Pex = OX.polarization_extrapolar(c.M, c.delta, c.dbar_t, c.C, c.dbar_kn, om, 0.25)
        errs.append(_rel(Pex, OP.polarization(c.M_full, c.delta_full, om, 0.25)))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_ebar_is_sixteen_rydberg_above_the_highest_kept_band():
    assert OX.e_bar(np.array([-0.3, 1.7, 0.2])) == 1.7 + 8.0
    c = tiny_case()
    assert np.isclose(c.ebar, c.wl.eps_unocc()[:, : c.nkeep].max() + 8.0)
