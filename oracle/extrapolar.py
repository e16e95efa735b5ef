"""Extrapolar correction of the band sums (Sec. V, the paragraph on the convergence with
the number of bands; the scheme of Bruneval and Gonze with the full screened interaction
instead of a plasmon-pole model). Test infrastructure: only the tests and the
benchmark's CPU baseline use this module.

The unoccupied sums of Eqs. polar_MB and SEc_AC are cut at a band N'. The correction puts
every band n' > N' at one energy e_bar, 16 Ry (8 Ha) above the highest band n' <= N'.
Their energy denominators then no longer depend on n', and the completeness of the
one-particle states replaces the sum over n' > N' of <M_I phi_n|phi_n'><phi_n'|phi_n M_J>
by the full-band integral <phi_n| M_I conj(M_J) |phi_n> minus the kept bands.

Polarization (transition t = (k, n occ, n' <= N'), occupied state kn of t,
Delta_bar_kn = e_bar - e_n(k)):
    P^EX = sum_t w(Delta_t) M_t M_t^H
         + sum_kn w(Delta_bar_kn) [C^kn - sum_{t in kn} M_t M_t^H]
         = sum_t [w(Delta_t) - w(Delta_bar_kn(t))] M_t M_t^H + sum_kn w(Delta_bar_kn) C^kn,
    C^kn_IJ = <phi_nk| M_I conj(M_J) |phi_nk> (an input: the full-band sum of
              M_{kn n',I} conj(M_{kn n',J})), w the a1 weight (prefactor and f included).
Self-energy (state s, partner bands n' <= N' kept):
    one extra pair per (q, s) at the energy e_bar with the coefficient
    cbar_s(w') = sum_IJ W^c_IJ(w') S^s_IJ - sum_{n' <= N'} c_{s n'}(w'),
    S^s_IJ = <phi_s| conj(M_I) M_J |phi_s> (the full-band sum of conj(m_I) m_J),
convolved over frequency like every other pair (a6).
"""
import numpy as np

from . import polarization as OP
from . import selfenergy as OE

EBAR_OFFSET_HA = 8.0   # 16 Ry


def e_bar(eps_kept):
    """The common energy of the bands beyond the cutoff: 16 Ry above the highest kept band."""
    return float(np.max(eps_kept)) + EBAR_OFFSET_HA


def completeness_term(C, dbar_kn, omega, prefactor, f_kn=None):
    """sum_kn w(Delta_bar_kn, omega_j) C^kn  -> [n_omega][N_b][N_b]."""
    w = OP.transition_weights(dbar_kn, omega, prefactor, f_kn)       # [nw][nkn]
    C = np.asarray(C, dtype=np.complex128)
    return np.einsum("jk,kab->jab", w, C)


def polarization_extrapolar(M, delta, dbar_t, C, dbar_kn, omega, prefactor, f=None, f_kn=None):
    """P^EX: the kept transitions at their own energies, the rest of the band sum at e_bar."""
    return (OP.polarization(M, delta, omega, prefactor, f)
            - OP.polarization(M, dbar_t, omega, prefactor, f)
            + completeness_term(C, dbar_kn, omega, prefactor, f_kn))


def extrapolar_coefficients(S, Wc, coeffs, pair_state, nsig):
    """cbar[j, s] = sum_IJ W^c_j[I, J] S^s[I, J] - sum_{p: state(p) = s} c[j, p] (one q)."""
    Wc = np.asarray(Wc, dtype=np.complex128)
    S = np.asarray(S, dtype=np.complex128)
    full = np.einsum("jab,sab->js", Wc, S).real
    c = np.asarray(coeffs, dtype=np.float64)
    ps = np.asarray(pair_state)
    kept = np.stack([c[:, ps == s].sum(axis=1) for s in range(nsig)], axis=1)
    return full - kept


def sigma_c_extrapolar(omega, omega_out, wq, coeffs, pair_state, eps_np, nsig, cbar, ebar):
    """Sigma^c with the extra pair of every (q, s) at e_bar_q added to the kept pairs."""
    c2, ps2, e2 = [], [], []
    for iq in range(len(wq)):
        c2.append(np.concatenate([np.asarray(coeffs[iq]), np.asarray(cbar[iq])], axis=1))
        ps2.append(np.concatenate([np.asarray(pair_state[iq]), np.arange(nsig)]))
        e2.append(np.concatenate([np.asarray(eps_np[iq], dtype=np.float64),
                                  np.full(nsig, float(ebar[iq]))]))
    return OE.sigma_c(omega, omega_out, wq, c2, ps2, e2, nsig)
