"""Exchange self-energy (the first NEXT row): Eq. HFterm_MB in the Coulomb eigenbasis plus
the divergent q -> 0 term of Eq. exchange_div in its erf form (Sec. III.D). Test
infrastructure: only the tests and the benchmark's CPU baseline use this module.

Per state n: Sigma_x,n = - sum_q w_q sum_{pairs p of n, n' occupied} sum_mu v_mu |m_p,mu|^2
- f_n (4 pi / V) C, with m_p,mu = <E_mu phi_n | phi_n'> (so the band-space factor is the
quadratic form conj(m)^T diag(v) m, the a5 form with W replaced by v), n' occupied when its
energy (from the Fermi level) is negative, f_n = 1 for an occupied state n and 0 otherwise,
V the crystal volume and C the BZ constant (V/8 pi^3) int_BZ d^3k/k^2 - sum_{k != 0} 1/k^2.
Reading: the BZ sum carries the weights w_q of the correlation term (sum_q w_q = 1).
"""
import numpy as np

from . import selfenergy as OE

FOUR_PI = 4.0 * np.pi


def sigma_x(wq, Msigs, pair_states, eps_pairs, vs, nsig, eps_states, cbz, volume):
    out = np.zeros(nsig)
    for w, M, st, ep, v in zip(wq, Msigs, pair_states, eps_pairs, vs):
        c = OE.pair_coefficients(M, np.diag(np.asarray(v, dtype=np.float64))[None])[0]
        occ = np.asarray(ep) < 0
        np.add.at(out, np.asarray(st)[occ], -w * c[occ])
    f = (np.asarray(eps_states, dtype=np.float64) < 0).astype(np.float64)
    return out - f * FOUR_PI / volume * cbz
