"""Inputs of the extrapolar-correction tests, built from a synthetic workload with more
unoccupied bands than are kept.

The workload's unoccupied bands n' < nkeep are the kept ones (n' <= N'); the rest stand in
for the bands beyond the cutoff. The completeness integrals that the real method takes
from the product basis, C^kn = <phi_nk| M_I conj(M_J) |phi_nk> and
S^s = <phi_s| conj(M_I) M_J |phi_s>, are formed here as the sums over this workload's whole
band set, which is then the complete set of the synthetic model. The brute-force reference
moves the energies of the dropped bands to e_bar and sums all bands directly.
"""
import numpy as np

import synth_inputs as S

EBAR_OFFSET_HA = 8.0   # 16 Ry, as in the correction itself


class ExtrapolarCase:
    def __init__(self, wl, iq, nkeep, spread=0.0, spread_seed=7):
        self.wl, self.iq, self.nkeep = wl, iq, nkeep
        nu = wl.nunocc[iq]
        nocc, nk, nb = wl.nocc, wl.nk, wl.nb[iq]
        assert 0 < nkeep <= nu
        self.nkn = nk * nocc
        t = np.arange(wl.K(iq))
        nprime = t % nu
        self.kept = t[nprime < nkeep]
        self.kn_of_t = t // nu
        eu = wl.eps_unocc()
        self.ebar = float(eu[:, :nkeep].max()) + EBAR_OFFSET_HA
        eo = wl.eps_occ().reshape(-1)                        # [kn]
        self.dbar_kn = self.ebar - eo
        delta = wl.delta(iq)
        self.M_full = wl.m_full(iq)
        # kept transitions
        self.M = self.M_full[self.kept]
        self.delta = delta[self.kept]
        self.dbar_t = self.dbar_kn[self.kn_of_t[self.kept]]
        # brute force: the dropped bands at e_bar (+ an optional spread around it)
        drop = nprime >= nkeep
        rng = np.random.default_rng(spread_seed)
        shift = spread * rng.uniform(-1.0, 1.0, size=len(t))
        self.delta_full = np.where(drop, self.dbar_kn[self.kn_of_t] + shift, delta)
        Mf = self.M_full.reshape(self.nkn, nu, nb)
        self.C = np.einsum("kna,knb->kab", Mf, Mf.conj())
        # self-energy pairs p = s * (N_occ + N_unocc) + n'
        ps, eps = wl.sigma_pairs(iq)
        nbnd = wl.n_pair_bands(iq)
        p = np.arange(len(ps))
        self.pkept = p[(p % nbnd) < nocc + nkeep]
        pdrop = (p % nbnd) >= nocc + nkeep
        self.Ms_full = wl.msig_rows(iq)
        self.ps_full = ps
        pshift = spread * rng.uniform(-1.0, 1.0, size=len(p))
        self.eps_full = np.where(pdrop, self.ebar + pshift, eps)
        self.Ms = self.Ms_full[self.pkept]
        self.ps = ps[self.pkept]
        self.eps = eps[self.pkept]
        nsig = len(wl.sigma_states())
        Ms3 = self.Ms_full.reshape(nsig, nbnd, nb)
        self.S = np.einsum("spa,spb->sab", Ms3.conj(), Ms3)
        self.nsig = nsig


def tiny_case(nb=10, nocc=2, nunocc=9, nkeep=4, mesh=(1, 1, 2), nw=6, seed=314, q=1,
              states=(0, 1, 2, 3), spread=0.0):
    wl = S.tiny(nb=nb, nocc=nocc, nunocc=nunocc, mesh=mesh, nw=nw, seed=seed, qs=(q,))
    wl.states = tuple(states)
    return ExtrapolarCase(wl, 0, nkeep, spread=spread)
