"""The whole FP64 chain of the hot path for one transfer momentum q, as the oracle computes it.

Test infrastructure: composes the oracle's own functions in the order of the method,
Eq. polar_MB -> Eqs. dielec_MB, screen_MB -> Eq. SEc_AC (pair coefficients, then the
frequency convolution), for the comparisons at the sizes of the mesh workload (N_b = 600,
K = 409,600), where one pass takes about a minute. The convolution weights T(eps) of the
distinct pair energies are independent of one another and are computed by worker
processes when a pool is given; everything else runs here (numpy BLAS threads).
"""
import numpy as np

from .polarization import polarization
from .screening import screened_wc_all
from .selfenergy import pair_coefficients, convolution_weights, sigma_c


def _weights_job(args):
    omega, omega_out, e = args
    return e, convolution_weights(omega, omega_out, e)


def convolution_tables(omega, omega_out, energies, pool=None):
    """dict energy -> T(energy) for the distinct values of `energies`."""
    es = sorted(set(float(e) for e in np.asarray(energies).reshape(-1)))
    jobs = [(np.asarray(omega, dtype=np.float64), np.asarray(omega_out, dtype=np.float64), e)
            for e in es]
    res = pool.map(_weights_job, jobs) if pool is not None else [_weights_job(j) for j in jobs]
    return dict(res)


def sigma_one_q(M, delta, omega, prefactor, v, Msig, pair_state, eps_np, wq, omega_out, nsig,
                pool=None):
    """P, W^c, pair coefficients and the partial Sigma^c of one q (weight wq).

    Returns (P [nw][N_b][N_b], Wc [nw][N_b][N_b], c [nw][n_pair], Sigma [nsig][n_out])."""
    P = polarization(M, delta, omega, prefactor)
    Wc = screened_wc_all(P, v)
    c = pair_coefficients(Msig, Wc)
    tables = convolution_tables(omega, omega_out, eps_np, pool)
    sig = sigma_c(omega, omega_out, [wq], [c], [pair_state], [eps_np], nsig, tables=tables)
    return P, Wc, c, sig
