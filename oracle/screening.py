"""Dielectric matrix and screened interaction in the Coulomb eigenbasis.

Eqs. dielec_MB and screen_MB (Sec. III.C): in the basis that diagonalises the
Coulomb matrix (eigenvalues v_mu),
    eps_{mu nu}(q, i w) = delta_{mu nu} - sqrt(v_mu) P_{mu nu}(q, i w) sqrt(v_nu)
    W_{mu nu}(q, i w)   = sqrt(v_mu) eps^{-1}_{mu nu}(q, i w) sqrt(v_nu)
and the correlation part W^c = W - diag(v) (text before Eq. SEc_MB).

Route taken here: X = v^1/2 P v^1/2, eps = 1 - X (Hermitian positive definite on
the imaginary axis because P is negative semidefinite), Cholesky factor of eps,
then W^c = v^1/2 (eps^{-1} - 1) v^1/2 written as v^1/2 eps^{-1} X v^1/2, so the small
difference eps^{-1} - 1 is never formed by subtraction.
"""
import numpy as np
import scipy.linalg as sla


def dielectric(P, v):
    """eps = 1 - v^1/2 P v^1/2 for one frequency (complex128 [N_b][N_b])."""
    s = np.sqrt(np.asarray(v, dtype=np.float64))
    X = s[:, None] * np.asarray(P, dtype=np.complex128) * s[None, :]
    return np.eye(len(s)) - X, X


def screened_wc(P, v):
    """W^c for one frequency; raises numpy.linalg.LinAlgError if eps is not HPD."""
    s = np.sqrt(np.asarray(v, dtype=np.float64))
    eps, X = dielectric(P, v)
    c = sla.cho_factor(eps, lower=True, check_finite=True)
    Y = sla.cho_solve(c, X)
    Wc = s[:, None] * Y * s[None, :]
    return 0.5 * (Wc + Wc.conj().T)


def screened_wc_all(P, v):
    """W^c for every frequency of P[n_omega][N_b][N_b]."""
    return np.stack([screened_wc(P[j], v) for j in range(P.shape[0])])
