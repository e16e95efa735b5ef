"""Polarization function in the mixed product basis on the imaginary axis.

Eq. polar_MB (Sec. III.C):
    P_IJ(q, w) = sum_sigma sum_k sum_{n occ} sum_{n' unocc}
                 <M_I phi_nk | phi_n'k+q> <phi_n'k+q | phi_nk M_J>
                 * ( 1/(w + e_nk - e_n'k+q + i eta) - 1/(w - e_nk + e_n'k+q - i eta) )
evaluated at w = i omega, where the bracket is real and needs no eta (Sec. III.C,
text after Eq. polar_MB). With M_{t,I} = <M_I phi_n|phi_n'> for a transition
t = (k, n, n'), the product of projections is M_{t,I} conj(M_{t,J}); the spin sum of a
spin-degenerate system gives a factor 2 and the BZ sum carries the density 1/N_k
(Sec. II), so P = (2/N_k) sum_t f_t bracket_t M_t M_t^H with symmetry weights f_t.
"""
import numpy as np


def bracket(delta, omega):
    """[1/(i w + e_n - e_n') - 1/(i w - e_n + e_n')] with Delta = e_n' - e_n.

    Returns a real array [n_omega][n_trans] (the imaginary parts cancel exactly on
    the imaginary axis).
    """
    iw = 1j * np.asarray(omega, dtype=np.float64)[:, None]
    d = np.asarray(delta, dtype=np.float64)[None, :]
    b = 1.0 / (iw - d) - 1.0 / (iw + d)
    return b.real


def transition_weights(delta, omega, prefactor, f=None):
    """w_tj = prefactor * f_t * bracket(Delta_t, omega_j); shape [n_omega][K]."""
    w = prefactor * bracket(delta, omega)
    if f is not None:
        w = w * np.asarray(f, dtype=np.float64)[None, :]
    return w


def polarization(M, delta, omega, prefactor, f=None):
    """P[j, I, J] = sum_t w_tj M[t, I] conj(M[t, J])  (complex128, [n_omega][N_b][N_b])."""
    M = np.asarray(M, dtype=np.complex128)
    w = transition_weights(delta, omega, prefactor, f)
    nw = w.shape[0]
    nb = M.shape[1]
    P = np.empty((nw, nb, nb), dtype=np.complex128)
    Mc = M.conj()
    for j in range(nw):
        P[j] = (M.T * w[j][None, :]) @ Mc
    return P


def polarization_entries(M_cols_I, M_cols_J, delta, omega, prefactor, f=None):
    """Selected entries: P[j, a, b] for column blocks (M[:, I_a], M[:, J_b])."""
    w = transition_weights(delta, omega, prefactor, f)
    A = np.asarray(M_cols_I, dtype=np.complex128)
    B = np.asarray(M_cols_J, dtype=np.complex128).conj()
    return np.stack([(A.T * w[j][None, :]) @ B for j in range(w.shape[0])])
