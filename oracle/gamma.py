"""q = Gamma: head and wings of P and W, their angular average, and the divergent part of
Sigma^c (Sec. III.D: Eqs. polar_Gamma and screen_Gamma with the expressions after them,
the spherical-harmonic expansion of the head, Eq. correlation_div, and the erf form of
the BZ constant derived for the exchange term). Test infrastructure: only the tests
and the benchmark's CPU baseline use this module.

Input (synthetic k.p stand-in): three extra columns p_t = (p_tx, p_ty, p_tz) per
transition, the linear-in-k coefficients of the projection onto the divergent Coulomb
eigenfunction, M_{t,1}(k) = k e.p_t. The polarization of the augmented projections
[p | M] (Eq. polar_MB, index order P_IJ = sum_t w_t M_tI conj(M_tJ)) then holds
    H_ab   = P_aug[a][b]          (head:  P_11 = k^2 e^T H e)
    s_nu,a = P_aug[a][3 + nu]     (wing:  P_1nu = k e^T s_nu, P_nu1 = k e^T conj(s_nu))
    P~     = P_aug[3:, 3:]        (body).

Readings (the printed wing/body expressions of Eq. screen_Gamma are not all consistent
with W = v^1/2 eps^-1 v^1/2 and v_1 = 4 pi / k^2, so the exact block inverse is taken):
with W~ = v^1/2 eps~^-1 v^1/2 (eps~ = 1 - v^1/2 P~ v^1/2) and
    u_nu = sum_mu s_mu W~_{mu nu}                              (3-vector per nu)
    L    = 1 - 4 pi H - 4 pi sum_nu u_nu conj(s_nu)^T          (3x3, Hermitian)
the full inverse gives, for every k and unit direction e,
    W_11     = 4 pi / (k^2 e^T L e)
    W_1nu    = 4 pi e^T u_nu / (k e^T L e),   W_nu1 = conj(W_1nu)
    W_mu,nu  = W~_mu,nu + 4 pi conj(e^T u_mu) (e^T u_nu) / (e^T L e).
For real data u_nu = w_nu sqrt(v_nu) / sqrt(4 pi) with the printed w_nu, and L is the
printed L.
Angular treatment: the head's l = 0 coefficient K_00 = sqrt(4 pi) <4 pi / e^T L e>
(average over the unit sphere), K^c_00 = K_00 - (4 pi)^(3/2); the body keeps the l = 0
part of its rank-one term, 4 pi sum_ab conj(u_mu,a) u_nu,b <e_a e_b / e^T L e>.
"""
import numpy as np
from scipy.integrate import dblquad
from scipy.special import erf

from . import selfenergy as OE

FOUR_PI = 4.0 * np.pi


def split_augmented(Paug):
    """H [nw][3][3], S [nw][nb][3] (S[j, nu, a] = s_nu,a), P~ [nw][nb][nb]."""
    Paug = np.asarray(Paug, dtype=np.complex128)
    H = Paug[:, :3, :3]
    S = np.transpose(Paug[:, :3, 3:], (0, 2, 1))
    return H, S, Paug[:, 3:, 3:]


def head_wing_terms(H, S, Wt_c, v):
    """u [nb][3] and L [3][3] for one frequency, from W~^c = W~ - diag(v)."""
    v = np.asarray(v, dtype=np.float64)
    Wt = np.asarray(Wt_c, dtype=np.complex128) + np.diag(v)
    u = Wt.T @ S                                   # u[nu, a] = sum_mu W~[mu, nu] S[mu, a]
    L = np.eye(3) - FOUR_PI * H - FOUR_PI * (u.T @ S.conj())
    return u, L


def full_w_at_k(P_full, v_body, k):
    """Brute force: W = v^1/2 eps^-1 v^1/2 of the (nb+1)-dimensional problem at finite k
    (index 0 the divergent eigenfunction, v_0 = 4 pi / k^2)."""
    vv = np.concatenate([[FOUR_PI / k ** 2], np.asarray(v_body, dtype=np.float64)])
    r = np.sqrt(vv)
    eps = np.eye(len(vv)) - r[:, None] * P_full * r[None, :]
    return r[:, None] * np.linalg.inv(eps) * r[None, :]


def sphere_average(f, epsabs=1e-13, epsrel=1e-12):
    """(1/4 pi) int f(e) dOmega by adaptive quadrature over (cos theta, phi)."""
    def g(phi, x):
        st = np.sqrt(max(0.0, 1.0 - x * x))
        return f(np.array([st * np.cos(phi), st * np.sin(phi), x]))
    val, _ = dblquad(g, -1.0, 1.0, 0.0, 2.0 * np.pi, epsabs=epsabs, epsrel=epsrel)
    return val / FOUR_PI


def angular_moments(L):
    """<1 / e^T L e> and A_ab = <e_a e_b / e^T L e> over the unit sphere."""
    Lr = np.real(np.asarray(L))            # e^T L e = e^T Re(L) e for Hermitian L, real e
    inv = sphere_average(lambda e: 1.0 / (e @ Lr @ e))
    A = np.empty((3, 3))
    for a in range(3):
        for b in range(a, 3):
            A[a, b] = A[b, a] = sphere_average(lambda e: e[a] * e[b] / (e @ Lr @ e))
    return inv, A


def gamma_all(Paug, v, Wt_c=None):
    """Per frequency: K^c_00, L, u and the body W^c with its l = 0 rank-one term.
    Wt_c (W~^c of the body) is computed from P~ by the screening oracle if not given."""
    from . import screening as OS
    H, S, Pt = split_augmented(Paug)
    nw = Pt.shape[0]
    if Wt_c is None:
        Wt_c = OS.screened_wc_all(Pt, v)
    K00c = np.empty(nw)
    Ls = np.empty((nw, 3, 3), dtype=np.complex128)
    us = np.empty((nw, len(v), 3), dtype=np.complex128)
    body = np.array(Wt_c, dtype=np.complex128)
    for j in range(nw):
        u, L = head_wing_terms(H[j], S[j], Wt_c[j], v)
        inv, A = angular_moments(L)
        K00c[j] = np.sqrt(FOUR_PI) * FOUR_PI * inv - FOUR_PI ** 1.5
        Ls[j], us[j] = L, u
        body[j] = body[j] + FOUR_PI * (u.conj() @ A @ u.T)
    return K00c, Ls, us, body


# ------------------------------------------------------------- BZ constant --
def q0_of_beta(beta):
    """Cutoff radius from exp(-beta q0^2) = beta."""
    return np.sqrt(-np.log(beta) / beta)


def bz_constant_sc(a, n, beta=0.005, chunk=64):
    """C = (V / 8 pi^3) int_BZ d^3k / k^2 - sum_{k != 0} 1/k^2 for a simple-cubic lattice
    (constant a) with an n x n x n k mesh, V = n^3 a^3, in the erf form:
        C = V / (4 pi) [erf(sqrt(beta) q0) / sqrt(pi beta)] - sum_{0<|q|<q0} e^{-beta q^2} / q^2
    over all q = k + G (the reciprocal lattice of the supercell, spacing 2 pi / (n a))."""
    V = (n * a) ** 3
    q0 = q0_of_beta(beta)
    dq = 2.0 * np.pi / (n * a)
    m = int(np.floor(q0 / dq))
    r = np.arange(-m, m + 1, dtype=np.float64)
    total = 0.0
    for i0 in range(0, len(r), chunk):
        x = r[i0:i0 + chunk, None, None] * dq
        y = r[None, :, None] * dq
        q2 = x * x + y * y + (r[None, None, :] * dq) ** 2
        sel = (q2 > 0) & (q2 < q0 * q0)
        total += np.sum(np.exp(-beta * q2[sel]) / q2[sel])
    return V / FOUR_PI * erf(np.sqrt(beta) * q0) / np.sqrt(np.pi * beta) - total


def bz_constant_sc_gauss(a, n, beta=0.005, beta_qmax2=16.0, chunk=32):
    """The same constant without the cutoff rule: the Gaussian-weighted integral over all
    reciprocal space in closed form, (V / 8 pi^3) 4 pi int_0^inf e^{-beta q^2} dq =
    V / (4 pi^(3/2) sqrt(beta)), minus the lattice sum of e^{-beta q^2} / q^2 out to
    beta q_max^2 = beta_qmax2 (terms beyond are below e^-16)."""
    V = (n * a) ** 3
    qmax = np.sqrt(beta_qmax2 / beta)
    dq = 2.0 * np.pi / (n * a)
    m = int(np.floor(qmax / dq))
    r = np.arange(-m, m + 1, dtype=np.float64) * dq
    total = 0.0
    for i0 in range(0, len(r), chunk):
        q2 = r[i0:i0 + chunk, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
        sel = q2 > 0
        total += np.sum(np.exp(-beta * q2[sel]) / q2[sel])
    return V / (4.0 * np.pi ** 1.5 * np.sqrt(beta)) - total


def sigma_div(omega, omega_out, K00c, cbz, volume, eps_states):
    """Eq. correlation_div for each state: -C / (4 pi^(3/2) V) int dw' K^c_00(w') /
    (i w + i w' - e_n), the frequency integral by the spline-in-lambda interpolant and
    tail of the a6 convolution (oracle route: adaptive quadrature)."""
    eps_states = np.asarray(eps_states, dtype=np.float64)
    nsig = len(eps_states)
    # one pair per state with c = K^c_00 and a weight that turns the convolution's
    # -1/(2 pi) into -C / (4 pi^(3/2) V)
    wq = cbz / (2.0 * np.sqrt(np.pi) * volume)
    coeffs = np.repeat(np.asarray(K00c, dtype=np.float64)[:, None], nsig, axis=1)
    return OE.sigma_c(omega, omega_out, [wq], [coeffs], [np.arange(nsig)], [eps_states], nsig)
