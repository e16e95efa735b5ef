"""Correlation self-energy on the imaginary axis.

Eq. SEc_AC (Sec. III.C):
    Sigma^c_n(i w) = -1/(2 pi) sum_q sum_{n' all} sum_{mu nu}
                     <phi_n'|phi_n E_mu> <E_nu phi_n|phi_n'>
                     int_{-inf}^{inf} dw' W^c_{mu nu}(q, i w') / (i w + i w' - e_n')
With m_p = <E_mu phi_n|phi_n'> for a pair p = (n, n'), the band-space factor is the
quadratic form c_p(w') = m_p^H W^c(i w') m_p, real because W^c is Hermitian on the
imaginary axis, and even in w'. The BZ sum over q carries weights w_q with
sum_q w_q = 1.

Frequency integration (Sec. III.C, paragraph after Eq. SEc_AC): the integrand is
known on a mesh dense near 0; between mesh points it is a cubic spline in
lambda = w/(1+w) (so w(lambda) = lambda/(1-lambda) maps [0,1) onto [0,inf)), and
beyond the last point a tail with the asymptotic w^-2 behaviour is fitted to the
last value. The paper gives no end conditions; the reading used here: not-a-knot
at the first node, the first cubic piece extrapolated on [0, lambda_1], the slope at
the last node clamped to the tail's (dc/dw = -2 c_N / w_N), and the tail
c(w') = c_N w_N^2 / w'^2 for w' > w_N.

The oracle integrates the spline and the tail by adaptive Gauss-Kronrod
quadrature (scipy.integrate.quad_vec), not by the analytic per-segment formulas of
the CUDA path, so the two routes are independent.
"""
import numpy as np
from scipy.interpolate import CubicSpline
from scipy.integrate import quad_vec


def pair_coefficients(Msig, Wc):
    """c[j, p] = Re(m_p^H W^c_j m_p) for rows m_p of Msig ([n_pair][N_b])."""
    Msig = np.asarray(Msig, dtype=np.complex128)
    out = np.empty((Wc.shape[0], Msig.shape[0]))
    for j in range(Wc.shape[0]):
        # the same double sum over (i, j) per pair; numpy picks the contraction order
        # (a matrix product, then the row-wise dot)
        out[j] = np.einsum("pi,ij,pj->p", Msig.conj(), Wc[j], Msig, optimize=True).real
    return out


class LambdaSpline:
    """Cubic spline in lambda of values given on the imaginary-frequency nodes."""

    def __init__(self, omega, values):
        omega = np.asarray(omega, dtype=np.float64)
        values = np.asarray(values, dtype=np.float64)
        self.omega = omega
        self.lam = omega / (1.0 + omega)
        wn = omega[-1]
        cn = values[..., -1]
        # tail slope dc/dw = -2 c_N / w_N, in lambda: times dw/dlambda = (1 + w)^2
        slope = -2.0 * cn / wn * (1.0 + wn) ** 2
        self.cn = cn
        self.spline = CubicSpline(self.lam, values, axis=-1,
                                  bc_type=("not-a-knot", (1, slope)), extrapolate=True)

    def __call__(self, w):
        """Interpolant at w' <= w_N (first piece extrapolated below w_1)."""
        lam = w / (1.0 + w)
        return self.spline(lam)


def _g(w, wp, eps):
    return 1.0 / (1j * (w + wp) - eps) + 1.0 / (1j * (w - wp) - eps)


def convolution_weights(omega, omega_out, eps, epsabs=1e-15, epsrel=1e-13):
    """T[i, j] such that int_{-inf}^{inf} dw' c(w')/(i w_i + i w' - eps) = sum_j T[i,j] c_j
    for the interpolant of node values c_j (cardinal-function form: the interpolant
    is linear in the node values). Complex128 [n_out][n_omega]."""
    omega = np.asarray(omega, dtype=np.float64)
    nw = len(omega)
    basis = LambdaSpline(omega, np.eye(nw))        # row j: cardinal function of node j
    wn = omega[-1]
    T = np.zeros((len(omega_out), nw), dtype=np.complex128)
    for i, w in enumerate(np.asarray(omega_out, dtype=np.float64)):
        pts = list(omega[:-1])
        if 0.0 < abs(w) < wn:
            pts.append(abs(w))
        pts = sorted(set(pts))

        def f_body(wp):
            g = _g(w, wp, eps)
            vals = basis(wp)
            return np.concatenate([(vals * g).real, (vals * g).imag])

        body, _ = quad_vec(f_body, 0.0, wn, epsabs=epsabs, epsrel=epsrel, points=pts,
                           limit=20000, norm="max")
        # tail: w' = w_N / u, c = c_N w_N^2 / w'^2  ->  int_0^1 du  c_N w_N g(w_N/u)
        tail_pts = [wn / abs(w)] if abs(w) > wn else None

        def f_tail(u):
            if u == 0.0:
                return np.zeros(2 * nw)
            g = _g(w, wn / u, eps) * wn
            e = np.zeros(nw, dtype=np.complex128)
            e[-1] = g
            return np.concatenate([e.real, e.imag])

        tail, _ = quad_vec(f_tail, 0.0, 1.0, epsabs=epsabs, epsrel=epsrel, points=tail_pts,
                           limit=20000, norm="max")
        tot = body + tail
        T[i] = tot[:nw] + 1j * tot[nw:]
    return T


def sigma_c(omega, omega_out, wq, coeffs, pair_state, eps_np, nsig, tables=None):
    """Sigma^c_s(i w_i) = -1/(2 pi) sum_q w_q sum_{p in s} sum_j T_ij(eps_p) c_{q,j,p}.

    coeffs[q]: [n_omega][n_pair_q]; pair_state[q], eps_np[q]: [n_pair_q].
    tables: optional dict energy -> T from convolution_weights(omega, omega_out, energy)
    (computed elsewhere, e.g. by worker processes); missing energies are computed here.
    Returns complex128 [nsig][n_out].
    """
    out = np.zeros((nsig, len(omega_out)), dtype=np.complex128)
    cache = dict(tables) if tables else {}
    for iq in range(len(wq)):
        c = np.asarray(coeffs[iq])
        for p in range(c.shape[1]):
            e = float(eps_np[iq][p])
            if e == 0.0:
                raise ValueError("pair energy exactly at the Fermi level")
            if e not in cache:
                cache[e] = convolution_weights(omega, omega_out, e)
            out[pair_state[iq][p]] += wq[iq] * (cache[e] @ c[:, p])
    return -out / (2.0 * np.pi)

