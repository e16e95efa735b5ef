"""Analytic continuation by a multipole fit.

Eq. modelf (Sec. III.C): f(w) = sum_{p=1}^{N_p} a_p / (w - w_p) for Re w >= 0, with
complex a_p and w_p, fitted to Sigma^c(i w_j) on the imaginary mesh; for Re w < 0 the
parameters enter conjugated. The paper does not state the cost or the solver; the
reading used here (shared with the CUDA kernel):

* cost C = 1/2 sum_j |f(i w_j) - y_j|^2, unweighted, over Re and Im parts;
* parameters theta = (Re a_p, Im a_p, Re w_p, Im w_p)_p;
* default start: w_p = s * (0.5, 2, 5, 10, 20)_p - 0.1 i s with s = sign of the state
  energy, then the residues from the linear least-squares problem at fixed poles;
* Levenberg-Marquardt (Marquardt 1963) with Marquardt's diagonal scaling:
  solve (A + mu diag A) d = -g with A = J^T J, g = J^T r; accept when the cost drops
  (mu /= 10, floor 1e-15), else mu *= 10 (give up above 1e15); start
  mu = 1e-3 max diag A; stop after an accepted step whose relative cost decrease is
  below ftol, when max|g| <= gtol, when C <= ctol * (1/2 sum |y|^2), or after maxit
  iterations.
"""
import numpy as np

POLE_STARTS = (0.5, 2.0, 5.0, 10.0, 20.0)
MAXIT = 200
FTOL = 1e-14
GTOL = 1e-300
CTOL = 1e-28
MU_MIN = 1e-15
MU_MAX = 1e15


def model(a, wp, z):
    """f(z) = sum_p a_p / (z - w_p); z array, a and wp complex arrays [N_p]."""
    z = np.asarray(z)[:, None]
    return (np.asarray(a)[None, :] / (z - np.asarray(wp)[None, :])).sum(axis=1)


def unpack(theta):
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 4)
    return th[:, 0] + 1j * th[:, 1], th[:, 2] + 1j * th[:, 3]


def pack(a, wp):
    return np.stack([np.real(a), np.imag(a), np.real(wp), np.imag(wp)], axis=1).reshape(-1)


def residual(theta, omega, y):
    a, wp = unpack(theta)
    r = model(a, wp, 1j * np.asarray(omega)) - y
    return np.concatenate([r.real, r.imag])


def jacobian(theta, omega):
    a, wp = unpack(theta)
    z = 1j * np.asarray(omega)[:, None]
    phi = 1.0 / (z - wp[None, :])                # d f / d a_p
    psi = a[None, :] * phi * phi                  # d f / d w_p
    cols = []
    for p in range(len(a)):
        for D in (phi[:, p], psi[:, p]):
            cols.append(np.concatenate([D.real, D.imag]))            # d/d Re
            cols.append(np.concatenate([-D.imag, D.real]))           # d/d Im  (i D)
    return np.stack(cols, axis=1)


def default_poles(npole, sign):
    s = 1.0 if sign >= 0 else -1.0
    return np.array([s * POLE_STARTS[p] - 0.1j * s for p in range(npole)])


def residues_at_poles(omega, y, wp):
    """Linear least squares for a_p at fixed poles."""
    Phi = 1.0 / (1j * np.asarray(omega)[:, None] - np.asarray(wp)[None, :])
    a, *_ = np.linalg.lstsq(Phi, y, rcond=None)
    return a


def lm_fit(omega, y, theta0, maxit=MAXIT):
    """Levenberg-Marquardt; returns (theta, cost, iterations, status)
    status: 0 converged (ftol/gtol/ctol), 1 iteration limit, 2 mu overflow."""
    omega = np.asarray(omega, dtype=np.float64)
    y = np.asarray(y, dtype=np.complex128)
    theta = np.array(theta0, dtype=np.float64)
    r = residual(theta, omega, y)
    C = 0.5 * r @ r
    cscale = 0.5 * np.sum(np.abs(y) ** 2)
    mu = None
    for it in range(maxit):
        if C <= CTOL * cscale:
            return theta, C, it, 0
        J = jacobian(theta, omega)
        A = J.T @ J
        g = J.T @ r
        if np.max(np.abs(g)) <= GTOL:
            return theta, C, it, 0
        d = np.diag(A).copy()
        if mu is None:
            mu = 1e-3 * np.max(d)
        while True:
            step = np.linalg.solve(A + mu * np.diag(d), -g)
            th_new = theta + step
            r_new = residual(th_new, omega, y)
            C_new = 0.5 * r_new @ r_new
            if C_new < C:
                mu = max(mu / 10.0, MU_MIN)
                break
            mu *= 10.0
            if mu > MU_MAX:
                return theta, C, it, 2
        dec = C - C_new
        theta, r, C_old, C = th_new, r_new, C, C_new
        if dec <= FTOL * C_old:
            return theta, C, it + 1, 0
    return theta, C, maxit, 1


def plain_fit(omega, y, npole, sign, maxit=MAXIT):
    """Default-start fit (the method without the learned initialiser)."""
    wp = default_poles(npole, sign)
    a = residues_at_poles(omega, y, wp)
    return lm_fit(omega, y, pack(a, wp), maxit=maxit)
