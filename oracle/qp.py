"""Quasiparticle energies (the fourth NEXT row): Eq. quasipart_corr solved with the
analytically continued correlation self-energy of Eq. modelf. Test infrastructure: only the
tests and the benchmark's CPU baseline use this module.

E_n = eps_n + Sigma_x,n + Re f_n(E_n) - v_xc,n with f(w) = sum_p a_p / (w - w_p); on the real
axis the conjugated form for Re w < 0 has the same real part, so Re f(E) = Re sum_p a_p/(E - w_p)
for every real E. Newton's method from E = eps_n (the paper's "standard iterative Newton
method"): g(E) = E - c - Re f(E), c = eps + Sigma_x - v_xc, g'(E) = 1 + Re sum_p a_p/(E - w_p)^2;
stop when |dE| <= 1e-14 max(1, |E|) or after 100 steps. Also returns the renormalisation
factor Z = 1 / g'(E).
"""
import numpy as np

MAXIT = 100
TOL = 1e-14


def qp_solve(params, eps, sigx, vxc):
    """params [n][npole][4] = (Re a, Im a, Re w, Im w); returns (E, Z, status) with status 0
    converged, 1 iteration limit."""
    params = np.asarray(params, dtype=np.float64)
    a = params[..., 0] + 1j * params[..., 1]
    w = params[..., 2] + 1j * params[..., 3]
    n = params.shape[0]
    E = np.empty(n)
    Z = np.empty(n)
    st = np.zeros(n, dtype=np.int32)
    for i in range(n):
        c = eps[i] + sigx[i] - vxc[i]
        e = float(eps[i])
        ok = False
        for _ in range(MAXIT):
            d = e - w[i]
            g = e - c - np.real(np.sum(a[i] / d))
            gp = 1.0 + np.real(np.sum(a[i] / d ** 2))
            step = g / gp
            e -= step
            if abs(step) <= TOL * max(1.0, abs(e)):
                ok = True
                break
        d = e - w[i]
        E[i] = e
        Z[i] = 1.0 / (1.0 + np.real(np.sum(a[i] / d ** 2)))
        st[i] = 0 if ok else 1
    return E, Z, st
