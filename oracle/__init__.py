"""CPU FP64 oracle for the GW hot path (test infrastructure only).

This package is the checker, not the product: only the tests, the smoke check of
the graft entry point and the CPU-baseline leg of the benchmark import it. It is a
plain, slow restatement of the method of Friedrich, Bluegel and Schindlmayr,
"Efficient implementation of the GW approximation within the all-electron FLAPW
method" (Sec. III.C "Formulation in the MPB", Sec. III.E "Gamma-point treatment"),
written in numpy/scipy double precision, one step per equation:

* polarization.py  -- transition weights and P_IJ(q, i omega)     (Eq. polar_MB)
* screening.py     -- dielectric matrix and W^c                     (Eqs. dielec_MB, screen_MB)
* selfenergy.py    -- pair coefficients and frequency convolution    (Eq. SEc_AC, Sec. III.C)
* continuation.py  -- multipole model and Levenberg-Marquardt fit    (Eq. modelf)
* mlp.py           -- the learned initialiser of the fit (FP64 forward/backward)
* gamma.py         -- head/wings/body treatment at q -> 0             (Eqs. polar_Gamma, screen_Gamma,
                      correlation_div)

It shares no code with the CUDA library and never imports it. Library primitives
(numpy matmul, Cholesky, triangular solves, scipy's adaptive Gauss-Kronrod
quadrature and cubic spline) serve as single steps.
"""
from . import polarization, screening, selfenergy, continuation, mlp  # noqa: F401
