// a7: analytic continuation of Sigma^c(i w) by the multipole model of Eq. modelf,
// f(z) = sum_p a_p / (z - w_p), fitted in FP64 by Levenberg-Marquardt
// (Marquardt 1963, diagonal scaling), one thread per curve.
//
// Cost C = 1/2 sum_j |f(i w_j) - y_j|^2 over the parameters
// theta = (Re a_p, Im a_p, Re w_p, Im w_p)_p. Each iteration accumulates
// A = J^T J and g = J^T r row by row from the analytic derivatives
// df/da_p = 1/(z - w_p), df/dw_p = a_p/(z - w_p)^2 (f is holomorphic in each
// parameter, so d/dRe = D and d/dIm = i D), solves (A + mu diag A) d = -g by
// Cholesky, and accepts the step when the cost drops (mu /= 10, floor 1e-15),
// otherwise mu *= 10 (give up above 1e15). Stops after an accepted step whose
// relative cost decrease is <= 1e-14, when C <= 1e-28 * (1/2 sum |y|^2), or after
// 200 iterations. Default start: w_p = s (0.5, 2, 5, 10, 20)_p - 0.1 i s (s the sign
// of the state energy) with residues from the linear least-squares problem.
#include "gw_internal.cuh"
#include "fit_common.cuh"

namespace gw {

__global__ void __launch_bounds__(128) k_lm_fit(int ncurve, int nw, OmegaArr om,
                                                const double2* __restrict__ sigma,
                                                const double* __restrict__ sign, int npole,
                                                const double* __restrict__ theta_init,
                                                double* __restrict__ params,
                                                double* __restrict__ cost_out,
                                                int* __restrict__ iters_out,
                                                int* __restrict__ status_out, int keep_better) {
  int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= ncurve) return;
  const double2* y = sigma + size_t(cidx) * nw;
  double th[LM_MAXP];
  const int P = 4 * npole;
  if (theta_init) {
    for (int k = 0; k < P; ++k) th[k] = theta_init[size_t(cidx) * P + k];
  } else {
    double s = sign ? (sign[cidx] >= 0.0 ? 1.0 : -1.0) : 1.0;
    lm_default_start(om.v, y, nw, npole, s, th);
  }
  double C;
  int iters, st;
  lm_run(om.v, y, nw, npole, th, &C, &iters, &st);
  if (keep_better) {
    // compare with the result already stored (the other start) and keep the lower cost
    double Cold = cost_out[cidx];
    if (!(C < Cold)) return;
  }
  for (int k = 0; k < P; ++k) params[size_t(cidx) * P + k] = th[k];
  cost_out[cidx] = C;
  iters_out[cidx] = iters;
  status_out[cidx] = st;
}

int launch_lm(int ncurve, int nw, const OmegaArr& om, const double* sigma, const double* sign,
              int npole, const double* theta_init, double* params, double* cost, int* iters,
              int* status, int keep_better, cudaStream_t s) {
  if (ncurve == 0) return GW_OK;
  k_lm_fit<<<(ncurve + 127) / 128, 128, 0, s>>>(ncurve, nw, om,
                                                reinterpret_cast<const double2*>(sigma), sign,
                                                npole, theta_init, params, cost, iters, status,
                                                keep_better);
  GW_LAUNCH_CHECK("k_lm_fit");
  return GW_OK;
}

}  // namespace gw
