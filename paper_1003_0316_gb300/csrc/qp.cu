// Quasiparticle energies (Eq. quasipart_corr with the continued self-energy of Eq. modelf),
// FP64, one thread per state: Newton's method on
//   g(E) = E - (eps + Sigma_x - v_xc) - Re f(E),   f(E) = sum_p a_p / (E - w_p),
//   g'(E) = 1 + Re sum_p a_p / (E - w_p)^2,
// from E = eps, until |dE| <= 1e-14 max(1, |E|) (status 0) or 100 steps (status 1). On the
// real axis the conjugated form of f for Re w < 0 has the same real part, so one formula
// serves both signs of E. Z = 1 / g'(E) is returned as well.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int QP_MAXIT = 100;
constexpr double QP_TOL = 1e-14;
constexpr int QP_MAXPOLE = 5;

// Re sum a/(E - w) and Re sum a/(E - w)^2
__device__ void qp_sums(const double* th, int npole, double e, double* f, double* fp) {
  double s1 = 0.0, s2 = 0.0;
  for (int p = 0; p < npole; ++p) {
    const double ar = th[4 * p], ai = th[4 * p + 1];
    const double dr = e - th[4 * p + 2], di = -th[4 * p + 3];
    const double inv = 1.0 / (dr * dr + di * di);
    const double ur = dr * inv, ui = -di * inv;          // 1 / (E - w)
    s1 += ar * ur - ai * ui;
    const double vr = ur * ur - ui * ui, vi = 2.0 * ur * ui;   // 1 / (E - w)^2
    s2 += ar * vr - ai * vi;
  }
  *f = s1;
  *fp = s2;
}

__global__ void k_qp(int n, int npole, const double* __restrict__ params, const double* __restrict__ eps,
                     const double* __restrict__ sigx, const double* __restrict__ vxc,
                     double* __restrict__ E, double* __restrict__ Z, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double th[4 * QP_MAXPOLE];
  for (int k = 0; k < 4 * npole; ++k) th[k] = params[size_t(i) * 4 * npole + k];
  const double c = eps[i] + sigx[i] - vxc[i];
  double e = eps[i];
  int st = 1;
  double f, fp;
  for (int it = 0; it < QP_MAXIT; ++it) {
    qp_sums(th, npole, e, &f, &fp);
    const double step = (e - c - f) / (1.0 + fp);
    e -= step;
    if (fabs(step) <= QP_TOL * fmax(1.0, fabs(e))) {
      st = 0;
      break;
    }
  }
  qp_sums(th, npole, e, &f, &fp);
  E[i] = e;
  if (Z) Z[i] = 1.0 / (1.0 + fp);
  if (status) status[i] = st;
}

}  // namespace

int qp_solve(int n, int npole, const double* params, const double* eps, const double* sigx,
             const double* vxc, double* E, double* Z, int* status, cudaStream_t s) {
  k_qp<<<(n + 127) / 128, 128, 0, s>>>(n, npole, params, eps, sigx, vxc, E, Z, status);
  GW_LAUNCH_CHECK("k_qp");
  return GW_OK;
}

}  // namespace gw
