// Device routines of the multipole fit (Eq. modelf), shared by the plain fit and the
// learned-start path.
#pragma once
#include "gw_internal.cuh"

namespace gw {

constexpr int LM_MAXPOLE = 5;
constexpr int LM_MAXP = 4 * LM_MAXPOLE;
constexpr int LM_MAXIT = 200;
constexpr double LM_FTOL = 1e-14;
constexpr double LM_CTOL = 1e-28;
constexpr double LM_GTOL = 1e-300;
constexpr double LM_MU_MIN = 1e-15;
constexpr double LM_MU_MAX = 1e15;

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_inv(double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2(1.0 / d, -r / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2(r / d, -1.0 / d);
  }
}

// Default start: poles s*(0.5, 2, 5, 10, 20)_p - 0.1 i s, residues from the normal
// equations of the linear least-squares problem at fixed poles (complex Cholesky).
__device__ inline void lm_default_start(const double* om, const double2* y, int nw, int npole,
                                        double s, double* th) {
  const double starts[5] = {0.5, 2.0, 5.0, 10.0, 20.0};
  double2 wp[LM_MAXPOLE];
  for (int p = 0; p < npole; ++p) wp[p] = make_double2(s * starts[p], -0.1 * s);
  // G = Phi^H Phi (Hermitian), h = Phi^H y
  double2 G[LM_MAXPOLE][LM_MAXPOLE], h[LM_MAXPOLE];
  for (int p = 0; p < npole; ++p) {
    h[p] = make_double2(0.0, 0.0);
    for (int q = 0; q < npole; ++q) G[p][q] = make_double2(0.0, 0.0);
  }
  for (int j = 0; j < nw; ++j) {
    double2 phi[LM_MAXPOLE];
    for (int p = 0; p < npole; ++p) phi[p] = c_inv(make_double2(-wp[p].x, om[j] - wp[p].y));
    for (int p = 0; p < npole; ++p) {
      double2 cp = make_double2(phi[p].x, -phi[p].y);
      double2 t = c_mul(cp, y[j]);
      h[p].x += t.x;
      h[p].y += t.y;
      for (int q = 0; q < npole; ++q) {
        double2 u = c_mul(cp, phi[q]);
        G[p][q].x += u.x;
        G[p][q].y += u.y;
      }
    }
  }
  // complex Cholesky G = L L^H
  double2 L[LM_MAXPOLE][LM_MAXPOLE];
  for (int j = 0; j < npole; ++j) {
    double d = G[j][j].x;
    for (int k = 0; k < j; ++k) d -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
    d = sqrt(d > 0.0 ? d : 1e-300);
    L[j][j] = make_double2(d, 0.0);
    for (int i = j + 1; i < npole; ++i) {
      double2 sum = G[i][j];
      for (int k = 0; k < j; ++k) {
        double2 t = c_mul(L[i][k], make_double2(L[j][k].x, -L[j][k].y));
        sum.x -= t.x;
        sum.y -= t.y;
      }
      L[i][j] = make_double2(sum.x / d, sum.y / d);
    }
  }
  double2 z[LM_MAXPOLE];
  for (int i = 0; i < npole; ++i) {
    double2 sum = h[i];
    for (int k = 0; k < i; ++k) {
      double2 t = c_mul(L[i][k], z[k]);
      sum.x -= t.x;
      sum.y -= t.y;
    }
    z[i] = make_double2(sum.x / L[i][i].x, sum.y / L[i][i].x);
  }
  for (int i = npole - 1; i >= 0; --i) {
    double2 sum = z[i];
    for (int k = i + 1; k < npole; ++k) {
      double2 t = c_mul(make_double2(L[k][i].x, -L[k][i].y), z[k]);
      sum.x -= t.x;
      sum.y -= t.y;
    }
    z[i] = make_double2(sum.x / L[i][i].x, sum.y / L[i][i].x);
  }
  for (int p = 0; p < npole; ++p) {
    th[4 * p] = z[p].x;
    th[4 * p + 1] = z[p].y;
    th[4 * p + 2] = wp[p].x;
    th[4 * p + 3] = wp[p].y;
  }
}

int launch_lm(int ncurve, int nw, const OmegaArr& om, const double* sigma, const double* sign,
              int npole, const double* theta_init, double* params, double* cost, int* iters,
              int* status, int keep_better, cudaStream_t s);

}  // namespace gw
