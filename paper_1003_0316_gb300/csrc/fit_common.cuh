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

// cost 1/2 sum_j |f(i w_j) - y_j|^2
__device__ inline double lm_cost(const double* om, const double2* y, int nw, int npole,
                                 const double* th) {
  double C = 0.0;
  for (int j = 0; j < nw; ++j) {
    double2 f = make_double2(0.0, 0.0);
    for (int p = 0; p < npole; ++p) {
      double2 a = make_double2(th[4 * p], th[4 * p + 1]);
      double2 den = make_double2(-th[4 * p + 2], om[j] - th[4 * p + 3]);
      double2 t = c_mul(a, c_inv(den));
      f.x += t.x;
      f.y += t.y;
    }
    double2 yj = y[j];
    double rx = f.x - yj.x, ry = f.y - yj.y;
    C += rx * rx + ry * ry;
  }
  return 0.5 * C;
}

// In-place Cholesky solve of the packed-lower SPD system (n <= LM_MAXP); returns false
// if a pivot is not positive.
__device__ inline bool chol_solve(double* Lp, int n, double* b) {
  auto at = [&](int i, int j) -> double& { return Lp[i * (i + 1) / 2 + j]; };
  for (int j = 0; j < n; ++j) {
    double d = at(j, j);
    for (int k = 0; k < j; ++k) d -= at(j, k) * at(j, k);
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    at(j, j) = d;
    for (int i = j + 1; i < n; ++i) {
      double s = at(i, j);
      for (int k = 0; k < j; ++k) s -= at(i, k) * at(j, k);
      at(i, j) = s / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= at(i, k) * b[k];
    b[i] = s / at(i, i);
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= at(k, i) * b[k];
    b[i] = s / at(i, i);
  }
  return true;
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

// Levenberg-Marquardt from th (updated in place).
__device__ inline void lm_run(const double* om, const double2* y, int nw, int npole, double* th,
                              double* cost, int* iters, int* status) {
  const int P = 4 * npole;
  double cscale = 0.0;
  for (int j = 0; j < nw; ++j) cscale += y[j].x * y[j].x + y[j].y * y[j].y;
  cscale *= 0.5;
  double C = lm_cost(om, y, nw, npole, th);
  double mu = -1.0;
  double A[LM_MAXP * (LM_MAXP + 1) / 2], g[LM_MAXP], Ld[LM_MAXP * (LM_MAXP + 1) / 2],
      step[LM_MAXP], thn[LM_MAXP];
  for (int it = 0; it < LM_MAXIT; ++it) {
    if (C <= LM_CTOL * cscale) {
      *cost = C;
      *iters = it;
      *status = 0;
      return;
    }
    for (int k = 0; k < P * (P + 1) / 2; ++k) A[k] = 0.0;
    for (int k = 0; k < P; ++k) g[k] = 0.0;
    for (int j = 0; j < nw; ++j) {
      double2 f = make_double2(0.0, 0.0);
      double2 D[2 * LM_MAXPOLE];
      for (int p = 0; p < npole; ++p) {
        double2 a = make_double2(th[4 * p], th[4 * p + 1]);
        double2 phi = c_inv(make_double2(-th[4 * p + 2], om[j] - th[4 * p + 3]));
        double2 t = c_mul(a, phi);
        f.x += t.x;
        f.y += t.y;
        D[2 * p] = phi;                  // d f / d a_p
        D[2 * p + 1] = c_mul(t, phi);    // d f / d w_p = a_p phi^2
      }
      double rx = f.x - y[j].x, ry = f.y - y[j].y;
      // real rows: Re part and Im part of the residual
      double rowR[LM_MAXP], rowI[LM_MAXP];
      for (int k = 0; k < 2 * npole; ++k) {
        rowR[2 * k] = D[k].x;         // d Re f / d Re x
        rowI[2 * k] = D[k].y;         // d Im f / d Re x
        rowR[2 * k + 1] = -D[k].y;    // d Re f / d Im x  (i D)
        rowI[2 * k + 1] = D[k].x;     // d Im f / d Im x
      }
      for (int a = 0; a < P; ++a) {
        g[a] += rowR[a] * rx + rowI[a] * ry;
        for (int b = 0; b <= a; ++b) A[a * (a + 1) / 2 + b] += rowR[a] * rowR[b] + rowI[a] * rowI[b];
      }
    }
    double gmax = 0.0, dmax = 0.0;
    for (int k = 0; k < P; ++k) {
      gmax = fmax(gmax, fabs(g[k]));
      dmax = fmax(dmax, A[k * (k + 1) / 2 + k]);
    }
    if (gmax <= LM_GTOL) {
      *cost = C;
      *iters = it;
      *status = 0;
      return;
    }
    if (mu < 0.0) mu = 1e-3 * dmax;
    double Cn;
    while (true) {
      for (int k = 0; k < P * (P + 1) / 2; ++k) Ld[k] = A[k];
      for (int k = 0; k < P; ++k) {
        Ld[k * (k + 1) / 2 + k] += mu * A[k * (k + 1) / 2 + k];
        step[k] = -g[k];
      }
      bool ok = chol_solve(Ld, P, step);
      if (ok) {
        for (int k = 0; k < P; ++k) thn[k] = th[k] + step[k];
        Cn = lm_cost(om, y, nw, npole, thn);
      }
      if (ok && Cn < C) {
        mu = fmax(mu / 10.0, LM_MU_MIN);
        break;
      }
      mu *= 10.0;
      if (mu > LM_MU_MAX) {
        *cost = C;
        *iters = it;
        *status = 2;
        return;
      }
    }
    double dec = C - Cn;
    double Cold = C;
    for (int k = 0; k < P; ++k) th[k] = thn[k];
    C = Cn;
    if (dec <= LM_FTOL * Cold) {
      *cost = C;
      *iters = it + 1;
      *status = 0;
      return;
    }
  }
  *cost = C;
  *iters = LM_MAXIT;
  *status = 1;
}

int launch_lm(int ncurve, int nw, const OmegaArr& om, const double* sigma, const double* sign,
              int npole, const double* theta_init, double* params, double* cost, int* iters,
              int* status, int keep_better, cudaStream_t s);

}  // namespace gw
