// a7: analytic continuation of Sigma^c(i w) by the multipole model of Eq. modelf,
// f(z) = sum_p a_p / (z - w_p), fitted in FP64 by Levenberg-Marquardt
// (Marquardt 1963, diagonal scaling), one warp per curve.
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

// One warp per curve: lanes take frequency points (j = lane, lane + 32) for the residual,
// the Jacobian rows and the cost; the normal matrix A = J^T J and g = J^T r are summed over
// points by lanes owning (a, b) entries; the damped system is factored column by column
// (lanes take the rows below the pivot) and solved by column sweeps. FP64 throughout; the
// iteration, damping and stopping rules are the ones stated at the top of this file.
constexpr int LM_WMAXNW = 64;
constexpr int LM_NPACK = LM_MAXP * (LM_MAXP + 1) / 2;

struct LmWarpSmem {
  double rowR[LM_WMAXNW][LM_MAXP];
  double rowI[LM_WMAXNW][LM_MAXP];
  double res[LM_WMAXNW][2];
  double A[LM_NPACK];
  double Ld[LM_NPACK];
  double g[LM_MAXP];
  double b[LM_MAXP];
  double dinv[LM_MAXP];     // reciprocals of the factor's diagonal
  double th[LM_MAXP];
  int flag;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// 1/2 sum_j |f(i w_j) - y_j|^2 for parameters t (all lanes hold t), warp-summed.
__device__ __forceinline__ double warp_cost(const double* om, const double2* yl, int nw, int npole,
                                            const double* t) {
  const int lane = threadIdx.x & 31;
  double c = 0.0;
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    if (j >= nw) break;
    double fx = 0.0, fy = 0.0;
    for (int p = 0; p < npole; ++p) {
      const double dx = -t[4 * p + 2], dy = om[j] - t[4 * p + 3];
      const double inv = 1.0 / (dx * dx + dy * dy);
      const double px = dx * inv, py = -dy * inv;          // phi = 1 / (i w_j - w_p)
      fx += t[4 * p] * px - t[4 * p + 1] * py;
      fy += t[4 * p] * py + t[4 * p + 1] * px;
    }
    const double rx = fx - yl[h].x, ry = fy - yl[h].y;
    c += rx * rx + ry * ry;
  }
  return 0.5 * warp_sum(c);
}

// NPOLE: poles of the model (a template parameter, so that the parameter vectors and the
// loops over them stay in registers)
template <int NPOLE>
__global__ void __launch_bounds__(32) k_lm_warp(int ncurve, int nw, OmegaArr om,
                                                const double2* __restrict__ sigma,
                                                const double* __restrict__ sign,
                                                const double* __restrict__ theta_init,
                                                double* __restrict__ params,
                                                double* __restrict__ cost_out,
                                                int* __restrict__ iters_out,
                                                int* __restrict__ status_out, int keep_better) {
  __shared__ LmWarpSmem S;
  const int cidx = blockIdx.x;
  const int lane = threadIdx.x;
  if (cidx >= ncurve) return;
  const double2* y = sigma + size_t(cidx) * nw;
  constexpr int npole = NPOLE;
  constexpr int P = 4 * npole;
  constexpr int NP = P * (P + 1) / 2;
  double2 yl[2];
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    yl[h] = j < nw ? y[j] : make_double2(0.0, 0.0);
  }
  if (lane == 0) {
    if (theta_init) {
      for (int k = 0; k < P; ++k) S.th[k] = theta_init[size_t(cidx) * P + k];
    } else {
      const double s = sign ? (sign[cidx] >= 0.0 ? 1.0 : -1.0) : 1.0;
      lm_default_start(om.v, y, nw, npole, s, S.th);
    }
  }
  __syncwarp();
  double th[P], thn[P];
  for (int k = 0; k < P; ++k) th[k] = S.th[k];
  const double cscale = 0.5 * warp_sum(yl[0].x * yl[0].x + yl[0].y * yl[0].y +
                                       yl[1].x * yl[1].x + yl[1].y * yl[1].y);
  double C = warp_cost(om.v, yl, nw, npole, th);
  // the packed entries e = lane + 32 h of A this lane sums: row ea[h], column eb[h]
  constexpr int EPL = (NP + 31) / 32;
  int ea[EPL], eb[EPL];
#pragma unroll
  for (int h = 0; h < EPL; ++h) {
    const int e = lane + 32 * h;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    ea[h] = a;
    eb[h] = e - a * (a + 1) / 2;
  }
  double mu = -1.0;
  int it = 0, st = 1;
  for (; it < LM_MAXIT; ++it) {
    if (C <= LM_CTOL * cscale) {
      st = 0;
      break;
    }
    // Jacobian rows and residuals of this lane's points
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j >= nw) break;
      double fx = 0.0, fy = 0.0;
      for (int p = 0; p < npole; ++p) {
        const double ax = th[4 * p], ay = th[4 * p + 1];
        const double dx = -th[4 * p + 2], dy = om.v[j] - th[4 * p + 3];
        const double inv = 1.0 / (dx * dx + dy * dy);
        const double px = dx * inv, py = -dy * inv;        // phi
        const double tx = ax * px - ay * py, ty = ax * py + ay * px;   // a phi
        fx += tx;
        fy += ty;
        const double qx = tx * px - ty * py, qy = tx * py + ty * px;   // a phi^2
        // d f / d Re a = phi, d f / d Im a = i phi, d f / d Re w = a phi^2, d f / d Im w = i a phi^2
        S.rowR[j][4 * p] = px;
        S.rowI[j][4 * p] = py;
        S.rowR[j][4 * p + 1] = -py;
        S.rowI[j][4 * p + 1] = px;
        S.rowR[j][4 * p + 2] = qx;
        S.rowI[j][4 * p + 2] = qy;
        S.rowR[j][4 * p + 3] = -qy;
        S.rowI[j][4 * p + 3] = qx;
      }
      S.res[j][0] = fx - yl[h].x;
      S.res[j][1] = fy - yl[h].y;
    }
    __syncwarp();
    // A (packed lower) and g, summed over points
#pragma unroll
    for (int h = 0; h < EPL; ++h) {
      const int e = lane + 32 * h;
      if (e >= NP) break;
      const int a = ea[h], bcol = eb[h];
      double v = 0.0;
      for (int j = 0; j < nw; ++j) v += S.rowR[j][a] * S.rowR[j][bcol] + S.rowI[j][a] * S.rowI[j][bcol];
      S.A[e] = v;
    }
    if (lane < P) {
      double v = 0.0;
      for (int j = 0; j < nw; ++j) v += S.rowR[j][lane] * S.res[j][0] + S.rowI[j][lane] * S.res[j][1];
      S.g[lane] = v;
    }
    __syncwarp();
    double gm = 0.0, dm = 0.0;
    if (lane < P) {
      gm = fabs(S.g[lane]);
      dm = S.A[lane * (lane + 1) / 2 + lane];
    }
    gm = warp_max(gm);
    dm = warp_max(dm);
    if (gm <= LM_GTOL) {
      st = 0;
      break;
    }
    if (mu < 0.0) mu = 1e-3 * dm;
    double Cn = 0.0;
    bool give_up = false;
    while (true) {
      for (int e = lane; e < NP; e += 32) S.Ld[e] = S.A[e];
      __syncwarp();
      if (lane < P) {
        S.Ld[lane * (lane + 1) / 2 + lane] += mu * S.A[lane * (lane + 1) / 2 + lane];
        S.b[lane] = -S.g[lane];
      }
      if (lane == 0) S.flag = 1;
      __syncwarp();
      // Cholesky, column by column: the pivot by lane 0, the rows below it by lanes
      for (int jc = 0; jc < P; ++jc) {
        if (lane == 0) {
          double d = S.Ld[jc * (jc + 1) / 2 + jc];
          for (int k = 0; k < jc; ++k) d -= S.Ld[jc * (jc + 1) / 2 + k] * S.Ld[jc * (jc + 1) / 2 + k];
          if (!(d > 0.0)) S.flag = 0;
          const double r = d > 0.0 ? sqrt(d) : 1.0;
          S.Ld[jc * (jc + 1) / 2 + jc] = r;
          S.dinv[jc] = 1.0 / r;
        }
        __syncwarp();
        const int i = jc + 1 + lane;
        if (i < P) {
          double v = S.Ld[i * (i + 1) / 2 + jc];
          for (int k = 0; k < jc; ++k) v -= S.Ld[i * (i + 1) / 2 + k] * S.Ld[jc * (jc + 1) / 2 + k];
          S.Ld[i * (i + 1) / 2 + jc] = v * S.dinv[jc];
        }
        __syncwarp();
      }
      const bool ok = S.flag != 0;
      if (ok) {
        // L z = b by column sweeps, then L^T x = z
        for (int k = 0; k < P; ++k) {
          const double zk = S.b[k] * S.dinv[k];
          __syncwarp();
          const int i = k + 1 + lane;
          if (i < P) S.b[i] -= S.Ld[i * (i + 1) / 2 + k] * zk;
          if (lane == 0) S.b[k] = zk;
          __syncwarp();
        }
        for (int k = P - 1; k >= 0; --k) {
          const double xk = S.b[k] * S.dinv[k];
          __syncwarp();
          if (lane < k) S.b[lane] -= S.Ld[k * (k + 1) / 2 + lane] * xk;
          if (lane == 0) S.b[k] = xk;
          __syncwarp();
        }
        for (int k = 0; k < P; ++k) thn[k] = th[k] + S.b[k];
        Cn = warp_cost(om.v, yl, nw, npole, thn);
      }
      if (ok && Cn < C) {
        mu = fmax(mu / 10.0, LM_MU_MIN);
        break;
      }
      mu *= 10.0;
      if (mu > LM_MU_MAX) {
        give_up = true;
        break;
      }
    }
    if (give_up) {
      st = 2;
      break;
    }
    const double dec = C - Cn, Cold = C;
    for (int k = 0; k < P; ++k) th[k] = thn[k];
    C = Cn;
    if (dec <= LM_FTOL * Cold) {
      st = 0;
      ++it;
      break;
    }
  }
  if (lane != 0) return;
  if (keep_better) {
    // compare with the result already stored (the other start) and keep the lower cost
    if (!(C < cost_out[cidx])) return;
  }
  for (int k = 0; k < P; ++k) params[size_t(cidx) * P + k] = th[k];
  cost_out[cidx] = C;
  iters_out[cidx] = it;
  status_out[cidx] = st;
}

int launch_lm(int ncurve, int nw, const OmegaArr& om, const double* sigma, const double* sign,
              int npole, const double* theta_init, double* params, double* cost, int* iters,
              int* status, int keep_better, cudaStream_t s) {
  if (ncurve == 0) return GW_OK;
  if (nw > LM_WMAXNW) return set_error(GW_EINVAL, "the fit takes at most %d frequencies", LM_WMAXNW);
  const double2* y = reinterpret_cast<const double2*>(sigma);
  auto go = [&](auto kern) {
    kern<<<ncurve, 32, 0, s>>>(ncurve, nw, om, y, sign, theta_init, params, cost, iters, status,
                               keep_better);
  };
  switch (npole) {
    case 1: go(k_lm_warp<1>); break;
    case 2: go(k_lm_warp<2>); break;
    case 3: go(k_lm_warp<3>); break;
    case 4: go(k_lm_warp<4>); break;
    default: go(k_lm_warp<5>); break;
  }
  GW_LAUNCH_CHECK("k_lm_warp");
  return GW_OK;
}

}  // namespace gw
