// a4: q = Gamma head and wings in FP64 (Sec. III.D: Eqs. polar_Gamma and screen_Gamma and
// the expressions after them, the l = 0 coefficient of the head's angular expansion,
// Eq. correlation_div with the BZ constant in the erf form derived for the exchange term).
//
// Input: the polarization of the augmented projections [p | M] (three k.p columns first),
// P_aug [nw][nb+3][nb+3], so that H = P_aug[:3,:3] (head), s_nu = P_aug[:3, 3+nu] (wing),
// P~ = P_aug[3:,3:] (body). Steps per frequency:
//   1. W~^c from P~ by the FP64 dielectric kernel (the a3 step);
//   2. u_nu = sum_mu s_mu W~_mu,nu (W~ = W~^c + diag v), L = 1 - 4 pi H - 4 pi sum_nu u_nu s_nu^H;
//   3. over the unit sphere (Gauss-Legendre in cos theta x uniform phi, exact for the
//      smooth integrand to rounding at the default order): <1/e^T L e> and
//      A_ab = <e_a e_b / e^T L e>; K^c_00 = sqrt(4 pi) 4 pi <1/e^T L e> - (4 pi)^(3/2);
//   4. body: W~^c_mu,nu += 4 pi sum_ab conj(u_mu,a) A_ab u_nu,b (the l = 0 part of the
//      rank-one term of Eq. screen_Gamma).
// The head and wing expressions are those of the exact block inverse of the full problem
// (the printed wing carries sqrt(v_nu) differently; for real data the two agree).
#include <algorithm>
#include <cmath>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr double FOUR_PI = 12.566370614359172;
constexpr int NTH = 64;          // Gauss-Legendre nodes in cos(theta)
constexpr int NPH = 128;         // uniform nodes in phi
constexpr int GTHREADS = 256;

struct SphereRule {
  double x[NTH];
  double w[NTH];
};

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n (three-term
// recurrence), started from the asymptotic node estimates; weights 2 / ((1 - x^2) P_n'(x)^2).
SphereRule make_rule() {
  SphereRule r{};
  const int n = NTH;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r.x[i] = x;
    r.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return r;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// P~ (rows and columns 3..nb+2 of P_aug) into Wc (the dielectric then works in place).
__global__ void k_gamma_extract(int nb, int nw, const double2* __restrict__ Paug,
                                double2* __restrict__ Wc) {
  const int na = nb + 3;
  const size_t total = size_t(nw) * nb * nb;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total;
       e += size_t(gridDim.x) * blockDim.x) {
    const size_t j = e / (size_t(nb) * nb);
    const int r = int((e / nb) % nb), c = int(e % nb);
    Wc[e] = Paug[(j * na + 3 + r) * na + 3 + c];
  }
}

// One CTA per frequency: u, L, the sphere moments, K^c_00 and A (to scratch).
__global__ void __launch_bounds__(GTHREADS) k_gamma_head(int nb, const double* __restrict__ v,
                                                         const double2* __restrict__ Paug,
                                                         const double2* __restrict__ Wc,
                                                         const SphereRule rule,
                                                         double2* __restrict__ u_out,
                                                         double2* __restrict__ L_out,
                                                         double* __restrict__ head_out,
                                                         double* __restrict__ A_out,
                                                         unsigned* status) {
  const int j = blockIdx.x;
  const int na = nb + 3;
  const double2* P = Paug + size_t(j) * na * na;
  const double2* W = Wc + size_t(j) * nb * nb;
  double2* u = u_out + size_t(j) * nb * 3;
  __shared__ double red[GTHREADS][7];
  __shared__ double2 Lsh[9];
  // u_nu,a = sum_mu s_mu,a W~_mu,nu  (thread per nu; column sweep of W, coalesced over nu)
  for (int nu = threadIdx.x; nu < nb; nu += blockDim.x) {
    double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int mu = 0; mu < nb; ++mu) {
      double2 w = W[size_t(mu) * nb + nu];
      if (mu == nu) w.x += v[mu];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double2 s = P[size_t(a) * na + 3 + mu];
        const double2 t = cmul(s, w);
        acc[a].x += t.x;
        acc[a].y += t.y;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) u[size_t(nu) * 3 + a] = acc[a];
  }
  __syncthreads();
  // L_ab = delta_ab - 4 pi H_ab - 4 pi sum_nu u_nu,a conj(s_nu,b)
  for (int ab = 0; ab < 9; ++ab) {
    const int a = ab / 3, b = ab % 3;
    double re = 0.0, im = 0.0;
    for (int nu = threadIdx.x; nu < nb; nu += blockDim.x) {
      const double2 t = cmulc(u[size_t(nu) * 3 + a], P[size_t(b) * na + 3 + nu]);
      re += t.x;
      im += t.y;
    }
    red[threadIdx.x][0] = re;
    red[threadIdx.x][1] = im;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        red[threadIdx.x][0] += red[threadIdx.x + st][0];
        red[threadIdx.x][1] += red[threadIdx.x + st][1];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double2 h = P[size_t(a) * na + b];
      Lsh[ab] = make_double2((a == b ? 1.0 : 0.0) - FOUR_PI * h.x - FOUR_PI * red[0][0],
                             -FOUR_PI * h.y - FOUR_PI * red[0][1]);
    }
    __syncthreads();
  }
  // sphere moments of 1 / e^T L e (e real: e^T L e = e^T Re(L) e)
  double Lr[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Lr[k] = Lsh[k].x;
  double m[7] = {0, 0, 0, 0, 0, 0, 0};       // <1/s>, A_xx, A_yy, A_zz, A_xy, A_xz, A_yz
  const double dphi = 2.0 * M_PI / NPH;
  for (int idx = threadIdx.x; idx < NTH * NPH; idx += blockDim.x) {
    const int it = idx / NPH, ip = idx % NPH;
    const double x = rule.x[it];
    const double st = sqrt(fmax(0.0, 1.0 - x * x));
    double sp, cp;
    sincos(dphi * ip, &sp, &cp);
    const double e0 = st * cp, e1 = st * sp, e2 = x;
    const double sig = e0 * (Lr[0] * e0 + Lr[1] * e1 + Lr[2] * e2) +
                       e1 * (Lr[3] * e0 + Lr[4] * e1 + Lr[5] * e2) +
                       e2 * (Lr[6] * e0 + Lr[7] * e1 + Lr[8] * e2);
    if (!(sig > 0.0)) raise_status(status, ST_EINVAL);
    const double f = rule.w[it] * dphi / sig;
    m[0] += f;
    m[1] += f * e0 * e0;
    m[2] += f * e1 * e1;
    m[3] += f * e2 * e2;
    m[4] += f * e0 * e1;
    m[5] += f * e0 * e2;
    m[6] += f * e1 * e2;
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) red[threadIdx.x][k] = m[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < 7; ++k) red[threadIdx.x][k] += red[threadIdx.x + st][k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double inv4pi = 1.0 / FOUR_PI;
    const double avg = red[0][0] * inv4pi;
    head_out[j] = sqrt(FOUR_PI) * FOUR_PI * avg - FOUR_PI * sqrt(FOUR_PI);
    double* A = A_out + size_t(j) * 9;
    A[0] = red[0][1] * inv4pi;
    A[4] = red[0][2] * inv4pi;
    A[8] = red[0][3] * inv4pi;
    A[1] = A[3] = red[0][4] * inv4pi;
    A[2] = A[6] = red[0][5] * inv4pi;
    A[5] = A[7] = red[0][6] * inv4pi;
    if (L_out)
      for (int k = 0; k < 9; ++k) L_out[size_t(j) * 9 + k] = Lsh[k];
  }
}

// Body: W~^c_mu,nu += 4 pi conj(u_mu)^T A u_nu; one CTA per (row mu, frequency).
__global__ void k_gamma_body(int nb, const double2* __restrict__ u_all, const double* __restrict__ A_all,
                             double2* __restrict__ Wc) {
  const int mu = blockIdx.x, j = blockIdx.y;
  const double2* u = u_all + size_t(j) * nb * 3;
  const double* A = A_all + size_t(j) * 9;
  double2 um[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) um[a] = make_double2(u[size_t(mu) * 3 + a].x, -u[size_t(mu) * 3 + a].y);
  double2* row = Wc + (size_t(j) * nb + mu) * nb;
  for (int nu = threadIdx.x; nu < nb; nu += blockDim.x) {
    double2 acc = make_double2(0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const double2 ub = u[size_t(nu) * 3 + b];
      double2 au = make_double2(0, 0);          // sum_a conj(u_mu,a) A_ab
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        au.x += um[a].x * A[a * 3 + b];
        au.y += um[a].y * A[a * 3 + b];
      }
      const double2 t = cmul(au, ub);
      acc.x += t.x;
      acc.y += t.y;
    }
    double2 w = row[nu];
    w.x += FOUR_PI * acc.x;
    w.y += FOUR_PI * acc.y;
    row[nu] = w;
  }
}

// Lattice sum of e^{-beta q^2} / q^2 over 0 < |q| < q0, q = dq * (i, j, k) (simple cubic),
// one partial sum per CTA.
__global__ void k_bz_sum(int m, double dq, double beta, double q0, double* __restrict__ part) {
  __shared__ double red[256];
  const int64_t side = 2 * int64_t(m) + 1;
  const int64_t total = side * side;          // (i, j) columns; each thread sweeps k
  double acc = 0.0;
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < total;
       c += int64_t(gridDim.x) * blockDim.x) {
    const double qx = dq * double(c / side - m), qy = dq * double(c % side - m);
    const double r2 = qx * qx + qy * qy;
    if (r2 >= q0 * q0) continue;
    const int kmax = int(floor(sqrt(q0 * q0 - r2) / dq));
    for (int k = -kmax; k <= kmax; ++k) {
      const double qz = dq * k;
      const double q2 = r2 + qz * qz;
      if (q2 > 0.0 && q2 < q0 * q0) acc += exp(-beta * q2) / q2;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// c[j][s] = head[j] for every state s; pair_state[s] = s.
__global__ void k_div_pairs(int nw, int nsig, const double* __restrict__ head, double* __restrict__ c,
                            int* __restrict__ state) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nw * nsig) c[i] = head[i / nsig];
  if (i < nsig) state[i] = i;
}

const SphereRule& rule() {
  static const SphereRule r = make_rule();
  return r;
}

}  // namespace

size_t gamma_workspace(int nb, int nw) {
  return dielectric_workspace(1, &nb, nw) + ws_round(size_t(nw) * 9 * sizeof(double)) +
         ws_round(size_t(nw) * nb * 3 * sizeof(double2)) + 256;
}

int gamma_screened_w(int nb, int nw, const double* v, const double* Paug, double* Wc,
                     double* head, double* L, double* u_out, void* ws, size_t ws_bytes,
                     cudaStream_t s, const DeviceCtx& ctx) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  const size_t dws = dielectric_workspace(1, &nb, nw);
  void* dws_ptr = cur.take(dws);
  double* A = static_cast<double*>(cur.take(size_t(nw) * 9 * sizeof(double)));
  double2* u = u_out ? reinterpret_cast<double2*>(u_out)
                     : static_cast<double2*>(cur.take(size_t(nw) * nb * 3 * sizeof(double2)));
  if ((dws && !dws_ptr) || !A || !u) return set_error(GW_EWORKSPACE, "gamma workspace too small");
  const size_t total = size_t(nw) * nb * nb;
  const unsigned g = unsigned(std::min<size_t>((total + 255) / 256, size_t(ctx.sm_count) * 8));
  k_gamma_extract<<<g, 256, 0, s>>>(nb, nw, reinterpret_cast<const double2*>(Paug),
                                    reinterpret_cast<double2*>(Wc));
  GW_LAUNCH_CHECK("k_gamma_extract");
  const double* Wcc = Wc;
  int rc = dielectric_wc(1, &nb, nw, &v, &Wcc, &Wc, dws_ptr, dws, s, ctx);
  if (rc) return rc;
  k_gamma_head<<<nw, GTHREADS, 0, s>>>(nb, v, reinterpret_cast<const double2*>(Paug),
                                       reinterpret_cast<const double2*>(Wc), rule(), u,
                                       reinterpret_cast<double2*>(L), head, A, ctx.status);
  GW_LAUNCH_CHECK("k_gamma_head");
  k_gamma_body<<<dim3(nb, nw), 128, 0, s>>>(nb, u, A, reinterpret_cast<double2*>(Wc));
  GW_LAUNCH_CHECK("k_gamma_body");
  return GW_OK;
}

size_t bz_constant_workspace(const DeviceCtx& ctx) {
  return ws_round(sizeof(double) * size_t(ctx.sm_count) * 4);
}

int bz_constant_sc(double a, int n, double beta, double* out, void* ws, size_t ws_bytes,
                   cudaStream_t s, const DeviceCtx& ctx) {
  const double V = std::pow(double(n) * a, 3.0);
  const double q0 = std::sqrt(-std::log(beta) / beta);
  const double dq = 2.0 * M_PI / (double(n) * a);
  const int m = int(std::floor(q0 / dq));
  const int blocks = ctx.sm_count * 4;
  if (!ws || ws_bytes < sizeof(double) * size_t(blocks))
    return set_error(GW_EWORKSPACE, "BZ constant workspace too small");
  double* part = static_cast<double*>(ws);
  k_bz_sum<<<blocks, 256, 0, s>>>(m, dq, beta, q0, part);
  GW_LAUNCH_CHECK("k_bz_sum");
  std::vector<double> h(blocks);
  GW_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
  GW_CUDA_TRY(cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double x : h) sum += x;
  *out = V / FOUR_PI * std::erf(std::sqrt(beta) * q0) / std::sqrt(M_PI * beta) - sum;
  return GW_OK;
}

size_t sigma_div_workspace(int nw, int nsig) {
  const int64_t np = nsig;
  return ws_round(size_t(nw) * nsig * sizeof(double)) + ws_round(size_t(nsig) * sizeof(int)) + 256 +
         convolve_workspace(1, &np, nw, 0);
}

int sigma_div(int nw, const OmegaArr& om, const double* head, double cbz, double volume, int nsig,
              const double* eps_state, int nw_out, const OmegaArr& om_out, double* sigma,
              void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  double* c = static_cast<double*>(cur.take(size_t(nw) * nsig * sizeof(double)));
  int* st = static_cast<int*>(cur.take(size_t(nsig) * sizeof(int)));
  if (!c || !st) return set_error(GW_EWORKSPACE, "sigma_div workspace too small");
  k_div_pairs<<<(nw * nsig + 255) / 256, 256, 0, s>>>(nw, nsig, head, c, st);
  GW_LAUNCH_CHECK("k_div_pairs");
  // the convolution's -1/(2 pi) w times the integral equals -C / (4 pi^(3/2) V) times it
  const double wq = cbz / (2.0 * std::sqrt(M_PI) * volume);
  const int64_t np = nsig;
  const double* cc = c;
  const int* sc = st;
  const size_t used = (cur.used + 255) & ~size_t(255);
  return convolve_acc(1, &wq, &np, nw, om, &cc, &sc, &eps_state, nw_out, om_out, nsig, sigma, true,
                      static_cast<char*>(ws) + used, ws_bytes - used, s, ctx);
}

}  // namespace gw
