// a5 pair coefficients and a6 frequency convolution of the correlation self-energy
// (Eq. SEc_AC and the paragraph after it).
//
// a5 (FP64 path): for each (q, frequency) the CTA tile computes
//   Y[p][I] = sum_J m[p][J] W^c[I][J]      (64 pairs x 64 basis functions)
// and folds it at once into c_p += Re sum_I conj(m[p][I]) Y[p][I]; partial sums per
// I-tile are reduced in a fixed order.
//
// a6: the node values c_j of each pair are interpolated by a cubic spline in
// lambda = w/(1+w); with w(lambda) = lambda/(1-lambda) the kernel of the w' integral,
//   [g(w+w') + g(w-w')] dw'/dlambda,  g(x) = 1/(i x - e),
// reduces by partial fractions to K(lambda) = -i b+/(A + b+ lambda) + i b-/(A + b- lambda)
// with A = i w - e and b(+-) = +-i - A (the 1/(1-lambda) parts cancel between the two
// terms). Each spline piece times K is integrated in closed form (moments of
// 1/(z0 + b t), by series when the pole is far and by recurrence from the complex
// logarithm otherwise), and the tail c_N w_N^2 / w'^2 beyond the last node likewise.
#include <vector>
#include <algorithm>

#include "gw_internal.cuh"

namespace gw {

// ------------------------------------------------------------------ a5 -------
constexpr int ST = 64;   // pair / basis tile
constexpr int SKC = 8;   // J chunk
constexpr int SMAXQ = 64;

struct PairLaunch {
  const double2* M[SMAXQ];
  const double2* W[SMAXQ];
  int64_t npair[SMAXQ];
  int nb[SMAXQ];
  int ptiles[SMAXQ];
  int itiles[SMAXQ];
  int64_t blk0[SMAXQ + 1];   // first block of q: blocks ordered (j, ptile, itile)
  size_t part0[SMAXQ];       // first partial double of q
  int nq;
  int nw;
};

__global__ void __launch_bounds__(256) k_paircoef_fp64(PairLaunch L, double* __restrict__ part) {
  int64_t blk = blockIdx.x;
  int q = 0;
  while (q + 1 < L.nq && blk >= L.blk0[q + 1]) ++q;
  int64_t loc = blk - L.blk0[q];
  const int it = int(loc % L.itiles[q]);
  loc /= L.itiles[q];
  const int pt = int(loc % L.ptiles[q]);
  const int j = int(loc / L.ptiles[q]);
  const int nb = L.nb[q];
  const int64_t np = L.npair[q];
  const double2* __restrict__ M = L.M[q];
  const double2* __restrict__ W = L.W[q] + size_t(j) * nb * nb;

  __shared__ double2 As[SKC][ST + 1];   // As[k][p] = m[p0+p][J0+k]
  __shared__ double2 Bs[SKC][ST + 1];   // Bs[k][i] = W[I0+i][J0+k]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t p0 = int64_t(pt) * ST;
  const int I0 = it * ST;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);

  for (int J0 = 0; J0 < nb; J0 += SKC) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int e = tid + 256 * r;
      int row = e >> 3, k = e & 7;
      int J = J0 + k;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (J < nb) {
        if (p0 + row < np) a = M[(p0 + row) * nb + J];
        if (I0 + row < nb) b = W[size_t(I0 + row) * nb + J];
      }
      As[k][row] = a;
      Bs[k][row] = b;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SKC; ++k) {
      double2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // Y[p][I] += m[p][J] * W[I][J]
          acc[a][b].x = fma(av[a].x, bv[b].x, fma(-av[a].y, bv[b].y, acc[a][b].x));
          acc[a][b].y = fma(av[a].x, bv[b].y, fma(av[a].y, bv[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
  }
  // c_p partial = Re sum_I conj(m[p][I]) Y[p][I]
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int64_t p = p0 + ty + 16 * a;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int I = I0 + tx + 16 * b;
      if (p < np && I < nb) {
        double2 m = M[p * nb + I];
        s = fma(m.x, acc[a][b].x, fma(m.y, acc[a][b].y, s));
      }
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (tx == 0 && p < np) part[L.part0[q] + (size_t(j) * L.itiles[q] + it) * np + p] = s;
  }
}

__global__ void k_paircoef_reduce(PairLaunch L, const double* __restrict__ part,
                                  double* const* __restrict__ cout_unused, double* c0, int q,
                                  int64_t np, int itiles, size_t part0, int nw) {
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= np * nw) return;
  int j = int(e / np);
  int64_t p = e % np;
  double s = 0.0;
  for (int it = 0; it < itiles; ++it) s += part[part0 + (size_t(j) * itiles + it) * np + p];
  c0[size_t(j) * np + p] = s;
}

size_t paircoef_workspace(int nq, const int64_t* npair, const int* nb, int nw, int precision) {
  if (precision != GW_FP64) return quad_tc_workspace(nq, npair, nb, nw, precision);
  size_t b = 0;
  for (int q = 0; q < nq; ++q) {
    int it = (nb[q] + ST - 1) / ST;
    b += size_t(nw) * it * size_t(npair[q]);
  }
  return ws_round(b * sizeof(double));
}

int paircoef(int nq, const int64_t* npair, const int* nb, const void* const* Msig, int dtype,
             int nw, const double* const* Wc, double* const* c, int precision, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  if (precision != GW_FP64)
    return quad_tc(nq, npair, nb, Msig, nw, Wc, c, precision, dtype == GW_R32, ws, ws_bytes, s,
                   ctx);
  double* part = static_cast<double*>(ws);
  for (int q0 = 0; q0 < nq; q0 += SMAXQ) {
    int n = std::min(SMAXQ, nq - q0);
    PairLaunch L{};
    L.nq = n;
    L.nw = nw;
    int64_t blk = 0;
    size_t p0 = 0;
    for (int q = 0; q < n; ++q) {
      int Q = q0 + q;
      L.M[q] = static_cast<const double2*>(Msig[Q]);
      L.W[q] = reinterpret_cast<const double2*>(Wc[Q]);
      L.npair[q] = npair[Q];
      L.nb[q] = nb[Q];
      L.ptiles[q] = int((npair[Q] + ST - 1) / ST);
      L.itiles[q] = (nb[Q] + ST - 1) / ST;
      L.blk0[q] = blk;
      L.part0[q] = p0;
      blk += int64_t(nw) * L.ptiles[q] * L.itiles[q];
      p0 += size_t(nw) * L.itiles[q] * size_t(npair[Q]);
    }
    L.blk0[n] = blk;
    if (blk > 0) {
      k_paircoef_fp64<<<unsigned(blk), 256, 0, s>>>(L, part);
      GW_LAUNCH_CHECK("k_paircoef_fp64");
    }
    for (int q = 0; q < n; ++q) {
      int64_t np = L.npair[q];
      if (np == 0) continue;
      int64_t tot = np * nw;
      k_paircoef_reduce<<<unsigned((tot + 255) / 256), 256, 0, s>>>(
          L, part, nullptr, c[q0 + q], q, np, L.itiles[q], L.part0[q], nw);
      GW_LAUNCH_CHECK("k_paircoef_reduce");
    }
  }
  return GW_OK;
}

// ------------------------------------------------------------------ a6 -------
struct cplx {
  double x, y;
};
__device__ __forceinline__ cplx mk(double x, double y) { return cplx{x, y}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ cplx operator*(double s, cplx a) { return mk(s * a.x, s * a.y); }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
__device__ __forceinline__ double cabs_(cplx a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cplx clog_(cplx a) { return mk(log(hypot(a.x, a.y)), atan2(a.y, a.x)); }

// 1/k for k = 1..60 (the series below multiply by these instead of dividing)
__constant__ double kInvInt[60] = {1.0, 0.5, 0.3333333333333333, 0.25, 0.2, 0.16666666666666666, 0.14285714285714285, 0.125, 0.1111111111111111, 0.1, 0.09090909090909091, 0.08333333333333333, 0.07692307692307693, 0.07142857142857142, 0.06666666666666667, 0.0625, 0.058823529411764705, 0.05555555555555555, 0.05263157894736842, 0.05, 0.047619047619047616, 0.045454545454545456, 0.043478260869565216, 0.041666666666666664, 0.04, 0.038461538461538464, 0.037037037037037035, 0.03571428571428571, 0.034482758620689655, 0.03333333333333333, 0.03225806451612903, 0.03125, 0.030303030303030304, 0.029411764705882353, 0.02857142857142857, 0.027777777777777776, 0.02702702702702703, 0.02631578947368421, 0.02564102564102564, 0.025, 0.024390243902439025, 0.023809523809523808, 0.023255813953488372, 0.022727272727272728, 0.022222222222222223, 0.021739130434782608, 0.02127659574468085, 0.020833333333333332, 0.02040816326530612, 0.02, 0.0196078431372549, 0.019230769230769232, 0.018867924528301886, 0.018518518518518517, 0.01818181818181818, 0.017857142857142856, 0.017543859649122806, 0.017241379310344827, 0.01694915254237288, 0.016666666666666666};

constexpr double SERIES_R = 0.3;
constexpr int SERIES_N = 36;

// I_k = int_0^H t^k / (z0 + b t) dt, k = 0..3
__device__ void moments(cplx z0, cplx b, double H, cplx I[4]) {
  cplx r = cdiv(H * b, z0);
  if (cabs_(r) < SERIES_R) {
    cplx term = mk(1.0, 0.0);
    cplx nr = mk(-r.x, -r.y);
    cplx s0 = mk(0, 0), s1 = mk(0, 0), s2 = mk(0, 0), s3 = mk(0, 0);
    const double rr = cabs_(r);
    double tmag = 1.0;
    for (int m = 0; m < SERIES_N; ++m) {
      s0 = s0 + kInvInt[m] * term;
      s1 = s1 + kInvInt[m + 1] * term;
      s2 = s2 + kInvInt[m + 2] * term;
      s3 = s3 + kInvInt[m + 3] * term;
      term = term * nr;
      tmag *= rr;
      if (tmag < 1e-18) break;     // |r|^(m+1) below the FP64 resolution of the sums (>= 1/4)
    }
    cplx iz = cdiv(mk(1.0, 0.0), z0);
    double h1 = H, h2 = H * H, h3 = h2 * H, h4 = h3 * H;
    I[0] = h1 * (s0 * iz);
    I[1] = h2 * (s1 * iz);
    I[2] = h3 * (s2 * iz);
    I[3] = h4 * (s3 * iz);
  } else {
    cplx ib = cdiv(mk(1.0, 0.0), b);
    I[0] = clog_(mk(1.0 + r.x, r.y)) * ib;
    double hk = 1.0;
    for (int k = 1; k < 4; ++k) {
      hk *= H;
      I[k] = (mk(hk / k, 0.0) - z0 * I[k - 1]) * ib;
    }
  }
}

// int_X^inf dx / (x^2 (A + i s x))
__device__ cplx tail_integral(cplx A, double sgn, double X) {
  cplx isg = mk(0.0, sgn);
  cplx rho = cdiv(A, mk(0.0, sgn * X));
  if (cabs_(rho) < 0.5) {
    cplx term = mk(1.0, 0.0), nr = mk(-rho.x, -rho.y), s = mk(0, 0);
    const double rr = cabs_(rho);
    double tmag = 1.0;
    for (int m = 0; m < 56; ++m) {
      s = s + kInvInt[m + 1] * term;
      term = term * nr;
      tmag *= rr;
      if (tmag < 1e-18) break;     // |rho|^(m+1) below the FP64 resolution of the sum (>= 1/2)
    }
    return cdiv(s, mk(0.0, sgn * X * X));
  }
  cplx a2 = A * A;
  cplx zx = mk(A.x / X, A.y / X + sgn);
  cplx L = clog_(cdiv(isg, zx));
  return cdiv(mk(1.0, 0.0), mk(A.x * X, A.y * X)) + cdiv(isg * L, a2);
}

// Coefficients C[k] (k = 0..3, powers of t = lambda - la) of spline piece s for the node values
// y: piece 0 is [0, lam_0] (segment 0 extrapolated, re-centred at lambda = 0), piece s >= 1 is
// segment s - 1. Slopes: not-a-knot at the first node, clamped at the last to the tail's
// dc/dw = -2 c_N / w_N (dc/dlambda = -2 c_N (1 + w_N)^2 / w_N).
__device__ void spline_slopes(const double* y, int n, const double* h, double wN, double* m,
                              double* cp) {
  double d0 = (y[1] - y[0]) / h[0], d1 = (y[2] - y[1]) / h[1];
  double b0 = h[1], c0 = h[0] + h[1];
  double r0 = ((2.0 * h[1] + 3.0 * h[0]) * h[1] * d0 + h[0] * h[0] * d1) / (h[0] + h[1]);
  cp[0] = c0 / b0;
  m[0] = r0 / b0;
  for (int i = 1; i < n - 1; ++i) {
    double dl = (y[i] - y[i - 1]) / h[i - 1], dr = (y[i + 1] - y[i]) / h[i];
    double a = h[i], b = 2.0 * (h[i - 1] + h[i]), cc = h[i - 1];
    double r = 3.0 * (h[i] * dl + h[i - 1] * dr);
    double den = b - a * cp[i - 1];
    cp[i] = cc / den;
    m[i] = (r - a * m[i - 1]) / den;
  }
  double sig = -2.0 * (1.0 + wN) * (1.0 + wN) / wN;
  m[n - 1] = sig * y[n - 1];
  for (int i = n - 2; i >= 0; --i) m[i] = m[i] - cp[i] * m[i + 1];
}

__device__ void piece_coeffs(const double* y, const double* m, const double* lam, const double* h,
                             int s, double C[4]) {
  const int g = s == 0 ? 0 : s - 1;
  const double dlt = (y[g + 1] - y[g]) / h[g];
  C[0] = y[g];
  C[1] = m[g];
  C[2] = (3.0 * dlt - 2.0 * m[g] - m[g + 1]) / h[g];
  C[3] = (m[g] + m[g + 1] - 2.0 * dlt) / (h[g] * h[g]);
  if (s == 0) {
    const double x0 = -lam[0];
    const double D0 = C[0] + x0 * (C[1] + x0 * (C[2] + x0 * C[3]));
    const double D1 = C[1] + x0 * (2.0 * C[2] + 3.0 * x0 * C[3]);
    const double D2 = C[2] + 3.0 * x0 * C[3];
    C[0] = D0;
    C[1] = D1;
    C[2] = D2;
  }
}

// Pairs with the same energy share the convolution weights T_ij(e): the spline is linear in the
// node values, so sum_j T_ij(e) c_j with T_ij = sum_{piece, k} K_{piece,k}(e, w_i) S_{piece,k,j}
// (S: the cardinal spline coefficients of the node mesh, K: the closed-form integrals of
// t^k against the kernel on the piece) plus the tail on the last node. The closed forms run
// once per distinct energy of a q point:
//   k_conv_init / k_conv_hash: every pair inserts the bit pattern of its energy into an
//     open-addressing table (atomicCAS), records its slot and counts the slot's pairs;
//   k_conv_scan: per q, the offsets of the slots' pair lists and the occupied slots;
//   k_conv_scatter: every pair writes its index into its slot's list;
//   k_conv_slot: one CTA per (occupied slot, 16 output frequencies): S (once per CTA), K (one
//     thread per output frequency and piece), T, then Sigma_s(i w_i) += w_q f sum_j T_ij c_jp
//     over the slot's pairs (FP64 atomics).
constexpr int CTHREADS = 256;
constexpr int CIC = 16;                       // output frequencies per slot CTA
constexpr unsigned long long EMPTY_KEY = ~0ull;   // a NaN pattern: never a valid energy

struct ConvQ {
  const double* c;        // [nw][npair]
  const int* state;
  const double* eps;
  int64_t npair;
  double wq;
  unsigned long long* keys;   // [tsize]
  int* cnt;                   // [tsize]
  int* off;                   // [tsize]
  int* fill;                  // [tsize]
  int* occ;                   // [tsize] occupied slots, compact
  int* nocc;                  // [1]
  int* slot_of;               // [npair]
  int* list;                  // [npair]
  int tsize;
};

struct ConvLaunch {
  ConvQ Q[SMAXQ];
  int64_t item0[SMAXQ + 1];   // prefix of pairs (hash, scatter) or of table slots (init)
  int nq;
};

__device__ __forceinline__ uint32_t mix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return uint32_t(k);
}

__device__ __forceinline__ int find_q(const ConvLaunch& L, int64_t e) {
  int q = 0;
  while (q + 1 < L.nq && e >= L.item0[q + 1]) ++q;
  return q;
}

__global__ void k_conv_init(ConvLaunch L) {
  const int64_t total = L.item0[L.nq];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int q = find_q(L, e);
    const int64_t i = e - L.item0[q];
    const ConvQ& Q = L.Q[q];
    Q.keys[i] = EMPTY_KEY;
    Q.cnt[i] = 0;
    Q.fill[i] = 0;
    if (i == 0) *Q.nocc = 0;
  }
}

__global__ void k_conv_hash(ConvLaunch L, int nsig, unsigned* status) {
  const int64_t total = L.item0[L.nq];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int q = find_q(L, e);
    const int64_t p = e - L.item0[q];
    const ConvQ& Q = L.Q[q];
    const double ep = Q.eps[p];
    const int st = Q.state[p];
    if (!(ep != 0.0) || !isfinite(ep) || st < 0 || st >= nsig) {
      raise_status(status, ST_EINVAL);
      Q.slot_of[p] = -1;
      continue;
    }
    const unsigned long long key = static_cast<unsigned long long>(__double_as_longlong(ep));
    const uint32_t mask = uint32_t(Q.tsize - 1);
    uint32_t h = mix64(key) & mask;
    // the table has at least twice as many slots as pairs: a free or matching slot exists
    for (int probe = 0; probe < Q.tsize; ++probe) {
      const unsigned long long prev = atomicCAS(Q.keys + h, EMPTY_KEY, key);
      if (prev == EMPTY_KEY || prev == key) break;
      h = (h + 1) & mask;
    }
    Q.slot_of[p] = int(h);
    atomicAdd(Q.cnt + h, 1);
  }
}

// one CTA of 1024 threads per q: exclusive scan of the counts (list offsets) and compaction of
// the occupied slots, in slot order
__global__ void __launch_bounds__(1024) k_conv_scan(ConvLaunch L) {
  const ConvQ& Q = L.Q[blockIdx.x];
  if (Q.npair == 0) return;
  __shared__ int sc[1024], so[1024];
  const int per = (Q.tsize + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(Q.tsize, b + per);
  int lc = 0, lo = 0;
  for (int i = b; i < e; ++i) {
    lc += Q.cnt[i];
    lo += Q.cnt[i] > 0;
  }
  sc[threadIdx.x] = lc;
  so[threadIdx.x] = lo;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {        // inclusive Hillis-Steele scan
    int vc = 0, vo = 0;
    if (threadIdx.x >= d) {
      vc = sc[threadIdx.x - d];
      vo = so[threadIdx.x - d];
    }
    __syncthreads();
    sc[threadIdx.x] += vc;
    so[threadIdx.x] += vo;
    __syncthreads();
  }
  int rc = sc[threadIdx.x] - lc, ro = so[threadIdx.x] - lo;
  for (int i = b; i < e; ++i) {
    Q.off[i] = rc;
    rc += Q.cnt[i];
    if (Q.cnt[i] > 0) Q.occ[ro++] = i;
  }
  if (threadIdx.x == 1023) *Q.nocc = so[1023];
}

__global__ void k_conv_scatter(ConvLaunch L) {
  const int64_t total = L.item0[L.nq];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int q = find_q(L, e);
    const int64_t p = e - L.item0[q];
    const ConvQ& Q = L.Q[q];
    const int h = Q.slot_of[p];
    if (h < 0) continue;
    Q.list[Q.off[h] + atomicAdd(Q.fill + h, 1)] = int(p);
  }
}

__global__ void __launch_bounds__(CTHREADS) k_conv_slot(ConvLaunch L, int nw, OmegaArr om,
                                                        OmegaArr om_out, int nw_out,
                                                        double* __restrict__ sigma) {
  extern __shared__ __align__(16) double csh[];
  const int n = nw;                                       // pieces
  double* S = csh;                                        // [n][4][nw]
  cplx* K = reinterpret_cast<cplx*>(S + 4 * n * nw);      // [CIC][n][4]
  cplx* T = K + CIC * n * 4;                              // [CIC][nw]
  cplx* tl = T + CIC * nw;                                // [CIC]
  __shared__ double lam[GW_MAX_NW], h[GW_MAX_NW];
  const int tid = threadIdx.x;
  if (tid < nw) lam[tid] = om.v[tid] / (1.0 + om.v[tid]);
  __syncthreads();
  if (tid < nw - 1) h[tid] = lam[tid + 1] - lam[tid];
  __syncthreads();
  const double wN = om.v[nw - 1];
  // cardinal spline coefficients: the spline of the unit node vector e_j, piece by piece
  for (int j = tid; j < nw; j += blockDim.x) {
    double y[GW_MAX_NW], m[GW_MAX_NW], cp[GW_MAX_NW];
    for (int i = 0; i < nw; ++i) y[i] = i == j ? 1.0 : 0.0;
    spline_slopes(y, n, h, wN, m, cp);
    for (int s = 0; s < n; ++s) {
      double C[4];
      piece_coeffs(y, m, lam, h, s, C);
      for (int k = 0; k < 4; ++k) S[(s * 4 + k) * nw + j] = C[k];
    }
  }
  __syncthreads();
  const double f = -1.0 / (2.0 * 3.14159265358979323846);
  const int nich = (nw_out + CIC - 1) / CIC;
  for (int q = 0; q < L.nq; ++q) {
    const ConvQ& Q = L.Q[q];
    if (Q.npair == 0) continue;
    const int64_t items = int64_t(*Q.nocc) * nich;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const int slot = Q.occ[it / nich];
      const int i0 = int(it % nich) * CIC;
      const int ni = min(CIC, nw_out - i0);
      const double e = __longlong_as_double(static_cast<long long>(Q.keys[slot]));
      // closed-form integrals of t^k against the kernel on every piece, and the tail
      for (int x = tid; x < ni * (n + 1); x += blockDim.x) {
        const int i = x / (n + 1), s = x % (n + 1);
        const cplx A = mk(-e, om_out.v[i0 + i]);
        if (s == n) {
          tl[i] = tail_integral(A, 1.0, wN) + tail_integral(A, -1.0, wN);
          continue;
        }
        const cplx bp = mk(-A.x, 1.0 - A.y);    // i - A
        const cplx bm = mk(-A.x, -1.0 - A.y);   // -i - A
        const double la = s == 0 ? 0.0 : lam[s - 1];
        const double H = s == 0 ? lam[0] : h[s - 1];
        cplx Ip[4], Im[4];
        moments(A + la * bp, bp, H, Ip);
        moments(A + la * bm, bm, H, Im);
        for (int k = 0; k < 4; ++k)
          K[(i * n + s) * 4 + k] = mk(0.0, -1.0) * (bp * Ip[k]) + mk(0.0, 1.0) * (bm * Im[k]);
      }
      __syncthreads();
      for (int x = tid; x < ni * nw; x += blockDim.x) {
        const int i = x / nw, j = x % nw;
        cplx t = mk(0.0, 0.0);
        for (int s = 0; s < n; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) t = t + S[(s * 4 + k) * nw + j] * K[(i * n + s) * 4 + k];
        if (j == nw - 1) t = t + (wN * wN) * tl[i];
        T[i * nw + j] = t;
      }
      __syncthreads();
      const int np = Q.cnt[slot], base = Q.off[slot];
      for (int x = tid; x < np * ni; x += blockDim.x) {
        const int r = x / ni, i = x % ni;
        const int p = Q.list[base + r];
        cplx v = mk(0.0, 0.0);
        for (int j = 0; j < nw; ++j) v = v + Q.c[size_t(j) * Q.npair + p] * T[i * nw + j];
        double2* out = reinterpret_cast<double2*>(sigma) + size_t(Q.state[p]) * nw_out + i0 + i;
        atomicAdd(&out->x, f * Q.wq * v.x);
        atomicAdd(&out->y, f * Q.wq * v.y);
      }
      __syncthreads();
    }
  }
}

static int conv_tsize(int64_t np) {
  int64_t t = 64;
  while (t < 2 * np) t <<= 1;
  return int(t);
}

static size_t conv_q_bytes(int64_t np) {
  const size_t t = size_t(conv_tsize(np));
  return ws_round(t * 8) + 4 * ws_round(t * 4) + ws_round(256) + 2 * ws_round(size_t(np) * 4);
}

static size_t conv_smem(int nw) {
  return size_t(4) * nw * nw * sizeof(double) + size_t(CIC) * nw * 4 * sizeof(cplx) +
         size_t(CIC) * nw * sizeof(cplx) + size_t(CIC) * sizeof(cplx);
}

size_t convolve_workspace(int nq, const int64_t* npair, int, int) {
  size_t b = 0;
  for (int q = 0; q < nq; ++q)
    if (npair[q] > 0) b += conv_q_bytes(npair[q]);
  return b + 256;
}

int convolve(int nq, const double* wq, const int64_t* npair, int nw, const OmegaArr& om,
             const double* const* c, const int* const* pair_state, const double* const* eps,
             int nw_out, const OmegaArr& om_out, int nsig, double* sigma, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  return convolve_acc(nq, wq, npair, nw, om, c, pair_state, eps, nw_out, om_out, nsig, sigma,
                      false, ws, ws_bytes, s, ctx);
}

int convolve_acc(int nq, const double* wq, const int64_t* npair, int nw, const OmegaArr& om,
                 const double* const* c, const int* const* pair_state, const double* const* eps,
                 int nw_out, const OmegaArr& om_out, int nsig, double* sigma, bool accumulate,
                 void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  if (!accumulate)
    GW_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * 2 * size_t(nsig) * nw_out, s));
  const size_t smem = conv_smem(nw);
  {
    int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_conv_slot), conv_smem(GW_MAX_NW),
                              ctx.device);
    if (rc) return rc;
  }
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  for (int q0 = 0; q0 < nq; q0 += SMAXQ) {
    const int n = std::min(SMAXQ, nq - q0);
    ConvLaunch L{};
    L.nq = n;
    int64_t slots = 0, pairs = 0;
    std::vector<int64_t> s0(n + 1), p0(n + 1);
    for (int q = 0; q < n; ++q) {
      ConvQ& Q = L.Q[q];
      const int64_t np = npair[q0 + q];
      Q.c = c[q0 + q];
      Q.state = pair_state[q0 + q];
      Q.eps = eps[q0 + q];
      Q.npair = np;
      Q.wq = wq[q0 + q];
      Q.tsize = np > 0 ? conv_tsize(np) : 0;
      s0[q] = slots;
      p0[q] = pairs;
      if (np > 0) {
        const size_t t = size_t(Q.tsize);
        Q.keys = static_cast<unsigned long long*>(cur.take(t * 8));
        Q.cnt = static_cast<int*>(cur.take(t * 4));
        Q.off = static_cast<int*>(cur.take(t * 4));
        Q.fill = static_cast<int*>(cur.take(t * 4));
        Q.occ = static_cast<int*>(cur.take(t * 4));
        Q.nocc = static_cast<int*>(cur.take(256));
        Q.slot_of = static_cast<int*>(cur.take(size_t(np) * 4));
        Q.list = static_cast<int*>(cur.take(size_t(np) * 4));
        if (!Q.keys || !Q.cnt || !Q.off || !Q.fill || !Q.occ || !Q.nocc || !Q.slot_of || !Q.list)
          return set_error(GW_EWORKSPACE, "convolution workspace too small");
      }
      slots += Q.tsize;
      pairs += np;
    }
    s0[n] = slots;
    p0[n] = pairs;
    if (pairs == 0) continue;
    const unsigned grid_cap = unsigned(ctx.sm_count) * 8;
    for (int q = 0; q <= n; ++q) L.item0[q] = s0[q];
    k_conv_init<<<unsigned(std::min<int64_t>((slots + 255) / 256, grid_cap)), 256, 0, s>>>(L);
    GW_LAUNCH_CHECK("k_conv_init");
    for (int q = 0; q <= n; ++q) L.item0[q] = p0[q];
    const unsigned pg = unsigned(std::min<int64_t>((pairs + 255) / 256, grid_cap));
    k_conv_hash<<<pg, 256, 0, s>>>(L, nsig, ctx.status);
    GW_LAUNCH_CHECK("k_conv_hash");
    k_conv_scan<<<unsigned(n), 1024, 0, s>>>(L);
    GW_LAUNCH_CHECK("k_conv_scan");
    k_conv_scatter<<<pg, 256, 0, s>>>(L);
    GW_LAUNCH_CHECK("k_conv_scatter");
    const int nich = (nw_out + CIC - 1) / CIC;
    const int64_t est = pairs * nich;          // upper bound on the slot items
    const unsigned sg = unsigned(std::max<int64_t>(1, std::min<int64_t>(est, int64_t(ctx.sm_count) * 4)));
    k_conv_slot<<<sg, CTHREADS, smem, s>>>(L, nw, om, om_out, nw_out, sigma);
    GW_LAUNCH_CHECK("k_conv_slot");
  }
  return GW_OK;
}

}  // namespace gw
