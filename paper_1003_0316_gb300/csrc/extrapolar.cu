// Extrapolar correction of the band sums (Sec. V, the paragraph on the convergence with the
// number of bands; the scheme of Bruneval and Gonze, kept with the full W^c instead of a
// plasmon-pole model). All bands beyond the cutoff N' sit at one energy e_bar; the
// completeness of the one-particle states then turns their sum into a full-band integral
// minus the kept bands:
//
//   polarization:  P^EX = sum_t [w(Delta_t) - w(Delta_bar_t)] M_t M_t^H      (the HERK, with
//                         the modified transition weights of the polarization kernels)
//                       + sum_kn w(Delta_bar_kn) C^kn                        (k_completeness)
//   self-energy:   one extra pair per (q, s) at e_bar with
//                  cbar_s(w') = sum_IJ W^c_IJ(w') S^s_IJ - sum_{n' <= N'} c_{s n'}(w')
//                  (k_extrapolar_trace, k_extrapolar_finish), convolved like every pair.
//
// k_completeness: one CTA per (q, 16 x 16 upper tile, group of 16 frequencies), one matrix
// entry per thread; the occupied states kn stream through in chunks of 32 whose weights sit
// in shared memory. Complex128 input is summed in FP64. Complex64 / float32 input (the
// split-precision paths) is summed in FP32 over a chunk and the chunk sums are folded into
// a two-float (hi, lo) running sum by an error-free two-sum, so the FP64 pipe is not used
// in the loop; the entry and its Hermitian mirror are added to P at the end.
#include <vector>
#include <algorithm>

#include "gw_internal.cuh"

namespace gw {
namespace {

constexpr int CT = 16;        // completeness tile edge
constexpr int CJG = 16;       // frequencies per CTA
constexpr int CKC = 32;       // occupied states per chunk
constexpr int CUNR = 8;       // loads in flight per thread
constexpr int CMAXQ = 64;

struct ComplLaunch {
  const void* C[CMAXQ];
  const double* dbar[CMAXQ];
  const double* f[CMAXQ];
  double2* P[CMAXQ];
  int64_t nkn[CMAXQ];
  int nb[CMAXQ];
  int tside[CMAXQ];
  int64_t item0[CMAXQ + 1];
  int nq;
  int nw;
  int njg;
};

__device__ __forceinline__ void upper_tile(int u, int T, int* ti, int* tj) {
  int r = 0;
  while (u >= T - r) { u -= T - r; ++r; }
  *ti = r;
  *tj = r + u;
}

// error-free sum of a and b: s + e == a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (b - bp);
  hi = s;
  lo += e;
}

template <int DT> struct CTraits;
template <> struct CTraits<GW_C128> { using T = double2; using W = double; static constexpr bool cplx = true; };
template <> struct CTraits<GW_C64> { using T = float2; using W = float; static constexpr bool cplx = true; };
template <> struct CTraits<GW_R32> { using T = float; using W = float; static constexpr bool cplx = false; };

__device__ __forceinline__ double2 ld_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float ld_c(const float* p) { return __ldg(p); }
__device__ __forceinline__ double re_of(double2 v) { return v.x; }
__device__ __forceinline__ double im_of(double2 v) { return v.y; }
__device__ __forceinline__ float re_of(float2 v) { return v.x; }
__device__ __forceinline__ float im_of(float2 v) { return v.y; }
__device__ __forceinline__ float re_of(float v) { return v; }
__device__ __forceinline__ float im_of(float) { return 0.0f; }

template <int DT>
__global__ void __launch_bounds__(256) k_completeness(ComplLaunch L, double pref, OmegaArr om,
                                                      unsigned* status) {
  using Tr = CTraits<DT>;
  using T = typename Tr::T;
  using W = typename Tr::W;
  constexpr bool FP64 = DT == GW_C128;
  constexpr int NV = Tr::cplx ? 2 : 1;      // real values per entry

  const int64_t item = blockIdx.x;
  int q = 0;
  while (q + 1 < L.nq && item >= L.item0[q + 1]) ++q;
  const int64_t local = item - L.item0[q];
  const int jg = int(local % L.njg);
  int ti, tj;
  upper_tile(int(local / L.njg), L.tside[q], &ti, &tj);
  const int nb = L.nb[q];
  const int I = ti * CT + (threadIdx.x >> 4);
  const int J = tj * CT + (threadIdx.x & 15);
  const bool act = I < nb && J < nb && I <= J;
  const int j0 = jg * CJG;
  const int nj = min(CJG, L.nw - j0);
  const int64_t nkn = L.nkn[q];
  const size_t nb2 = size_t(nb) * nb;
  const T* __restrict__ C = static_cast<const T*>(L.C[q]) + (act ? size_t(I) * nb + J : 0);
  const double* __restrict__ dbar = L.dbar[q];
  const double* __restrict__ fk = L.f[q];

  __shared__ W wsh[CKC][CJG];
  // FP64 path: acc holds the sums. FP32 paths: part is the chunk sum, (acc, lo) the
  // two-float running sum.
  W part[CJG][NV];
  W acc[CJG][NV];
  float lo[CJG][NV];
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      part[jj][v] = W(0);
      acc[jj][v] = W(0);
      lo[jj][v] = 0.0f;
    }

  for (int64_t k0 = 0; k0 < nkn; k0 += CKC) {
    const int kc = int(nkn - k0 < CKC ? nkn - k0 : CKC);
    __syncthreads();
    for (int e = threadIdx.x; e < CKC * CJG; e += blockDim.x) {
      const int kk = e / CJG, jj = e % CJG;
      W w = W(0);
      if (kk < kc && jj < nj) {
        const double db = dbar[k0 + kk];
        if (!(db > 0.0)) raise_status(status, ST_EINVAL);
        const double a = -2.0 * pref * (fk ? fk[k0 + kk] : 1.0);
        const double wv = om.v[j0 + jj];
        if (FP64) {
          w = W(a * db / (db * db + wv * wv));
        } else {
          const float dbf = float(db), wf = float(wv);
          w = W(float(a) * dbf / fmaf(dbf, dbf, wf * wf));
        }
      }
      wsh[kk][jj] = w;
    }
    __syncthreads();
    if (!act) continue;
    for (int kk = 0; kk < kc; kk += CUNR) {
      T val[CUNR];
#pragma unroll
      for (int u = 0; u < CUNR; ++u)
        val[u] = (kk + u < kc) ? ld_c(C + size_t(k0 + kk + u) * nb2) : T{};
#pragma unroll
      for (int u = 0; u < CUNR; ++u) {
        const W cr = W(re_of(val[u]));
        const W ci = W(im_of(val[u]));
#pragma unroll
        for (int jj = 0; jj < CJG; ++jj) {
          const W w = wsh[kk + u][jj];     // zero beyond kc and nj
          if constexpr (FP64) {
            acc[jj][0] = fma(w, cr, acc[jj][0]);
            acc[jj][NV - 1] = fma(w, ci, acc[jj][NV - 1]);
          } else {
            part[jj][0] = fmaf(w, cr, part[jj][0]);
            if constexpr (NV == 2) part[jj][NV - 1] = fmaf(w, ci, part[jj][NV - 1]);
          }
        }
      }
    }
    if constexpr (!FP64) {
#pragma unroll
      for (int jj = 0; jj < CJG; ++jj)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float h = float(acc[jj][v]);
          two_sum_acc(h, lo[jj][v], float(part[jj][v]));
          acc[jj][v] = W(h);
          part[jj][v] = W(0);
        }
    }
  }
  if (!act) return;
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj) {
    if (jj >= nj) break;
    const double re = double(acc[jj][0]) + (FP64 ? 0.0 : double(lo[jj][0]));
    const double im = NV == 2 ? double(acc[jj][NV - 1]) + (FP64 ? 0.0 : double(lo[jj][NV - 1])) : 0.0;
    double2* Pj = L.P[q] + size_t(j0 + jj) * nb2;
    double2* up = Pj + size_t(I) * nb + J;
    if (I == J) {
      up->x += re;                         // Hermitian: real diagonal
    } else {
      double2 a = *up;
      a.x += re;
      a.y += im;
      *up = a;
      double2* dn = Pj + size_t(J) * nb + I;
      double2 b = *dn;
      b.x += re;
      b.y -= im;
      *dn = b;
    }
  }
}

// ------------------------------------------------------------ self-energy side
constexpr int SJG = 8;       // frequencies per CTA
constexpr int SSG = 4;       // states per CTA
constexpr int SNCH = 32;     // element chunks per (q, group)

struct TraceLaunch {
  const double2* S[CMAXQ];
  const double2* W[CMAXQ];
  int nb[CMAXQ];
  int nq, nw, nsig, njg, nsg;
};

// part[((q * SNCH + ch) * nw + j) * nsig + s] = sum over the chunk's entries of Re(W_j S_s)
__global__ void __launch_bounds__(256) k_extrapolar_trace(TraceLaunch L, double* __restrict__ part) {
  int64_t item = blockIdx.x;
  const int ch = int(item % SNCH);
  item /= SNCH;
  const int sg = int(item % L.nsg);
  item /= L.nsg;
  const int jg = int(item % L.njg);
  const int q = int(item / L.njg);
  const int nb = L.nb[q];
  const int64_t nb2 = int64_t(nb) * nb;
  const int64_t per = (nb2 + SNCH - 1) / SNCH;
  const int64_t beg = per * ch, end = min(nb2, beg + per);
  const int j0 = jg * SJG, s0 = sg * SSG;
  const double2* __restrict__ Wq = L.W[q];
  const double2* __restrict__ Sq = L.S[q];
  double acc[SSG][SJG];
#pragma unroll
  for (int a = 0; a < SSG; ++a)
#pragma unroll
    for (int b = 0; b < SJG; ++b) acc[a][b] = 0.0;
  for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    double2 w[SJG];
#pragma unroll
    for (int b = 0; b < SJG; ++b)
      w[b] = j0 + b < L.nw ? __ldg(Wq + size_t(j0 + b) * nb2 + e) : make_double2(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < SSG; ++a) {
      if (s0 + a >= L.nsig) break;
      const double2 sv = __ldg(Sq + size_t(s0 + a) * nb2 + e);
#pragma unroll
      for (int b = 0; b < SJG; ++b) acc[a][b] = fma(w[b].x, sv.x, fma(-w[b].y, sv.y, acc[a][b]));
    }
  }
  __shared__ double red[8][SSG * SJG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < SSG; ++a)
#pragma unroll
    for (int b = 0; b < SJG; ++b) {
      double v = acc[a][b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][a * SJG + b] = v;
    }
  __syncthreads();
  if (threadIdx.x < SSG * SJG) {
    const int a = threadIdx.x / SJG, b = threadIdx.x % SJG;
    double v = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) v += red[w8][threadIdx.x];
    if (s0 + a < L.nsig && j0 + b < L.nw)
      part[((size_t(q) * SNCH + ch) * L.nw + j0 + b) * L.nsig + s0 + a] = v;
  }
}

struct FinishLaunch {
  const double* c[CMAXQ];        // [nw][npair] kept pair coefficients
  const int* state[CMAXQ];       // [npair]
  int64_t npair[CMAXQ];
  double ebar[CMAXQ];
  int nq, nw, nsig;
};

// cbar[q][j][s] = sum of the chunk traces (fixed order) - sum_{p: state(p) = s} c[q][j][p];
// also the extra pairs' states and energies for the convolution
__global__ void k_extrapolar_finish(FinishLaunch L, const double* __restrict__ part,
                                    double* __restrict__ cbar, int* __restrict__ state_x,
                                    double* __restrict__ eps_x, unsigned* status) {
  const int64_t n = int64_t(L.nq) * L.nw * L.nsig;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int s = int(i % L.nsig);
    const int j = int((i / L.nsig) % L.nw);
    const int q = int(i / (int64_t(L.nsig) * L.nw));
    double t = 0.0;
    for (int ch = 0; ch < SNCH; ++ch) t += part[((size_t(q) * SNCH + ch) * L.nw + j) * L.nsig + s];
    const double* cj = L.c[q] + size_t(j) * L.npair[q];
    const int* st = L.state[q];
    double kept = 0.0;
    for (int64_t p = 0; p < L.npair[q]; ++p) {
      const int sp = st[p];
      if (sp < 0 || sp >= L.nsig) {
        if (j == 0 && s == 0) raise_status(status, ST_EINVAL);
        continue;
      }
      if (sp == s) kept += cj[p];
    }
    cbar[i] = t - kept;
    if (j == 0) {
      eps_x[size_t(q) * L.nsig + s] = L.ebar[q];
      if (q == 0) state_x[s] = s;
    }
  }
}

}  // namespace

int completeness_add(int nq, const ComplQ* qs, int dtype, double pref, int nw, const OmegaArr& om,
                     cudaStream_t s, const DeviceCtx& ctx) {
  const int njg = (nw + CJG - 1) / CJG;
  for (int q0 = 0; q0 < nq; q0 += CMAXQ) {
    const int n = std::min(CMAXQ, nq - q0);
    ComplLaunch L{};
    L.nq = n;
    L.nw = nw;
    L.njg = njg;
    int64_t item = 0;
    for (int q = 0; q < n; ++q) {
      const ComplQ& Q = qs[q0 + q];
      L.C[q] = Q.C;
      L.dbar[q] = Q.dbar;
      L.f[q] = Q.f;
      L.P[q] = reinterpret_cast<double2*>(Q.P);
      L.nkn[q] = Q.nkn;
      L.nb[q] = Q.nb;
      L.tside[q] = (Q.nb + CT - 1) / CT;
      L.item0[q] = item;
      if (Q.nkn > 0) item += int64_t(L.tside[q]) * (L.tside[q] + 1) / 2 * njg;
    }
    L.item0[n] = item;
    if (item == 0) continue;
    if (item > 2147483647LL) return set_error(GW_EINVAL, "completeness term: too many tiles");
    if (dtype == GW_C128)
      k_completeness<GW_C128><<<unsigned(item), 256, 0, s>>>(L, pref, om, ctx.status);
    else if (dtype == GW_C64)
      k_completeness<GW_C64><<<unsigned(item), 256, 0, s>>>(L, pref, om, ctx.status);
    else
      k_completeness<GW_R32><<<unsigned(item), 256, 0, s>>>(L, pref, om, ctx.status);
    GW_LAUNCH_CHECK("k_completeness");
  }
  return GW_OK;
}

size_t sigma_extrapolar_workspace(int nq, int nw, int nsig, int) {
  const size_t per = size_t(nw) * nsig;
  return ws_round(size_t(nq) * SNCH * per * sizeof(double))     // chunk traces
         + ws_round(size_t(nq) * per * sizeof(double))          // cbar
         + ws_round(size_t(nsig) * sizeof(int))                 // extra pairs' states
         + ws_round(size_t(nq) * nsig * sizeof(double)) + 1024; // extra pairs' energies
}

int sigma_extrapolar(int nq, const double* wq, const int* nb, int nsig, const double* const* S,
                     int nw, const OmegaArr& om, const double* const* Wc, const int64_t* npair,
                     const int* const* pair_state, const double* const* c, const double* ebar,
                     int nw_out, const OmegaArr& om_out, double* sigma, double* cbar_out, void* ws,
                     size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  const size_t per = size_t(nw) * nsig;
  double* part = static_cast<double*>(cur.take(size_t(nq) * SNCH * per * sizeof(double)));
  double* cbar_ws = static_cast<double*>(cur.take(size_t(nq) * per * sizeof(double)));
  int* state_x = static_cast<int*>(cur.take(size_t(nsig) * sizeof(int)));
  double* eps_x = static_cast<double*>(cur.take(size_t(nq) * nsig * sizeof(double)));
  if (!part || !cbar_ws || !state_x || !eps_x)
    return set_error(GW_EWORKSPACE, "extrapolar workspace too small");
  double* cbar = cbar_out ? cbar_out : cbar_ws;
  for (int q0 = 0; q0 < nq; q0 += CMAXQ) {
    const int n = std::min(CMAXQ, nq - q0);
    TraceLaunch T{};
    T.nq = n;
    T.nw = nw;
    T.nsig = nsig;
    T.njg = (nw + SJG - 1) / SJG;
    T.nsg = (nsig + SSG - 1) / SSG;
    FinishLaunch F{};
    F.nq = n;
    F.nw = nw;
    F.nsig = nsig;
    for (int q = 0; q < n; ++q) {
      T.S[q] = reinterpret_cast<const double2*>(S[q0 + q]);
      T.W[q] = reinterpret_cast<const double2*>(Wc[q0 + q]);
      T.nb[q] = nb[q0 + q];
      F.c[q] = c[q0 + q];
      F.state[q] = pair_state[q0 + q];
      F.npair[q] = npair[q0 + q];
      F.ebar[q] = ebar[q0 + q];
    }
    const int64_t items = int64_t(n) * T.njg * T.nsg * SNCH;
    k_extrapolar_trace<<<unsigned(items), 256, 0, s>>>(T, part);
    GW_LAUNCH_CHECK("k_extrapolar_trace");
    const int64_t cnt = int64_t(n) * per;
    double* cb = cbar + size_t(q0) * per;
    double* ex = eps_x + size_t(q0) * nsig;
    k_extrapolar_finish<<<unsigned(std::min<int64_t>((cnt + 255) / 256, 4096)), 256, 0, s>>>(
        F, part, cb, state_x, ex, ctx.status);
    GW_LAUNCH_CHECK("k_extrapolar_finish");
  }
  std::vector<const double*> cq(nq), eq(nq);
  std::vector<const int*> sq(nq, state_x);
  std::vector<int64_t> np(nq, nsig);
  for (int q = 0; q < nq; ++q) {
    cq[q] = cbar + size_t(q) * per;
    eq[q] = eps_x + size_t(q) * nsig;
  }
  return convolve_acc(nq, wq, np.data(), nw, om, cq.data(), sq.data(), eq.data(), nw_out, om_out,
                      nsig, sigma, true, s, ctx);
}

}  // namespace gw
