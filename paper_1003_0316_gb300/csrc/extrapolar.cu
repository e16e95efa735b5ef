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
// Completeness term: one CTA per (q, 16 x 16 upper tile, group of 16 frequencies), one matrix
// entry per thread; the occupied states kn stream through in chunks of 32 whose weights sit
// in shared memory. Complex128 input is summed in FP64 (k_completeness_fp64). Complex64 /
// float32 input (the split-precision paths, k_completeness_async) is staged through shared
// memory by asynchronous copies, summed in FP32 over a chunk, and the chunk sums are folded
// into a two-float (hi, lo) running sum by an error-free two-sum, so the FP64 pipe is not used
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
constexpr int CNST = 2;       // FP32 kernels: shared-memory stages of CKC states

struct ComplLaunch {
  const void* C[CMAXQ];
  const double* dbar[CMAXQ];
  const double* f[CMAXQ];
  double2* P[CMAXQ];
  int64_t nkn[CMAXQ];
  int nb[CMAXQ];
  int tside[CMAXQ];     // 16 x 16 tiles per side
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

// element type of the FP32 paths' completeness input
template <int DT> struct CTraits;
template <> struct CTraits<GW_C64> { using T = float2; static constexpr bool cplx = true; };
template <> struct CTraits<GW_R32> { using T = float; static constexpr bool cplx = false; };

__device__ __forceinline__ float re_of(float2 v) { return v.x; }
__device__ __forceinline__ float im_of(float2 v) { return v.y; }
__device__ __forceinline__ float re_of(float v) { return v; }
__device__ __forceinline__ float im_of(float) { return 0.0f; }

// Adds re + i im to P_j[I][J] and its Hermitian mirror (a real diagonal).
__device__ __forceinline__ void add_hermitian(double2* Pj, int nb, int I, int J, double re, double im) {
  double2* up = Pj + size_t(I) * nb + J;
  if (I == J) {
    up->x += re;
    return;
  }
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

// FP64 path (complex128 input): the sums stay in FP64 registers; CUNR loads in flight.
__global__ void __launch_bounds__(256) k_completeness_fp64(ComplLaunch L, double pref, OmegaArr om,
                                                           unsigned* status) {
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
  const double2* __restrict__ C =
      static_cast<const double2*>(L.C[q]) + (act ? size_t(I) * nb + J : 0);
  const double* __restrict__ dbar = L.dbar[q];
  const double* __restrict__ fk = L.f[q];

  __shared__ double wsh[CKC][CJG];
  double acc[CJG][2];
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj) acc[jj][0] = acc[jj][1] = 0.0;

  for (int64_t k0 = 0; k0 < nkn; k0 += CKC) {
    const int kc = int(nkn - k0 < CKC ? nkn - k0 : CKC);
    __syncthreads();
    for (int e = threadIdx.x; e < CKC * CJG; e += blockDim.x) {
      const int kk = e / CJG, jj = e % CJG;
      double w = 0.0;
      if (kk < kc && jj < nj) {
        const double db = dbar[k0 + kk];
        if (!(db > 0.0)) raise_status(status, ST_EINVAL);
        const double wv = om.v[j0 + jj];
        w = -2.0 * pref * (fk ? fk[k0 + kk] : 1.0) * db / (db * db + wv * wv);
      }
      wsh[kk][jj] = w;
    }
    __syncthreads();
    if (!act) continue;
    for (int kk = 0; kk < kc; kk += CUNR) {
      double2 val[CUNR];
#pragma unroll
      for (int u = 0; u < CUNR; ++u)
        val[u] = (kk + u < kc) ? __ldg(C + size_t(k0 + kk + u) * nb2) : make_double2(0.0, 0.0);
#pragma unroll
      for (int u = 0; u < CUNR; ++u) {
#pragma unroll
        for (int jj = 0; jj < CJG; ++jj) {
          const double w = wsh[kk + u][jj];     // zero beyond kc and nj
          acc[jj][0] = fma(w, val[u].x, acc[jj][0]);
          acc[jj][1] = fma(w, val[u].y, acc[jj][1]);
        }
      }
    }
  }
  if (!act) return;
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj) {
    if (jj >= nj) break;
    add_hermitian(L.P[q] + size_t(j0 + jj) * nb2, nb, I, J, acc[jj][0], acc[jj][1]);
  }
}

// The FP32 paths (complex64 / float32 input) with the C entries staged through shared memory
// by per-thread asynchronous copies: chunk c + 1 is in flight while chunk c is summed. Each
// thread copies and reads only its own entry, so its own wait_group is the only data
// dependence; the weights are shared and follow a block barrier.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int DT>
__global__ void __launch_bounds__(256, 1) k_completeness_async(ComplLaunch L, double pref, OmegaArr om,
                                                            unsigned* status) {
  using Tr = CTraits<DT>;
  using T = typename Tr::T;
  constexpr int NV = Tr::cplx ? 2 : 1;
  static_assert(DT != GW_C128, "FP32 paths only");

  const int64_t item = blockIdx.x;
  int q = 0;
  while (q + 1 < L.nq && item >= L.item0[q + 1]) ++q;
  const int64_t local = item - L.item0[q];
  const int jg = int(local % L.njg);
  int ti, tj;
  upper_tile(int(local / L.njg), L.tside[q], &ti, &tj);
  const int nb = L.nb[q];
  const int tid = threadIdx.x;
  const int I = ti * CT + (tid >> 4);
  const int J = tj * CT + (tid & 15);
  const bool act = I < nb && J < nb && I <= J;
  const int j0 = jg * CJG;
  const int nj = min(CJG, L.nw - j0);
  const int64_t nkn = L.nkn[q];
  const size_t nb2 = size_t(nb) * nb;
  const T* __restrict__ C = static_cast<const T*>(L.C[q]) + (act ? size_t(I) * nb + J : 0);
  const double* __restrict__ dbar = L.dbar[q];
  const double* __restrict__ fk = L.f[q];

  extern __shared__ __align__(16) unsigned char csm[];
  T* stage = reinterpret_cast<T*>(csm);                     // [CNST][CKC][256]
  __shared__ __align__(16) float wsh[CKC][CJG];

  auto prefetch = [&](int64_t k0, int buf) {
    if (act) {
      const int kc = int(nkn - k0 < CKC ? nkn - k0 : CKC);
      T* dst = stage + size_t(buf) * CKC * 256 + tid;
      for (int kk = 0; kk < kc; ++kk) {
        if (NV == 2) cp_async8(dst + kk * 256, C + size_t(k0 + kk) * nb2);
        else cp_async4(dst + kk * 256, C + size_t(k0 + kk) * nb2);
      }
    }
    cp_async_commit();
  };

  float part[CJG][NV], acc[CJG][NV], lo[CJG][NV];
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj)
#pragma unroll
    for (int v = 0; v < NV; ++v) part[jj][v] = acc[jj][v] = lo[jj][v] = 0.0f;

  // CNST - 1 chunks in flight while one is summed; every iteration commits one group (empty
  // past the end) so that wait_group CNST - 1 always means "the current chunk has landed"
  for (int c = 0; c < CNST - 1; ++c) {
    if (int64_t(c) * CKC < nkn) prefetch(int64_t(c) * CKC, c);
    else cp_async_commit();
  }
  int buf = 0;
  for (int64_t k0 = 0; k0 < nkn; k0 += CKC, buf = (buf + 1) % CNST) {
    const int kc = int(nkn - k0 < CKC ? nkn - k0 : CKC);
    const int64_t kn_next = k0 + int64_t(CNST - 1) * CKC;
    if (kn_next < nkn) prefetch(kn_next, (buf + CNST - 1) % CNST);
    else cp_async_commit();
    __syncthreads();                            // the previous chunk's weights are consumed
    for (int e = tid; e < CKC * CJG; e += blockDim.x) {
      const int kk = e / CJG, jj = e % CJG;
      float w = 0.0f;
      if (kk < kc && jj < nj) {
        const double db = dbar[k0 + kk];
        if (!(db > 0.0)) raise_status(status, ST_EINVAL);
        const float a = float(-2.0 * pref * (fk ? fk[k0 + kk] : 1.0));
        const float dbf = float(db), wf = float(om.v[j0 + jj]);
        w = a * dbf / fmaf(dbf, dbf, wf * wf);
      }
      wsh[kk][jj] = w;
    }
    cp_async_wait<CNST - 1>();                  // this thread's copies of chunk k0 landed
    __syncthreads();
    if (act) {
      const T* src = stage + size_t(buf) * CKC * 256 + tid;
      for (int kk = 0; kk < kc; ++kk) {
        const T cv = src[kk * 256];
        const float cr = float(re_of(cv)), ci = float(im_of(cv));
        const float4* wrow = reinterpret_cast<const float4*>(wsh[kk]);
#pragma unroll
        for (int j4 = 0; j4 < CJG / 4; ++j4) {
          const float4 w4 = wrow[j4];
          const float ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            part[4 * j4 + t][0] = fmaf(ws[t], cr, part[4 * j4 + t][0]);
            if constexpr (NV == 2) part[4 * j4 + t][NV - 1] = fmaf(ws[t], ci, part[4 * j4 + t][NV - 1]);
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < CJG; ++jj)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          two_sum_acc(acc[jj][v], lo[jj][v], part[jj][v]);
          part[jj][v] = 0.0f;
        }
    }
  }
  if (!act) return;
#pragma unroll
  for (int jj = 0; jj < CJG; ++jj) {
    if (jj >= nj) break;
    const double re = double(acc[jj][0]) + double(lo[jj][0]);
    const double im = NV == 2 ? double(acc[jj][NV - 1]) + double(lo[jj][NV - 1]) : 0.0;
    add_hermitian(L.P[q] + size_t(j0 + jj) * nb2, nb, I, J, re, im);
  }
}

constexpr size_t async_smem(int dt) {
  return size_t(CNST) * CKC * 256 * (dt == GW_C64 ? 8 : 4);
}

// ------------------------------------------------------------ self-energy side
constexpr int SJG = 8;       // frequencies per CTA
constexpr int SSG = 4;       // states per CTA
constexpr int SNCH = 128;    // element chunks per (q, group)

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

// cbar[q][j][s] = sum of the chunk traces (fixed order) - sum_{p: state(p) = s} c[q][j][p]:
// one warp per (q, j, s), lanes striding over the pairs and a fixed shuffle tree, so the
// result does not depend on scheduling; lane 0 also writes the extra pair's energy and state
__global__ void __launch_bounds__(256) k_extrapolar_finish(FinishLaunch L,
                                                           const double* __restrict__ part,
                                                           double* __restrict__ cbar,
                                                           int* __restrict__ state_x,
                                                           double* __restrict__ eps_x,
                                                           unsigned* status) {
  const int64_t n = int64_t(L.nq) * L.nw * L.nsig;
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (i >= n) return;                         // whole warps
  const int s = int(i % L.nsig);
  const int j = int((i / L.nsig) % L.nw);
  const int q = int(i / (int64_t(L.nsig) * L.nw));
  const double* __restrict__ cj = L.c[q] + size_t(j) * L.npair[q];
  const int* __restrict__ st = L.state[q];
  double kept = 0.0;
  bool bad = false;
  for (int64_t p = lane; p < L.npair[q]; p += 32) {
    const int sp = __ldg(st + p);
    bad |= sp < 0 || sp >= L.nsig;
    if (sp == s) kept += __ldg(cj + p);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if (bad && j == 0 && s == 0) raise_status(status, ST_EINVAL);
  if (lane == 0) {
    double t = 0.0;
    for (int ch = 0; ch < SNCH; ++ch) t += part[((size_t(q) * SNCH + ch) * L.nw + j) * L.nsig + s];
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
    if (dtype == GW_C128) {
      k_completeness_fp64<<<unsigned(item), 256, 0, s>>>(L, pref, om, ctx.status);
    } else if (dtype == GW_C64) {
      int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_completeness_async<GW_C64>),
                                async_smem(GW_C64), ctx.device);
      if (rc) return rc;
      k_completeness_async<GW_C64><<<unsigned(item), 256, async_smem(GW_C64), s>>>(L, pref, om,
                                                                                ctx.status);
    } else {
      int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_completeness_async<GW_R32>),
                                async_smem(GW_R32), ctx.device);
      if (rc) return rc;
      k_completeness_async<GW_R32><<<unsigned(item), 256, async_smem(GW_R32), s>>>(L, pref, om,
                                                                                ctx.status);
    }
    GW_LAUNCH_CHECK("k_completeness");
  }
  return GW_OK;
}

size_t sigma_extrapolar_workspace(int nq, int nw, int nsig, int) {
  const size_t per = size_t(nw) * nsig;
  return ws_round(size_t(nq) * SNCH * per * sizeof(double))     // chunk traces
         + ws_round(size_t(nq) * per * sizeof(double))          // cbar
         + ws_round(size_t(nsig) * sizeof(int))                 // extra pairs' states
         + ws_round(size_t(nq) * nsig * sizeof(double)) + 1024  // extra pairs' energies
         + convolve_workspace(nq, std::vector<int64_t>(nq, nsig).data(), nw, 0);
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
    k_extrapolar_finish<<<unsigned((cnt * 32 + 255) / 256), 256, 0, s>>>(F, part, cb, state_x, ex,
                                                                         ctx.status);
    GW_LAUNCH_CHECK("k_extrapolar_finish");
  }
  std::vector<const double*> cq(nq), eq(nq);
  std::vector<const int*> sq(nq, state_x);
  std::vector<int64_t> np(nq, nsig);
  for (int q = 0; q < nq; ++q) {
    cq[q] = cbar + size_t(q) * per;
    eq[q] = eps_x + size_t(q) * nsig;
  }
  const size_t used = (cur.used + 255) & ~size_t(255);
  return convolve_acc(nq, wq, np.data(), nw, om, cq.data(), sq.data(), eq.data(), nw_out, om_out,
                      nsig, sigma, true, static_cast<char*>(ws) + used, ws_bytes - used, s, ctx);
}

}  // namespace gw
