// a1 transition weights and the FP64 path of a2, the polarization
// P_IJ(q, i w_j) = sum_t w_tj M_tI conj(M_tJ)  (Eq. polar_MB at w = i omega).
//
// FP64 path: one CTA per (q, upper 64x64 tile, frequency, K-split). Each CTA
// streams its slice of transitions through shared memory in chunks of 8 rows,
// scales the I-side rows by w_tj (computed on the fly from Delta_t), and
// accumulates 4x4 complex outputs per thread with DFMA. Partial tiles go to the
// workspace and a reduction kernel sums the K-splits in a fixed order, writes the
// upper triangle and its Hermitian mirror.
#include <vector>
#include <algorithm>

#include "gw_internal.cuh"

namespace gw {

// ------------------------------------------------------------------ a1 -------
__global__ void k_weights(int64_t K, const double* __restrict__ delta,
                          const double* __restrict__ f, double pref, int nw, OmegaArr om,
                          double* __restrict__ w, unsigned* status) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (; t < K; t += stride) {
    double d = delta[t];
    double ft = f ? f[t] : 1.0;
    if (!(d > 0.0)) raise_status(status, ST_EINVAL);
    double d2 = d * d;
    double s = -2.0 * pref * ft * d;
    for (int j = 0; j < nw; ++j) {
      // bracket 1/(i w - D) - 1/(i w + D) = -2 D / (D^2 + w^2)
      w[int64_t(j) * K + t] = s / (d2 + om.v[j] * om.v[j]);
    }
  }
}

int launch_weights(int64_t K, const double* delta, const double* f, double pref, int nw,
                   const OmegaArr& om, double* w, cudaStream_t s, const DeviceCtx& ctx) {
  int64_t blocks = (K + 255) / 256;
  int64_t cap = int64_t(ctx.sm_count) * 8;
  if (blocks > cap) blocks = cap;
  k_weights<<<int(blocks), 256, 0, s>>>(K, delta, f, pref, nw, om, w, ctx.status);
  GW_LAUNCH_CHECK("k_weights");
  return GW_OK;
}

// Delta_t = e_unocc[kq[k]][n'] - e_occ[k][n] for t = (k nocc + n) nunocc + n'
__global__ void k_make_delta(int nk, int nocc, int nunocc, const double* __restrict__ eo, int ldo,
                             const double* __restrict__ eu, int ldu, const int* __restrict__ kq,
                             double* __restrict__ delta, unsigned* status) {
  const int64_t K = int64_t(nk) * nocc * nunocc;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < K;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int np = int(t % nunocc);
    const int64_t kn = t / nunocc;
    const int n = int(kn % nocc), k = int(kn / nocc);
    const int k2 = kq[k];
    if (k2 < 0 || k2 >= nk) {
      raise_status(status, ST_EINVAL);
      delta[t] = 0.0;
      continue;
    }
    delta[t] = eu[size_t(k2) * ldu + np] - eo[size_t(k) * ldo + n];
  }
}

int launch_make_delta(int nk, int nocc, int nunocc, const double* eo, int ldo, const double* eu,
                      int ldu, const int* kq, double* delta, cudaStream_t s, const DeviceCtx& ctx) {
  const int64_t K = int64_t(nk) * nocc * nunocc;
  if (K == 0) return GW_OK;
  const int64_t blocks = std::min<int64_t>((K + 255) / 256, int64_t(ctx.sm_count) * 8);
  k_make_delta<<<unsigned(blocks), 256, 0, s>>>(nk, nocc, nunocc, eo, ldo, eu, ldu, kq, delta,
                                                ctx.status);
  GW_LAUNCH_CHECK("k_make_delta");
  return GW_OK;
}

// ------------------------------------------------------------------ a2 -------
constexpr int HT = 64;   // output tile edge
constexpr int HKC = 8;   // rows per shared-memory chunk
constexpr int MAXQ = 64; // q entries per launch

struct PolLaunch {
  const double2* M[MAXQ];
  const double* delta[MAXQ];
  const double* dbar[MAXQ];   // extrapolar correction (NULL: none)
  const double* f[MAXQ];
  double2* P[MAXQ];
  int64_t K[MAXQ];
  int nb[MAXQ];
  int tside[MAXQ];        // tiles per side
  int splits[MAXQ];
  int64_t item0[MAXQ + 1];  // first work item of each q (prefix), item0[nq] = total
  size_t part0[MAXQ];       // first partial tile (in tiles) of each q
  int nq;
  int nw;
};

__device__ __forceinline__ void tile_of(int u, int T, int* ti, int* tj) {
  // u-th upper tile (ti <= tj), row-major over the upper triangle
  int r = 0;
  while (u >= T - r) { u -= T - r; ++r; }
  *ti = r;
  *tj = r + u;
}

__global__ void __launch_bounds__(256) k_herk_fp64(PolLaunch L, double pref, OmegaArr om,
                                                  double2* __restrict__ part, unsigned* status) {
  int64_t item = blockIdx.x;
  int q = 0;
  while (q + 1 < L.nq && item >= L.item0[q + 1]) ++q;
  int64_t local = item - L.item0[q];
  const int S = L.splits[q];
  const int T = L.tside[q];
  const int nw = L.nw;
  int split = int(local % S);
  int64_t rest = local / S;
  int j = int(rest % nw);
  int u = int(rest / nw);
  int ti, tj;
  tile_of(u, T, &ti, &tj);
  const int nb = L.nb[q];
  const int64_t K = L.K[q];
  const double2* __restrict__ M = L.M[q];
  const double* __restrict__ delta = L.delta[q];
  const double* __restrict__ fw = L.f[q];
  const double* __restrict__ dbar = L.dbar[q];
  const double wj2 = om.v[j] * om.v[j];
  int64_t per = (K + S - 1) / S;
  int64_t t_beg = per * split;
  int64_t t_end = t_beg + per < K ? t_beg + per : K;

  __shared__ double2 As[HKC][HT];
  __shared__ double2 Bs[HKC][HT];
  __shared__ double ws_[HKC];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);

  const int I0 = ti * HT, J0 = tj * HT;
  for (int64_t t0 = t_beg; t0 < t_end; t0 += HKC) {
    if (tid < HKC) {
      int64_t t = t0 + tid;
      double w = 0.0;
      if (t < t_end) {
        double d = delta[t];
        if (!(d > 0.0)) raise_status(status, ST_EINVAL);
        double ft = fw ? fw[t] : 1.0;
        w = -2.0 * pref * ft * d / (d * d + wj2);
        if (dbar) {
          // extrapolar correction: the same projections at Delta_bar enter with minus sign
          const double db = dbar[t];
          if (!(db > 0.0)) raise_status(status, ST_EINVAL);
          w += 2.0 * pref * ft * db / (db * db + wj2);
        }
      }
      ws_[tid] = w;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int e = tid + 256 * r;
      int k = e >> 6, i = e & 63;
      int64_t t = t0 + k;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (t < t_end) {
        if (I0 + i < nb) a = M[t * nb + I0 + i];
        if (J0 + i < nb) b = M[t * nb + J0 + i];
      }
      double w = ws_[k];
      As[k][i] = make_double2(a.x * w, a.y * w);
      Bs[k][i] = b;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < HKC; ++k) {
      double2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // acc += a * conj(b)
          acc[a][b].x = fma(av[a].x, bv[b].x, fma(av[a].y, bv[b].y, acc[a][b].x));
          acc[a][b].y = fma(av[a].y, bv[b].x, fma(-av[a].x, bv[b].y, acc[a][b].y));
        }
    }
    __syncthreads();
  }
  double2* out = part + (L.part0[q] + size_t(rest) * S + split) * (HT * HT);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) out[(ty + 16 * a) * HT + tx + 16 * b] = acc[a][b];
}

// Sum the K-splits of one (q, j, tile) and write the tile and its mirror.
__global__ void __launch_bounds__(256) k_herk_reduce(PolLaunch L, const double2* __restrict__ part,
                                                     bool accumulate) {
  int64_t blk = blockIdx.x;  // one block per (q, tile, j)
  int q = 0;
  // item0 counts (tile, j, split); blocks count (tile, j)
  int64_t acc_blocks = 0;
  for (q = 0; q < L.nq; ++q) {
    int64_t nblk = (L.item0[q + 1] - L.item0[q]) / L.splits[q];
    if (blk < acc_blocks + nblk) break;
    acc_blocks += nblk;
  }
  int64_t rest = blk - acc_blocks;
  const int S = L.splits[q];
  const int nw = L.nw;
  int j = int(rest % nw);
  int u = int(rest / nw);
  int ti, tj;
  tile_of(u, L.tside[q], &ti, &tj);
  const int nb = L.nb[q];
  const double2* src = part + (L.part0[q] + size_t(rest) * S) * (HT * HT);
  double2* P = L.P[q] + size_t(j) * nb * nb;
  for (int e = threadIdx.x; e < HT * HT; e += blockDim.x) {
    int i = e / HT, jj = e % HT;
    int I = ti * HT + i, J = tj * HT + jj;
    if (I >= nb || J >= nb) continue;
    if (ti == tj && I > J) continue;
    double2 s = make_double2(0.0, 0.0);
    for (int sp = 0; sp < S; ++sp) {
      double2 v = src[size_t(sp) * HT * HT + e];
      s.x += v.x;
      s.y += v.y;
    }
    if (I == J) s.y = 0.0;
    if (accumulate) {                          // each entry is written by this thread only
      const double2 o = P[size_t(I) * nb + J];
      s = make_double2(o.x + s.x, o.y + s.y);
      if (I == J) s.y = 0.0;
    }
    P[size_t(I) * nb + J] = s;
    if (I != J) P[size_t(J) * nb + I] = make_double2(s.x, -s.y);
  }
}

static void plan_fp64(int nq, const int64_t* K, const int* nb, int nw, int sm_count, int waves,
                      std::vector<int>& splits, std::vector<int64_t>& tiles) {
  splits.resize(nq);
  tiles.resize(nq);
  int64_t base = 0;
  for (int q = 0; q < nq; ++q) {
    int T = (nb[q] + HT - 1) / HT;
    tiles[q] = int64_t(T) * (T + 1) / 2;
    base += tiles[q] * nw;
  }
  // K splits: at least `waves` (default four) waves of CTAs (one CTA per SM: 136 registers x 256 threads) and
  // whole waves as far as possible, since every CTA of a launch takes about the same time and a
  // partly filled last wave idles the rest of the GPU; at least 512 rows per split. Among the
  // split counts from the four-wave minimum to twice it, the smallest whose fill of the last
  // wave is within 1 % of the best is taken.
  const int64_t slots = std::max(1, sm_count);
  const int64_t b = std::max<int64_t>(base, 1);
  const int64_t s_lo = std::max<int64_t>(1, (int64_t(waves) * slots + b - 1) / b), s_hi = 2 * s_lo;
  auto items_at = [&](int64_t sp) {
    int64_t it = 0;
    for (int q = 0; q < nq; ++q)
      it += tiles[q] * nw * std::min<int64_t>(sp, std::max<int64_t>(1, K[q] / 512));
    return it;
  };
  auto fill = [&](int64_t sp) {
    const int64_t it = items_at(sp);
    return double(it) / double((it + slots - 1) / slots * slots);
  };
  double best = 0.0;
  for (int64_t sp = s_lo; sp <= s_hi; ++sp) best = std::max(best, fill(sp));
  int64_t pick = s_lo;
  for (int64_t sp = s_lo; sp <= s_hi; ++sp)
    if (fill(sp) >= best - 0.01) {
      pick = sp;
      break;
    }
  for (int q = 0; q < nq; ++q)
    splits[q] = int(std::max<int64_t>(1, std::min<int64_t>(pick, std::max<int64_t>(1, K[q] / 512))));
}

size_t pol_fp64_workspace(int nq, const int64_t* K, const int* nb, int nw, const PolOpts& o) {
  std::vector<int> splits;
  std::vector<int64_t> tiles;
  int sm = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  plan_fp64(nq, K, nb, nw, sm, o.fp64_waves, splits, tiles);
  size_t ntile = 0;
  for (int q = 0; q < nq; ++q) ntile += size_t(tiles[q]) * nw * splits[q];
  return ws_round(ntile * HT * HT * sizeof(double2));
}

int pol_fp64(int nq, const PolQ* qs, double pref, int nw, const OmegaArr& om, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx, PolOpts& o) {
  std::vector<int64_t> K(nq);
  std::vector<int> nb(nq);
  for (int q = 0; q < nq; ++q) {
    K[q] = qs[q].K;
    nb[q] = qs[q].nb;
  }
  std::vector<int> splits;
  std::vector<int64_t> tiles;
  plan_fp64(nq, K.data(), nb.data(), nw, ctx.sm_count, o.fp64_waves, splits, tiles);
  if (o.input_events)                  // every q's inputs before the first launch
    for (int q = 0; q < nq; ++q)
      if (o.input_events[q])
        GW_CUDA_TRY(cudaStreamWaitEvent(s, static_cast<cudaEvent_t>(o.input_events[q]), 0));
  for (int q0 = 0; q0 < nq; q0 += MAXQ) {
    int n = std::min(MAXQ, nq - q0);
    PolLaunch L{};
    L.nq = n;
    L.nw = nw;
    int64_t item = 0;
    size_t part = 0;
    for (int q = 0; q < n; ++q) {
      const PolQ& Q = qs[q0 + q];
      L.M[q] = static_cast<const double2*>(Q.M);
      L.delta[q] = Q.delta;
      L.dbar[q] = Q.dbar;
      L.f[q] = Q.f;
      L.P[q] = reinterpret_cast<double2*>(Q.P);
      L.K[q] = Q.K;
      L.nb[q] = Q.nb;
      L.tside[q] = (Q.nb + HT - 1) / HT;
      L.splits[q] = splits[q0 + q];
      L.item0[q] = item;
      L.part0[q] = part;
      int64_t items = tiles[q0 + q] * nw * splits[q0 + q];
      item += items;
      part += size_t(items);
    }
    L.item0[n] = item;
    if (item == 0) continue;
    if (part * HT * HT * sizeof(double2) > ws_bytes)
      return set_error(GW_EWORKSPACE, "internal: FP64 partial buffer exceeds workspace");
    double2* pbuf = static_cast<double2*>(ws);
    int rc = record_herk_event(o, o.launches, false, s);
    if (rc) return rc;
    k_herk_fp64<<<unsigned(item), 256, 0, s>>>(L, pref, om, pbuf, ctx.status);
    GW_LAUNCH_CHECK("k_herk_fp64");
    if ((rc = record_herk_event(o, o.launches, true, s))) return rc;
    ++o.launches;
    int64_t nblk = 0;
    for (int q = 0; q < n; ++q) nblk += tiles[q0 + q] * nw;
    k_herk_reduce<<<unsigned(nblk), 256, 0, s>>>(L, pbuf, o.accumulate);
    GW_LAUNCH_CHECK("k_herk_reduce");
  }
  return GW_OK;
}

}  // namespace gw
