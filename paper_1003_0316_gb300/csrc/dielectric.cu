// a3: dielectric matrix and W^c in FP64 (Eqs. dielec_MB, screen_MB; W^c = W - v).
//
//   eps = 1 - v^1/2 P v^1/2      (Hermitian positive definite on the imaginary axis)
//   eps = L L^H                   blocked right-looking Cholesky
//   Z   = L^{-1}                  blocked triangular inversion
//   W^c = v^1/2 (Z^H Z - 1) v^1/2
//
// One CTA per (q, frequency) system works through the three phases in place on a
// workspace copy of eps, with 32x32 complex tiles staged in shared memory; each
// thread owns one row and four columns of a tile. The phases are FP64-pipe bound:
// about 4 N^3 real flops per system (N^3/6 complex multiply-adds each).
#include <vector>
#include <algorithm>
#include <mutex>

#include "gw_internal.cuh"

namespace gw {

constexpr int DB = 32;        // tile edge
constexpr int DLD = DB + 1;   // padded smem row
constexpr int DTHREADS = 256;

struct DieSys {
  const double2* P;
  double2* Wc;
  const double* v;
  double2* E;      // N x N workspace (factor / inverse)
  double2* T;      // N x DB workspace panel
  int n;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// Load a DB x DB tile of a row-major N x N (ld) matrix at (r0, c0) into smem.
// mode 0: plain; mode 1: keep only the lower triangle (col <= row), zeros elsewhere.
__device__ __forceinline__ void load_tile(double2* S, const double2* A, int ld, int n_rows,
                                          int n_cols, int r0, int c0, int mode) {
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    int r = e / DB, c = e % DB;
    int R = r0 + r, C = c0 + c;
    double2 v = make_double2(0.0, 0.0);
    if (R < n_rows && C < n_cols && (mode == 0 || C <= R)) v = A[size_t(R) * ld + C];
    S[r * DLD + c] = v;
  }
}

// acc[b] += sum_k opA(tr, k) * SB[k][tc + 8 b]; opA = SA[tr][k] or conj(SA[k][tr]).
template <bool A_CONJ_T>
__device__ __forceinline__ void tile_mac(double2 acc[4], const double2* SA, const double2* SB,
                                         int tr, int tc) {
#pragma unroll 8
  for (int k = 0; k < DB; ++k) {
    double2 a = A_CONJ_T ? cconj(SA[k * DLD + tr]) : SA[tr * DLD + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) cfma(acc[b], a, SB[k * DLD + tc + 8 * b]);
  }
}

constexpr int DMAXSYS = 256;   // systems per launch (descriptors passed by value)
struct DieBatch {
  DieSys s[DMAXSYS];
};

__global__ void __launch_bounds__(DTHREADS) k_dielectric(const DieBatch batch, unsigned* status) {
  extern __shared__ double2 smem[];
  double2* SA = smem;
  double2* SB = smem + DB * DLD;
  double2* SD = smem + 2 * DB * DLD;
  __shared__ int s_fail;

  const DieSys sys = batch.s[blockIdx.x];
  const int n = sys.n;
  double2* E = sys.E;
  const int tid = threadIdx.x;
  const int tr = tid >> 3, tc = tid & 7;
  if (tid == 0) s_fail = 0;

  // ---- phase 0: eps = 1 - v^1/2 P v^1/2 (full matrix) ---------------------
  for (size_t e = tid; e < size_t(n) * n; e += DTHREADS) {
    int r = int(e / n), c = int(e % n);
    double s = sqrt(sys.v[r] * sys.v[c]);
    double2 p = sys.P[e];
    double2 x = make_double2(-s * p.x, -s * p.y);
    if (r == c) x.x += 1.0;
    if (!isfinite(x.x) || !isfinite(x.y)) atomicOr(&s_fail, 2);
    E[e] = x;
  }
  __syncthreads();

  const int nt = (n + DB - 1) / DB;
  // ---- phase 1: Cholesky, lower, in place ---------------------------------
  for (int kt = 0; kt < nt; ++kt) {
    const int k0 = kt * DB;
    const int kb = min(DB, n - k0);
    load_tile(SD, E, n, n, n, k0, k0, 1);
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
      if (tid == 0) {
        double d = SD[c * DLD + c].x;
        if (!(d > 0.0) || !isfinite(d)) {
          atomicOr(&s_fail, 1);
          d = 1.0;
        }
        SD[c * DLD + c] = make_double2(sqrt(d), 0.0);
      }
      __syncthreads();
      double dinv = 1.0 / SD[c * DLD + c].x;
      for (int r = c + 1 + tid; r < kb; r += DTHREADS) {
        double2 x = SD[r * DLD + c];
        SD[r * DLD + c] = make_double2(x.x * dinv, x.y * dinv);
      }
      __syncthreads();
      for (int e = tid; e < DB * DB; e += DTHREADS) {
        int r = e / DB, s = e % DB;
        if (r < kb && s > c && s <= r) {
          double2 a = SD[r * DLD + c], b = cconj(SD[s * DLD + c]);
          double2 x = SD[r * DLD + s];
          x.x -= a.x * b.x - a.y * b.y;
          x.y -= a.x * b.y + a.y * b.x;
          SD[r * DLD + s] = x;
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < DB * DB; e += DTHREADS) {
      int r = e / DB, c = e % DB;
      if (r < kb && c <= r) E[size_t(k0 + r) * n + k0 + c] = SD[r * DLD + c];
    }
    __syncthreads();
    // panel: X L11^H = A21, one row per thread
    for (int r = k0 + kb + tid; r < n; r += DTHREADS) {
      double2 x[DB];
      double2* row = E + size_t(r) * n + k0;
#pragma unroll
      for (int c = 0; c < DB; ++c) x[c] = c < kb ? row[c] : make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < DB; ++c) {
        if (c < kb) {
          double2 s = x[c];
#pragma unroll
          for (int k = 0; k < c; ++k) {
            double2 l = cconj(SD[c * DLD + k]);
            s.x -= x[k].x * l.x - x[k].y * l.y;
            s.y -= x[k].x * l.y + x[k].y * l.x;
          }
          double di = 1.0 / SD[c * DLD + c].x;
          x[c] = make_double2(s.x * di, s.y * di);
        }
      }
#pragma unroll
      for (int c = 0; c < DB; ++c)
        if (c < kb) row[c] = x[c];
    }
    __syncthreads();
    // trailing update: A22 -= X X^H (lower tiles)
    for (int it = kt + 1; it < nt; ++it) {
      load_tile(SA, E, n, n, n, it * DB, k0, 0);   // X rows of tile it
      for (int jt = kt + 1; jt <= it; ++jt) {
        // SB[k][c] = conj(X[jt*DB + c][k0 + k])
        for (int e = tid; e < DB * DB; e += DTHREADS) {
          int k = e / DB, c = e % DB;
          int R = jt * DB + c;
          double2 v = make_double2(0.0, 0.0);
          if (R < n && k < kb) v = cconj(E[size_t(R) * n + k0 + k]);
          SB[k * DLD + c] = v;
        }
        __syncthreads();
        double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0),
                          make_double2(0, 0)};
        tile_mac<false>(acc, SA, SB, tr, tc);
        int R = it * DB + tr;
        if (R < n) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int C = jt * DB + tc + 8 * b;
            if (C < n && C <= R) {
              double2 x = E[size_t(R) * n + C];
              E[size_t(R) * n + C] = make_double2(x.x - acc[b].x, x.y - acc[b].y);
            }
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) raise_status(status, (s_fail & 1) ? ST_ENOTHPD : ST_ENONFINITE);
    return;
  }

  // ---- phase 2: Z = L^{-1}, lower, in place --------------------------------
  for (int kt = nt - 1; kt >= 0; --kt) {
    const int k0 = kt * DB;
    const int kb = min(DB, n - k0);
    load_tile(SD, E, n, n, n, k0, k0, 1);
    __syncthreads();
    // invert the diagonal block: column c handled by thread c
    if (tid < DB) {
      int c = tid;
      double2 z[DB];
#pragma unroll
      for (int i = 0; i < DB; ++i) z[i] = make_double2(0.0, 0.0);
      if (c < kb) {
        z[c] = make_double2(1.0 / SD[c * DLD + c].x, 0.0);
#pragma unroll
        for (int i = 0; i < DB; ++i) {
          if (i > c && i < kb) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = c; k < i; ++k) cfma(s, SD[i * DLD + k], z[k]);
            double di = 1.0 / SD[i * DLD + i].x;
            z[i] = make_double2(-s.x * di, -s.y * di);
          }
        }
      }
      // stash the inverted column in SB (column c)
#pragma unroll
      for (int i = 0; i < DB; ++i) SB[i * DLD + c] = z[i];
    }
    __syncthreads();
    // SD <- inverse of the diagonal block
    for (int e = tid; e < DB * DB; e += DTHREADS) {
      int r = e / DB, c = e % DB;
      SD[r * DLD + c] = SB[r * DLD + c];
    }
    __syncthreads();
    if (k0 + kb < n) {
      // T[R] = Z22[R][:] * L21 over the trailing rows (Z22 already inverted)
      for (int it = kt + 1; it < nt; ++it) {
        double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0),
                          make_double2(0, 0)};
        for (int st = kt + 1; st <= it; ++st) {
          load_tile(SA, E, n, n, n, it * DB, st * DB, st == it ? 1 : 0);   // Z22 block
          load_tile(SB, E, n, n, n, st * DB, k0, 0);                        // L21 block
          __syncthreads();
          tile_mac<false>(acc, SA, SB, tr, tc);
          __syncthreads();
        }
        int R = it * DB + tr;
        if (R < n) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int C = tc + 8 * b;
            sys.T[size_t(R) * DB + C] = acc[b];
          }
        }
      }
      __syncthreads();
      // Z21 = -T * Z11
      for (int it = kt + 1; it < nt; ++it) {
        load_tile(SA, sys.T, DB, n, DB, it * DB, 0, 0);
        __syncthreads();
        double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0),
                          make_double2(0, 0)};
        tile_mac<false>(acc, SA, SD, tr, tc);
        int R = it * DB + tr;
        if (R < n) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int C = tc + 8 * b;
            if (C < kb) E[size_t(R) * n + k0 + C] = make_double2(-acc[b].x, -acc[b].y);
          }
        }
        __syncthreads();
      }
    }
    for (int e = tid; e < DB * DB; e += DTHREADS) {
      int r = e / DB, c = e % DB;
      if (r < kb && c <= r) E[size_t(k0 + r) * n + k0 + c] = SD[r * DLD + c];
    }
    __syncthreads();
  }

  // ---- phase 3: W^c = v^1/2 (Z^H Z - 1) v^1/2 ------------------------------
  for (int rt = 0; rt < nt; ++rt) {
    for (int ct = 0; ct <= rt; ++ct) {
      double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0),
                        make_double2(0, 0)};
      for (int kt2 = rt; kt2 < nt; ++kt2) {
        load_tile(SA, E, n, n, n, kt2 * DB, rt * DB, 1);   // Z[K][R] (lower part)
        load_tile(SB, E, n, n, n, kt2 * DB, ct * DB, 1);   // Z[K][S]
        __syncthreads();
        tile_mac<true>(acc, SA, SB, tr, tc);
        __syncthreads();
      }
      int R = rt * DB + tr;
      if (R < n) {
        double vr = sys.v[R];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int C = ct * DB + tc + 8 * b;
          if (C < n && C <= R) {
            double2 x = acc[b];
            if (C == R) {
              x.x -= 1.0;
              x.y = 0.0;
            }
            double s = sqrt(vr * sys.v[C]);
            x = make_double2(s * x.x, s * x.y);
            sys.Wc[size_t(R) * n + C] = x;
            if (C != R) sys.Wc[size_t(C) * n + R] = cconj(x);
          }
        }
      }
    }
  }
}

size_t dielectric_workspace(int nq, const int* nb, int nw) {
  size_t b = 0;
  size_t nsys = 0;
  for (int q = 0; q < nq; ++q) {
    size_t n = size_t(nb[q]);
    b += size_t(nw) * ws_round((n * n + n * DB) * sizeof(double2));
    nsys += nw;
  }
  return b;
}

int dielectric_wc(int nq, const int* nb, int nw, const double* const* v, const double* const* P,
                  double* const* Wc, void* ws, size_t ws_bytes, cudaStream_t s,
                  const DeviceCtx& ctx) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  std::vector<DieSys> sys;
  for (int q = 0; q < nq; ++q) {
    size_t n = size_t(nb[q]);
    for (int j = 0; j < nw; ++j) {
      DieSys d;
      d.P = reinterpret_cast<const double2*>(P[q]) + size_t(j) * n * n;
      d.Wc = reinterpret_cast<double2*>(Wc[q]) + size_t(j) * n * n;
      d.v = v[q];
      char* blk = static_cast<char*>(cur.take((n * n + n * DB) * sizeof(double2)));
      if (!blk) return set_error(GW_EWORKSPACE, "internal: dielectric workspace too small");
      d.E = reinterpret_cast<double2*>(blk);
      d.T = d.E + n * n;
      d.n = int(n);
      sys.push_back(d);
    }
  }
  size_t smem = 3 * DB * DLD * sizeof(double2);
  static bool attr_set[64] = {};
  if (!attr_set[ctx.device]) {
    GW_CUDA_TRY(cudaFuncSetAttribute(k_dielectric, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
    attr_set[ctx.device] = true;
  }
  for (size_t b0 = 0; b0 < sys.size(); b0 += DMAXSYS) {
    size_t nb_ = std::min<size_t>(DMAXSYS, sys.size() - b0);
    DieBatch batch;
    for (size_t i = 0; i < nb_; ++i) batch.s[i] = sys[b0 + i];
    k_dielectric<<<unsigned(nb_), DTHREADS, smem, s>>>(batch, ctx.status);
    GW_LAUNCH_CHECK("k_dielectric");
  }
  return GW_OK;
}

// ---------------------------------------------------------------- no-alloc variant
// Scratch for callers that cannot allocate: a static device array (one per device that
// loads the library). Host code only ever uses the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GW_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static char* g_noalloc_ptr[64];

static int noalloc_scratch(const DeviceCtx& ctx, char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[ctx.device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[ctx.device] = static_cast<char*>(p);
  }
  *out = g_noalloc_ptr[ctx.device];
  return GW_OK;
}

int dielectric_wc_noalloc(int nb, int nw, const double* v, const double* P, double* Wc,
                          cudaStream_t s, const DeviceCtx& ctx) {
  const size_t n = size_t(nb);
  const size_t per = ws_round((n * n + n * DB) * sizeof(double2));
  if (per > GW_NOALLOC_SCRATCH_BYTES)
    return set_error(GW_EINVAL, "nb=%d needs %zu bytes of scratch per system, more than the "
                     "%u-byte static scratch of the no-alloc entry point", nb, per,
                     GW_NOALLOC_SCRATCH_BYTES);
  char* base = nullptr;
  int rc = noalloc_scratch(ctx, &base);
  if (rc) return rc;
  const size_t fit = std::min<size_t>(GW_NOALLOC_SCRATCH_BYTES / per, DMAXSYS);
  const size_t smem = 3 * DB * DLD * sizeof(double2);
  static bool attr_set[64] = {};
  if (!attr_set[ctx.device]) {
    GW_CUDA_TRY(cudaFuncSetAttribute(k_dielectric, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
    attr_set[ctx.device] = true;
  }
  for (int j0 = 0; j0 < nw; j0 += int(fit)) {
    const int cnt = std::min<int>(int(fit), nw - j0);
    DieBatch batch;
    for (int i = 0; i < cnt; ++i) {
      DieSys& d = batch.s[i];
      const int j = j0 + i;
      d.P = reinterpret_cast<const double2*>(P) + size_t(j) * n * n;
      d.Wc = reinterpret_cast<double2*>(Wc) + size_t(j) * n * n;
      d.v = v;
      d.E = reinterpret_cast<double2*>(base + size_t(i) * per);
      d.T = d.E + n * n;
      d.n = nb;
    }
    k_dielectric<<<unsigned(cnt), DTHREADS, smem, s>>>(batch, ctx.status);
    GW_LAUNCH_CHECK("k_dielectric (no-alloc)");
  }
  return GW_OK;
}

}  // namespace gw
