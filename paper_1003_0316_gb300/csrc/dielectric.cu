// a3: dielectric matrix and W^c in FP64 (Eqs. dielec_MB, screen_MB; W^c = W - v).
//
//   eps = 1 - v^1/2 P v^1/2      (Hermitian positive definite on the imaginary axis)
//   eps = L L^H                   blocked right-looking Cholesky
//   Z   = L^{-1}                  blocked triangular inversion
//   W^c = v^1/2 (Z^H Z - 1) v^1/2
//
// The caller-workspace entry points factorise a workspace copy of eps right-looking over many
// CTAs (per 32-wide panel: the diagonal block, the panel below it, the trailing update of the
// lower 32x32 tiles), invert the factor by block columns (the diagonal blocks first, then one
// CTA per (system, block column) for the forward substitution of that column) and form W^c
// with one CTA per (system, 32-row block), so every phase uses every SM; each thread owns one
// row and four columns of a 32x32 tile staged in shared memory. About 4 N^3 real flops per
// system (N^3/6 complex multiply-adds per phase). Storage and the small steps (diagonal
// blocks, their inverses) are FP64; the tile products and the panel solve run in float-float
// arithmetic on the FP32 pipe, which GB300 executes 64 times faster than FP64 (see FF below):
// about 2^-48 relative per operation. The no-allocation entry point keeps the factorisation
// and the inverse inside one CTA per system, in FP64.
#include <vector>
#include <algorithm>
#include <mutex>

#include "gw_internal.cuh"

namespace gw {

constexpr int DB = 32;        // tile edge
constexpr int DLD = DB + 1;   // padded smem row
constexpr int DTHREADS = 256;

// One system. P and W^c are complex128 in global memory; the factor, the inverse and the
// panel (E, T) and the shared-memory tiles hold T: double2 for Hermitian systems, double for
// real symmetric ones (inversion-symmetric systems: the imaginary parts of P are zero and are
// not read, W^c is written with zero imaginary parts).
template <typename T>
struct DieSysT {
  const double2* P;
  double2* Wc;
  const double* v;
  T* E;      // N x N workspace (factor / inverse)
  T* Tp;     // N x DB workspace panel (inverse inside the CTA)
  T* Z;      // the inverse factor read by the W^c phase: E, or a buffer of its own
  T* D;      // inverted diagonal blocks [nt][DB][DB] (inverse by block columns), or NULL
  int n;
};

// scalar operations for the complex and the real systems
__device__ __forceinline__ double re_(double2 a) { return a.x; }
__device__ __forceinline__ double re_(double a) { return a; }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cconj(double a) { return a; }
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfma(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void csubmul(double2& x, double2 a, double2 b) {   // x -= a b
  x.x -= a.x * b.x - a.y * b.y;
  x.y -= a.x * b.y + a.y * b.x;
}
__device__ __forceinline__ void csubmul(double& x, double a, double b) { x -= a * b; }
__device__ __forceinline__ double2 scal(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double scal(double a, double s) { return a * s; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double csub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 add_re(double2 a, double d) { return make_double2(a.x + d, a.y); }
__device__ __forceinline__ double add_re(double a, double d) { return a + d; }
__device__ __forceinline__ bool fin(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ bool fin(double a) { return isfinite(a); }
template <typename T> __device__ __forceinline__ T real_of(double d);
template <> __device__ __forceinline__ double2 real_of<double2>(double d) { return make_double2(d, 0.0); }
template <> __device__ __forceinline__ double real_of<double>(double d) { return d; }
template <typename T> __device__ __forceinline__ T from_c(double2 p);
template <> __device__ __forceinline__ double2 from_c<double2>(double2 p) { return p; }
template <> __device__ __forceinline__ double from_c<double>(double2 p) { return p.x; }
__device__ __forceinline__ double2 to_c(double2 a) { return a; }
__device__ __forceinline__ double2 to_c(double a) { return make_double2(a, 0.0); }

// Load a DB x DB tile of a row-major N x N (ld) matrix at (r0, c0) into smem.
// mode 0: plain; mode 1: keep only the lower triangle (col <= row), zeros elsewhere.
template <typename T>
__device__ __forceinline__ void load_tile(T* S, const T* A, int ld, int n_rows, int n_cols, int r0,
                                          int c0, int mode) {
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    int r = e / DB, c = e % DB;
    int R = r0 + r, C = c0 + c;
    T v = T{};
    if (R < n_rows && C < n_cols && (mode == 0 || C <= R)) v = A[size_t(R) * ld + C];
    S[r * DLD + c] = v;
  }
}

// acc[b] += sum_k opA(tr, k) * SB[k][tc + 8 b]; opA = SA[tr][k] or conj(SA[k][tr]).
template <bool A_CONJ_T, typename T>
__device__ __forceinline__ void tile_mac(T acc[4], const T* SA, const T* SB, int tr, int tc) {
#pragma unroll 8
  for (int k = 0; k < DB; ++k) {
    T a = A_CONJ_T ? cconj(SA[k * DLD + tr]) : SA[tr * DLD + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) cfma(acc[b], a, SB[k * DLD + tc + 8 * b]);
  }
}

// ---- float-float tile products on the FP32 pipe ----------------------------------------------
// GB300 executes FP64 fused multiply-adds at 1/64 of its FP32 rate, so the tile products of the
// factorisation's trailing update, of the inverse by block columns and of Z^H Z run in
// float-float arithmetic: every FP64 operand becomes an unevaluated sum h + l of two FP32
// values (48 significant bits), each product h_x h_y is split exactly into its rounded value
// and error with one FMA (Dekker's product), the cross terms h_x l_y + l_x h_y are added in
// FP32 (l_x l_y and the rounding of the cross terms lie below 2^-48 of the product), and the
// running sum keeps its exact rounding errors by Knuth's two-sum in a compensation term; the
// result returns to FP64 as s + c. About 2^-48 relative per operation against 2^-53 for FP64.
// Intrinsics (__fmul_rn, __fadd_rn) keep the compiler from fusing the error-free steps.
struct FF {                // h + l, |l| <= ulp(h) / 2
  float h, l;
};
struct FFC {
  FF re, im;
};
struct FAcc {              // running sum s and compensation c: the value s + c
  float s, c;
};
struct FAccC {
  FAcc re, im;
};
template <typename T> struct FFOf;
template <> struct FFOf<double> { using tile = FF; using acc = FAcc; };
template <> struct FFOf<double2> { using tile = FFC; using acc = FAccC; };

__device__ __forceinline__ FF to_ff(double x) {
  const float h = __double2float_rn(x);
  return FF{h, __double2float_rn(x - double(h))};
}
__device__ __forceinline__ FF to_ff_t(double x) { return to_ff(x); }
__device__ __forceinline__ FFC to_ff_t(double2 x) { return FFC{to_ff(x.x), to_ff(x.y)}; }
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.h, -x.l}; }
__device__ __forceinline__ FFC ff_conj(FFC x) { return FFC{x.re, ff_neg(x.im)}; }
__device__ __forceinline__ FF ff_conj(FF x) { return x; }

// a += x y
__device__ __forceinline__ void ff_mac(FAcc& a, FF x, FF y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);                       // x.h y.h = p + e exactly
  const float t = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h));      // cross terms
  const float sum = __fadd_rn(a.s, p);                           // two-sum: a.s + p = sum + err
  const float bp = __fadd_rn(sum, -a.s);
  const float err = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(sum, -bp)), __fadd_rn(p, -bp));
  a.s = sum;
  a.c = __fadd_rn(a.c, __fadd_rn(err, __fadd_rn(e, t)));
}
__device__ __forceinline__ void ff_cmac(FAcc& a, FF x, FF y) { ff_mac(a, x, y); }
__device__ __forceinline__ void ff_cmac(FAccC& a, FFC x, FFC y) {   // a += x y, complex
  ff_mac(a.re, x.re, y.re);
  ff_mac(a.re, ff_neg(x.im), y.im);
  ff_mac(a.im, x.re, y.im);
  ff_mac(a.im, x.im, y.re);
}
__device__ __forceinline__ double ff_value(FAcc a) { return double(a.s) + double(a.c); }
__device__ __forceinline__ double ff_value_t(FAcc a) { return ff_value(a); }
__device__ __forceinline__ double2 ff_value_t(FAccC a) { return make_double2(ff_value(a.re), ff_value(a.im)); }

// the float-float value h + l of an accumulator (two-sum of s and c)
__device__ __forceinline__ FF ff_renorm(FAcc a) {
  const float h = __fadd_rn(a.s, a.c);
  const float bp = __fadd_rn(h, -a.s);
  return FF{h, __fadd_rn(__fadd_rn(a.s, -__fadd_rn(h, -bp)), __fadd_rn(a.c, -bp))};
}
__device__ __forceinline__ FF ff_renorm_t(FAcc a) { return ff_renorm(a); }
__device__ __forceinline__ FFC ff_renorm_t(FAccC a) { return FFC{ff_renorm(a.re), ff_renorm(a.im)}; }
__device__ __forceinline__ FAcc ff_acc(FF x) { return FAcc{x.h, x.l}; }
__device__ __forceinline__ FAccC ff_acc(FFC x) { return FAccC{ff_acc(x.re), ff_acc(x.im)}; }
// x y rounded to float-float (the correction is below ulp(p), so a fast two-sum renormalises)
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.h, y.h);
  const float q = __fadd_rn(__fmaf_rn(x.h, y.h, -p), __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h)));
  const float h = __fadd_rn(p, q);
  return FF{h, __fadd_rn(q, -__fadd_rn(h, -p))};
}
__device__ __forceinline__ FF ff_scale(FF x, FF r) { return ff_mul(x, r); }
__device__ __forceinline__ FFC ff_scale(FFC x, FF r) { return FFC{ff_mul(x.re, r), ff_mul(x.im, r)}; }
// acc -= x conj(l)
__device__ __forceinline__ void ff_csubmul_conj(FAcc& a, FF x, FF l) { ff_mac(a, ff_neg(x), l); }
__device__ __forceinline__ void ff_csubmul_conj(FAccC& a, FFC x, FFC l) {
  ff_mac(a.re, ff_neg(x.re), l.re);
  ff_mac(a.re, ff_neg(x.im), l.im);
  ff_mac(a.im, ff_neg(x.im), l.re);
  ff_mac(a.im, x.re, l.im);
}
__device__ __forceinline__ double ff_to_d(FF x) { return double(x.h) + double(x.l); }
__device__ __forceinline__ double ff_to_t(FF x) { return ff_to_d(x); }
__device__ __forceinline__ double2 ff_to_t(FFC x) { return make_double2(ff_to_d(x.re), ff_to_d(x.im)); }

// e - a rounded to float-float (e a float-float value, a an accumulator)
__device__ __forceinline__ FF ff_sub_acc(FF e, FAcc a) {
  const float sh = __fadd_rn(e.h, -a.s);                          // two-sum of e.h and -a.s
  const float bp = __fadd_rn(sh, -e.h);
  const float err = __fadd_rn(__fadd_rn(e.h, -__fadd_rn(sh, -bp)), __fadd_rn(-a.s, -bp));
  return ff_renorm(FAcc{sh, __fadd_rn(err, __fadd_rn(e.l, -a.c))});
}
__device__ __forceinline__ FF ff_sub_acc_t(FF e, FAcc a) { return ff_sub_acc(e, a); }
__device__ __forceinline__ FFC ff_sub_acc_t(FFC e, FAccC a) {
  return FFC{ff_sub_acc(e.re, a.re), ff_sub_acc(e.im, a.im)};
}
__device__ __forceinline__ FF ff_negate(FF x) { return ff_neg(x); }
__device__ __forceinline__ FFC ff_negate(FFC x) { return FFC{ff_neg(x.re), ff_neg(x.im)}; }

// The caller-workspace path keeps eps, its factor, the inverse factor and the inverted
// diagonal blocks in float-float form (the bytes of the FP64 element: complex FFC, real FF),
// so the tile products load them without FP64 conversions; the diagonal blocks are factorised
// and inverted in FP64 and the output W^c is FP64.
template <typename T>
using StorOf = typename FFOf<T>::tile;
template <typename T>
__device__ __forceinline__ StorOf<T>* stor(T* p) { return reinterpret_cast<StorOf<T>*>(p); }
template <typename T>
__device__ __forceinline__ const StorOf<T>* stor(const T* p) {
  return reinterpret_cast<const StorOf<T>*>(p);
}

// a DB x DB tile of float-float storage into shared memory (mode 1: lower triangle only)
template <typename FT>
__device__ __forceinline__ void load_tile_s(FT* S, const FT* A, int ld, int n_rows, int n_cols,
                                            int r0, int c0, int mode) {
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    int r = e / DB, c = e % DB;
    int R = r0 + r, C = c0 + c;
    FT v = FT{};
    if (R < n_rows && C < n_cols && (mode == 0 || C <= R)) v = A[size_t(R) * ld + C];
    S[r * DLD + c] = v;
  }
}
// the same into FP64 shared memory
template <typename T>
__device__ __forceinline__ void load_tile_s2d(T* S, const StorOf<T>* A, int ld, int n_rows,
                                              int n_cols, int r0, int c0, int mode) {
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    int r = e / DB, c = e % DB;
    int R = r0 + r, C = c0 + c;
    T v = T{};
    if (R < n_rows && C < n_cols && (mode == 0 || C <= R)) v = ff_to_t(A[size_t(R) * ld + C]);
    S[r * DLD + c] = v;
  }
}

// load_tile into float-float shared memory
template <typename T>
__device__ __forceinline__ void load_tile_ff(typename FFOf<T>::tile* S, const T* A, int ld,
                                             int n_rows, int n_cols, int r0, int c0, int mode) {
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    int r = e / DB, c = e % DB;
    int R = r0 + r, C = c0 + c;
    T v = T{};
    if (R < n_rows && C < n_cols && (mode == 0 || C <= R)) v = A[size_t(R) * ld + C];
    S[r * DLD + c] = to_ff_t(v);
  }
}

// acc[b] += sum_k opA(tr, k) * SB[k][tc + 8 b] in float-float; opA = SA[tr][k] or conj(SA[k][tr])
template <bool A_CONJ_T, typename FT, typename FA>
__device__ __forceinline__ void tile_mac_ff(FA acc[4], const FT* SA, const FT* SB, int tr, int tc) {
#pragma unroll 4
  for (int k = 0; k < DB; ++k) {
    const FT a = A_CONJ_T ? ff_conj(SA[k * DLD + tr]) : SA[tr * DLD + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) ff_cmac(acc[b], a, SB[k * DLD + tc + 8 * b]);
  }
}

constexpr int DMAXSYS = 256;   // systems per launch (descriptors passed by value)
template <typename T>
struct DieBatchT {
  DieSysT<T> s[DMAXSYS];
};

template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_dielectric(const DieBatchT<T> batch, unsigned* status,
                                                         bool invert) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  T* smem = reinterpret_cast<T*>(dsm_raw);
  T* SA = smem;
  T* SB = smem + DB * DLD;
  T* SD = smem + 2 * DB * DLD;
  __shared__ int s_fail;

  const DieSysT<T> sys = batch.s[blockIdx.x];
  const int n = sys.n;
  T* E = sys.E;
  const int tid = threadIdx.x;
  const int tr = tid >> 3, tc = tid & 7;
  if (tid == 0) s_fail = 0;

  // ---- phase 0: eps = 1 - v^1/2 P v^1/2 (full matrix) ---------------------
  for (size_t e = tid; e < size_t(n) * n; e += DTHREADS) {
    int r = int(e / n), c = int(e % n);
    double s = sqrt(sys.v[r] * sys.v[c]);
    T x = scal(from_c<T>(sys.P[e]), -s);
    if (r == c) x = add_re(x, 1.0);
    if (!fin(x)) atomicOr(&s_fail, 2);
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
        double d = re_(SD[c * DLD + c]);
        if (!(d > 0.0) || !isfinite(d)) {
          atomicOr(&s_fail, 1);
          d = 1.0;
        }
        SD[c * DLD + c] = real_of<T>(sqrt(d));
      }
      __syncthreads();
      double dinv = 1.0 / re_(SD[c * DLD + c]);
      for (int r = c + 1 + tid; r < kb; r += DTHREADS) SD[r * DLD + c] = scal(SD[r * DLD + c], dinv);
      __syncthreads();
      for (int e = tid; e < DB * DB; e += DTHREADS) {
        int r = e / DB, s = e % DB;
        if (r < kb && s > c && s <= r) {
          T x = SD[r * DLD + s];
          csubmul(x, SD[r * DLD + c], cconj(SD[s * DLD + c]));
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
      T x[DB];
      T* row = E + size_t(r) * n + k0;
#pragma unroll
      for (int c = 0; c < DB; ++c) x[c] = c < kb ? row[c] : T{};
#pragma unroll
      for (int c = 0; c < DB; ++c) {
        if (c < kb) {
          T s = x[c];
#pragma unroll
          for (int k = 0; k < c; ++k) csubmul(s, x[k], cconj(SD[c * DLD + k]));
          x[c] = scal(s, 1.0 / re_(SD[c * DLD + c]));
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
          T v = T{};
          if (R < n && k < kb) v = cconj(E[size_t(R) * n + k0 + k]);
          SB[k * DLD + c] = v;
        }
        __syncthreads();
        T acc[4] = {T{}, T{}, T{}, T{}};
        tile_mac<false>(acc, SA, SB, tr, tc);
        int R = it * DB + tr;
        if (R < n) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int C = jt * DB + tc + 8 * b;
            if (C < n && C <= R) E[size_t(R) * n + C] = csub(E[size_t(R) * n + C], acc[b]);
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
  if (!invert) return;   // the inverse follows by block columns (k_dielectric_dinv, _zcol)

  // ---- phase 2: Z = L^{-1}, lower, in place --------------------------------
  for (int kt = nt - 1; kt >= 0; --kt) {
    const int k0 = kt * DB;
    const int kb = min(DB, n - k0);
    load_tile(SD, E, n, n, n, k0, k0, 1);
    __syncthreads();
    // invert the diagonal block: column c handled by thread c
    if (tid < DB) {
      int c = tid;
      T z[DB];
#pragma unroll
      for (int i = 0; i < DB; ++i) z[i] = T{};
      if (c < kb) {
        z[c] = real_of<T>(1.0 / re_(SD[c * DLD + c]));
#pragma unroll
        for (int i = 0; i < DB; ++i) {
          if (i > c && i < kb) {
            T s = T{};
            for (int k = c; k < i; ++k) cfma(s, SD[i * DLD + k], z[k]);
            z[i] = scal(s, -1.0 / re_(SD[i * DLD + i]));
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
        T acc[4] = {T{}, T{}, T{}, T{}};
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
          for (int b = 0; b < 4; ++b) sys.Tp[size_t(R) * DB + tc + 8 * b] = acc[b];
        }
      }
      __syncthreads();
      // Z21 = -T * Z11
      for (int it = kt + 1; it < nt; ++it) {
        load_tile(SA, sys.Tp, DB, n, DB, it * DB, 0, 0);
        __syncthreads();
        T acc[4] = {T{}, T{}, T{}, T{}};
        tile_mac<false>(acc, SA, SD, tr, tc);
        int R = it * DB + tr;
        if (R < n) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int C = tc + 8 * b;
            if (C < kb) E[size_t(R) * n + k0 + C] = scal(acc[b], -1.0);
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

  // phase 3 (W^c from Z) runs as its own launch over (system, block row): k_dielectric_w
}

// ---- phase 3: W^c = v^1/2 (Z^H Z - 1) v^1/2, one CTA per (system, 32-row block rt) ---------
// (the lower tiles ct <= rt of the block row and their Hermitian mirror)
template <typename T, bool FS>
__global__ void __launch_bounds__(DTHREADS) k_dielectric_w(const DieBatchT<T> batch) {
  using FT = typename FFOf<T>::tile;
  using FA = typename FFOf<T>::acc;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  FT* SA = reinterpret_cast<FT*>(dsm_raw);      // float-float tiles (the size of T)
  FT* SB = SA + DB * DLD;
  const DieSysT<T> sys = batch.s[blockIdx.x];
  const int n = sys.n;
  const int nt = (n + DB - 1) / DB;
  const int rt = blockIdx.y;
  if (rt >= nt) return;                      // whole CTA, before any barrier
  const T* E = sys.Z;
  const int tid = threadIdx.x;
  const int tr = tid >> 3, tc = tid & 7;
  __shared__ double svr[DB], svc[DB];        // square roots of v of the tile's rows and columns
  if (tid < DB) svr[tid] = rt * DB + tid < n ? sqrt(sys.v[rt * DB + tid]) : 0.0;
  for (int ct = 0; ct <= rt; ++ct) {
    __syncthreads();                          // the previous tile's epilogue has read svc
    if (tid < DB) svc[tid] = ct * DB + tid < n ? sqrt(sys.v[ct * DB + tid]) : 0.0;
    FA acc[4] = {};
    for (int kt2 = rt; kt2 < nt; ++kt2) {
      if (FS) {                              // Z in float-float storage
        load_tile_s(SA, stor(E), n, n, n, kt2 * DB, rt * DB, 1);   // Z[K][R] (lower part)
        load_tile_s(SB, stor(E), n, n, n, kt2 * DB, ct * DB, 1);   // Z[K][S]
      } else {                               // Z in FP64 (the no-allocation entry)
        load_tile_ff<T>(SA, E, n, n, n, kt2 * DB, rt * DB, 1);
        load_tile_ff<T>(SB, E, n, n, n, kt2 * DB, ct * DB, 1);
      }
      __syncthreads();
      tile_mac_ff<true>(acc, SA, SB, tr, tc);
      __syncthreads();
    }
    int R = rt * DB + tr;
    if (R < n) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int C = ct * DB + tc + 8 * b;
        if (C < n && C <= R) {
          T x = ff_value_t(acc[b]);
          if (C == R) x = real_of<T>(re_(x) - 1.0);
          x = scal(x, svr[tr] * svc[tc + 8 * b]);
          sys.Wc[size_t(R) * n + C] = to_c(x);
          if (C != R) sys.Wc[size_t(C) * n + R] = to_c(cconj(x));
        }
      }
    }
  }
}

// ---- the inverse Z = L^{-1} by block columns (the columns of Z are independent forward
// substitutions L Z_c = I_c): first every diagonal block inverted, one CTA per (system, block)
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_dielectric_dinv(const DieBatchT<T> batch) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  T* SD = reinterpret_cast<T*>(dsm_raw);
  const DieSysT<T> sys = batch.s[blockIdx.x];
  const int n = sys.n;
  const int nt = (n + DB - 1) / DB;
  const int r = blockIdx.y;
  if (r >= nt) return;
  const int k0 = r * DB;
  const int kb = min(DB, n - k0);
  load_tile_s2d(SD, stor(sys.E), n, n, n, k0, k0, 1);
  __syncthreads();
  if (threadIdx.x < DB) {
    const int c = threadIdx.x;
    T z[DB];
#pragma unroll
    for (int i = 0; i < DB; ++i) z[i] = T{};
    if (c < kb) {
      z[c] = real_of<T>(1.0 / re_(SD[c * DLD + c]));
#pragma unroll
      for (int i = 0; i < DB; ++i) {
        if (i > c && i < kb) {
          T acc = T{};
          for (int k = c; k < i; ++k) cfma(acc, SD[i * DLD + k], z[k]);
          z[i] = scal(acc, -1.0 / re_(SD[i * DLD + i]));
        }
      }
    }
    StorOf<T>* Dr = stor(sys.D) + size_t(r) * DB * DB;
#pragma unroll
    for (int i = 0; i < DB; ++i) Dr[i * DB + c] = to_ff_t(z[i]);
  }
}

// then one CTA per (system, block column c): for r = c, c + 1, ...
//   Z[r][c] = D_r (delta_rc - sum_{k = c}^{r-1} L[r][k] Z[k][c])
// with the earlier blocks Z[k][c] of the same column read back from global memory.
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_dielectric_zcol(const DieBatchT<T> batch) {
  using FT = typename FFOf<T>::tile;
  using FA = typename FFOf<T>::acc;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  FT* SA = reinterpret_cast<FT*>(dsm_raw);      // float-float tiles (the size of T)
  FT* SB = SA + DB * DLD;
  const DieSysT<T> sys = batch.s[blockIdx.x];
  const int n = sys.n;
  const int nt = (n + DB - 1) / DB;
  const int c = blockIdx.y;
  if (c >= nt) return;                       // whole CTA, before any barrier
  const int tid = threadIdx.x;
  const int tr = tid >> 3, tc = tid & 7;
  StorOf<T>* Z = stor(sys.Z);
  const StorOf<T>* L = stor(sys.E);
  for (int r = c; r < nt; ++r) {
    FT out[4] = {FT{}, FT{}, FT{}, FT{}};
    if (r == c) {
      const FT* Dr = stor(sys.D) + size_t(r) * DB * DB;
#pragma unroll
      for (int b = 0; b < 4; ++b) out[b] = Dr[tr * DB + tc + 8 * b];
    } else {
      FA acc[4] = {};
      for (int k = c; k < r; ++k) {
        load_tile_s(SA, L, n, n, n, r * DB, k * DB, 0);              // L[r][k]
        load_tile_s(SB, Z, n, n, n, k * DB, c * DB, k == c ? 1 : 0); // Z[k][c]
        __syncthreads();
        tile_mac_ff<false>(acc, SA, SB, tr, tc);
        __syncthreads();
      }
      // out = -D_r acc: the product tile in SB, D_r in SA
#pragma unroll
      for (int b = 0; b < 4; ++b) SB[tr * DLD + tc + 8 * b] = ff_renorm_t(acc[b]);
      const FT* Dr = stor(sys.D) + size_t(r) * DB * DB;
      for (int e = tid; e < DB * DB; e += DTHREADS) SA[(e / DB) * DLD + e % DB] = Dr[e];
      __syncthreads();
      FA o[4] = {};
      tile_mac_ff<false>(o, SA, SB, tr, tc);
      __syncthreads();
#pragma unroll
      for (int b = 0; b < 4; ++b) out[b] = ff_negate(ff_renorm_t(o[b]));
    }
    const int R = r * DB + tr;
    if (R < n) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int C = c * DB + tc + 8 * b;
        if (C < n) Z[size_t(R) * n + C] = out[b];
      }
    }
    __syncthreads();                          // this block row is read by the next ones
  }
}

// ---- the factorisation over many CTAs (the caller-workspace entry points) -----------------
// A right-looking blocked Cholesky with one launch per step and panel kt: the diagonal block
// (one CTA per system), the panel below it (one CTA per system and 256 rows, one row per
// thread), the trailing update of the lower tiles (one CTA per system and 32 x 32 tile). Every
// SM takes part however few systems there are (20 systems of N_b = 4096 would leave 132 of
// 152 SMs idle with one CTA per system).

// eps = 1 - v^1/2 P v^1/2 over the full matrix: grid (32-row blocks, system); the square roots
// of v are taken once per row and column block (FP64 square roots are costly on GB300's FP64
// pipe) and kept in shared memory
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_eps_fill(const DieBatchT<T> batch, unsigned* status) {
  __shared__ double svr[DB], svc[DTHREADS];
  const DieSysT<T>& sys = batch.s[blockIdx.y];
  const int n = sys.n;
  const int r0 = blockIdx.x * DB;
  if (r0 >= n) return;                       // whole CTA, before any barrier
  const int tid = threadIdx.x;
  if (tid < DB) svr[tid] = r0 + tid < n ? sqrt(sys.v[r0 + tid]) : 0.0;
  bool bad = false;
  for (int c0 = 0; c0 < n; c0 += DTHREADS) {
    __syncthreads();                          // the previous chunk's svc is read
    svc[tid] = c0 + tid < n ? sqrt(sys.v[c0 + tid]) : 0.0;
    __syncthreads();
    const int c = c0 + tid;
    if (c >= n) continue;
    for (int rr = 0; rr < DB && r0 + rr < n; ++rr) {
      const size_t e = size_t(r0 + rr) * n + c;
      T x = scal(from_c<T>(sys.P[e]), -(svr[rr] * svc[tid]));
      if (r0 + rr == c) x = add_re(x, 1.0);
      if (!fin(x)) bad = true;
      stor(sys.E)[e] = to_ff_t(x);
    }
  }
  if (bad) raise_status(status, ST_ENONFINITE);
}

// in-place Cholesky of the kb x kb lower block held in shared memory (SD, ld DLD); returns
// false (through *fail) on a non-positive or non-finite pivot, which is replaced by 1
template <typename T>
__device__ void chol_block_smem(T* SD, int kb, int* fail) {
  const int tid = threadIdx.x;
  for (int c = 0; c < kb; ++c) {
    if (tid == 0) {
      double d = re_(SD[c * DLD + c]);
      if (!(d > 0.0) || !isfinite(d)) {
        *fail = 1;
        d = 1.0;
      }
      SD[c * DLD + c] = real_of<T>(sqrt(d));
    }
    __syncthreads();
    const double dinv = 1.0 / re_(SD[c * DLD + c]);
    for (int r = c + 1 + tid; r < kb; r += DTHREADS) SD[r * DLD + c] = scal(SD[r * DLD + c], dinv);
    __syncthreads();
    for (int e = tid; e < DB * DB; e += DTHREADS) {
      const int r = e / DB, s = e % DB;
      if (r < kb && s > c && s <= r) {
        T x = SD[r * DLD + s];
        csubmul(x, SD[r * DLD + c], cconj(SD[s * DLD + c]));
        SD[r * DLD + s] = x;
      }
    }
    __syncthreads();
  }
}

// step 1 of panel kt: the diagonal block, one CTA per system
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_chol_diag(const DieBatchT<T> batch, int kt,
                                                        unsigned* status) {
  __shared__ T SD[DB * DLD];
  __shared__ int s_fail;
  const DieSysT<T>& sys = batch.s[blockIdx.x];
  const int n = sys.n, nt = (n + DB - 1) / DB;
  if (kt >= nt) return;                      // whole CTA, before any barrier
  const int k0 = kt * DB, kb = min(DB, n - k0);
  if (threadIdx.x == 0) s_fail = 0;
  load_tile_s2d(SD, stor(sys.E), n, n, n, k0, k0, 1);
  __syncthreads();
  chol_block_smem(SD, kb, &s_fail);
  for (int e = threadIdx.x; e < DB * DB; e += DTHREADS) {
    const int r = e / DB, c = e % DB;
    if (r < kb && c <= r) stor(sys.E)[size_t(k0 + r) * n + k0 + c] = to_ff_t(SD[r * DLD + c]);
  }
  if (threadIdx.x == 0 && s_fail) raise_status(status, ST_ENOTHPD);
}

// step 2: the panel X L_kk^H = A_ik below the diagonal block, one row per thread, in
// float-float (the reciprocals of the diagonal in FP64); grid (256-row blocks of the trailing
// rows, system)
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_chol_panel(const DieBatchT<T> batch, int kt) {
  using FT = typename FFOf<T>::tile;
  using FA = typename FFOf<T>::acc;
  __shared__ FT SD[DB * DLD];
  __shared__ FF rinv[DB];
  const DieSysT<T>& sys = batch.s[blockIdx.y];
  const int n = sys.n, nt = (n + DB - 1) / DB;
  if (kt >= nt - 1) return;                  // no rows below the last block
  const int k0 = kt * DB;                    // a full block: kt < nt - 1
  const int r0 = k0 + DB + blockIdx.x * DTHREADS;
  if (r0 >= n) return;                       // whole CTA, before any barrier
  load_tile_s(SD, stor(sys.E), n, n, n, k0, k0, 1);
  if (threadIdx.x < DB)
    rinv[threadIdx.x] = to_ff(1.0 / re_(ff_to_t(stor(sys.E)[size_t(k0 + threadIdx.x) * n + k0 + threadIdx.x])));
  __syncthreads();
  const int r = r0 + threadIdx.x;
  if (r < n) {
    FT x[DB];
    FT* row = stor(sys.E) + size_t(r) * n + k0;
#pragma unroll
    for (int c = 0; c < DB; ++c) x[c] = row[c];
#pragma unroll
    for (int c = 0; c < DB; ++c) {
      FA acc = ff_acc(x[c]);
#pragma unroll
      for (int k = 0; k < c; ++k) ff_csubmul_conj(acc, x[k], SD[c * DLD + k]);
      x[c] = ff_scale(ff_renorm_t(acc), rinv[c]);
    }
#pragma unroll
    for (int c = 0; c < DB; ++c) row[c] = x[c];
  }
}

// step 3: the trailing update A_ij -= L_ik L_jk^H for kt < j <= i (lower tiles; the diagonal
// tiles keep their lower triangle); grid (tiles of the largest system, system)
template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_chol_update(const DieBatchT<T> batch, int kt) {
  using FT = typename FFOf<T>::tile;
  using FA = typename FFOf<T>::acc;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  FT* SA = reinterpret_cast<FT*>(dsm_raw);      // float-float tiles (the size of T)
  FT* SB = SA + DB * DLD;
  const DieSysT<T>& sys = batch.s[blockIdx.y];
  const int n = sys.n, nt = (n + DB - 1) / DB;
  const int m = nt - kt - 1;                 // trailing block rows
  const int64_t t = blockIdx.x;
  if (m <= 0 || t >= int64_t(m) * (m + 1) / 2) return;   // whole CTA, before any barrier
  // t -> (ii, jj), 0 <= jj <= ii < m, row by row
  int ii = int((sqrt(8.0 * double(t) + 1.0) - 1.0) * 0.5);
  while (int64_t(ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (int64_t(ii) * (ii + 1) / 2 > t) --ii;
  const int jj = int(t - int64_t(ii) * (ii + 1) / 2);
  const int it = kt + 1 + ii, jt = kt + 1 + jj;
  const int k0 = kt * DB;
  const int tid = threadIdx.x, tr = tid >> 3, tc = tid & 7;
  FT* E = stor(sys.E);
  load_tile_s(SA, E, n, n, n, it * DB, k0, 0);                // L_ik
  for (int e = tid; e < DB * DB; e += DTHREADS) {             // SB[k][c] = conj(L_jk[c][k])
    const int k = e / DB, c = e % DB;
    const int R = jt * DB + c;
    SB[k * DLD + c] = R < n ? ff_conj(E[size_t(R) * n + k0 + k]) : FT{};
  }
  __syncthreads();
  FA acc[4] = {};
  tile_mac_ff<false>(acc, SA, SB, tr, tc);
  const int R = it * DB + tr;
  if (R < n) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int C = jt * DB + tc + 8 * b;
      if (C < n && C <= R) E[size_t(R) * n + C] = ff_sub_acc_t(E[size_t(R) * n + C], acc[b]);
    }
  }
}

template <typename T>
static int launch_cholesky_grid(const DieBatchT<T>& batch, int nsys, int ntmax, cudaStream_t s,
                                const DeviceCtx& ctx) {
  const size_t smem_u = 2 * DB * DLD * sizeof(T);
  int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_chol_update<T>), smem_u, ctx.device);
  if (rc) return rc;
  int nmax = 0;
  for (int i = 0; i < nsys; ++i) nmax = std::max(nmax, batch.s[i].n);
  k_eps_fill<T><<<dim3(unsigned((nmax + DB - 1) / DB), unsigned(nsys)), DTHREADS, 0, s>>>(batch,
                                                                                        ctx.status);
  GW_LAUNCH_CHECK("k_eps_fill");
  for (int kt = 0; kt < ntmax; ++kt) {
    k_chol_diag<T><<<unsigned(nsys), DTHREADS, 0, s>>>(batch, kt, ctx.status);
    GW_LAUNCH_CHECK("k_chol_diag");
    const int rows = nmax - (kt + 1) * DB;
    if (rows <= 0) continue;
    const unsigned pb = unsigned((rows + DTHREADS - 1) / DTHREADS);
    k_chol_panel<T><<<dim3(pb, unsigned(nsys)), DTHREADS, 0, s>>>(batch, kt);
    GW_LAUNCH_CHECK("k_chol_panel");
    const int64_t m = ntmax - kt - 1;
    k_chol_update<T><<<dim3(unsigned(m * (m + 1) / 2), unsigned(nsys)), DTHREADS, smem_u, s>>>(batch, kt);
    GW_LAUNCH_CHECK("k_chol_update");
  }
  return GW_OK;
}

template <typename T>
static int launch_dielectric(std::vector<DieSysT<T>>& sys, cudaStream_t s, const DeviceCtx& ctx) {
  const size_t smem = 3 * DB * DLD * sizeof(T);
  const size_t smem_w = 2 * DB * DLD * sizeof(T);
  {
    int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_dielectric<T>), smem, ctx.device);
    if (!rc) rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_dielectric_w<T, true>), smem_w, ctx.device);
    if (!rc) rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_dielectric_w<T, false>), smem_w, ctx.device);
    if (!rc) rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_dielectric_zcol<T>), smem_w, ctx.device);
    if (rc) return rc;
  }
  const bool by_columns = !sys.empty() && sys[0].D != nullptr;
  for (size_t b0 = 0; b0 < sys.size(); b0 += DMAXSYS) {
    size_t nb_ = std::min<size_t>(DMAXSYS, sys.size() - b0);
    DieBatchT<T> batch;
    int ntmax = 1;
    for (size_t i = 0; i < nb_; ++i) {
      batch.s[i] = sys[b0 + i];
      ntmax = std::max(ntmax, (batch.s[i].n + DB - 1) / DB);
    }
    if (by_columns) {
      // caller workspace: the factorisation over many CTAs, then the inverse by block columns
      int rc = launch_cholesky_grid<T>(batch, int(nb_), ntmax, s, ctx);
      if (rc) return rc;
    } else {
      // no-allocation entry: factorisation and inverse inside one CTA per system
      k_dielectric<T><<<unsigned(nb_), DTHREADS, smem, s>>>(batch, ctx.status, true);
      GW_LAUNCH_CHECK("k_dielectric");
    }
    if (by_columns) {
      const dim3 g2(static_cast<unsigned>(nb_), static_cast<unsigned>(ntmax));
      k_dielectric_dinv<T><<<g2, DTHREADS, DB * DLD * sizeof(T), s>>>(batch);
      GW_LAUNCH_CHECK("k_dielectric_dinv");
      k_dielectric_zcol<T><<<g2, DTHREADS, smem_w, s>>>(batch);
      GW_LAUNCH_CHECK("k_dielectric_zcol");
    }
    if (by_columns)
      k_dielectric_w<T, true><<<dim3(unsigned(nb_), unsigned(ntmax)), DTHREADS, smem_w, s>>>(batch);
    else
      k_dielectric_w<T, false><<<dim3(unsigned(nb_), unsigned(ntmax)), DTHREADS, smem_w, s>>>(batch);
    GW_LAUNCH_CHECK("k_dielectric_w");
  }
  return GW_OK;
}

template <typename T>
static size_t dielectric_ws_t(int nq, const int* nb, int nw) {
  size_t b = 0;
  for (int q = 0; q < nq; ++q) {
    size_t n = size_t(nb[q]);
    const size_t nt = (n + DB - 1) / DB;
    b += size_t(nw) * ws_round((2 * n * n + nt * DB * DB) * sizeof(T));   // E, Z, D
  }
  return b;
}

template <typename T>
static int dielectric_t(int nq, const int* nb, int nw, const double* const* v,
                        const double* const* P, double* const* Wc, void* ws, size_t ws_bytes,
                        cudaStream_t s, const DeviceCtx& ctx) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  std::vector<DieSysT<T>> sys;
  for (int q = 0; q < nq; ++q) {
    size_t n = size_t(nb[q]);
    for (int j = 0; j < nw; ++j) {
      DieSysT<T> d;
      d.P = reinterpret_cast<const double2*>(P[q]) + size_t(j) * n * n;
      d.Wc = reinterpret_cast<double2*>(Wc[q]) + size_t(j) * n * n;
      d.v = v[q];
      const size_t nt = (n + DB - 1) / DB;
      char* blk = static_cast<char*>(cur.take((2 * n * n + nt * DB * DB) * sizeof(T)));
      if (!blk) return set_error(GW_EWORKSPACE, "internal: dielectric workspace too small");
      d.E = reinterpret_cast<T*>(blk);       // eps, then its Cholesky factor
      d.Tp = nullptr;                         // (the in-CTA inverse's panel: not used here)
      d.Z = d.E + n * n;                      // the inverse factor, by block columns
      d.D = d.Z + n * n;                      // the inverted diagonal blocks
      d.n = int(n);
      sys.push_back(d);
    }
  }
  return launch_dielectric<T>(sys, s, ctx);
}

size_t dielectric_workspace(int nq, const int* nb, int nw) {
  return dielectric_ws_t<double2>(nq, nb, nw);
}
size_t dielectric_real_workspace(int nq, const int* nb, int nw) {
  return dielectric_ws_t<double>(nq, nb, nw);
}

int dielectric_wc(int nq, const int* nb, int nw, const double* const* v, const double* const* P,
                  double* const* Wc, void* ws, size_t ws_bytes, cudaStream_t s,
                  const DeviceCtx& ctx) {
  return dielectric_t<double2>(nq, nb, nw, v, P, Wc, ws, ws_bytes, s, ctx);
}

int dielectric_wc_real(int nq, const int* nb, int nw, const double* const* v,
                       const double* const* P, double* const* Wc, void* ws, size_t ws_bytes,
                       cudaStream_t s, const DeviceCtx& ctx) {
  return dielectric_t<double>(nq, nb, nw, v, P, Wc, ws, ws_bytes, s, ctx);
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
  for (int j0 = 0; j0 < nw; j0 += int(fit)) {
    const int cnt = std::min<int>(int(fit), nw - j0);
    std::vector<DieSysT<double2>> sys(cnt);
    for (int i = 0; i < cnt; ++i) {
      DieSysT<double2>& d = sys[i];
      const int j = j0 + i;
      d.P = reinterpret_cast<const double2*>(P) + size_t(j) * n * n;
      d.Wc = reinterpret_cast<double2*>(Wc) + size_t(j) * n * n;
      d.v = v;
      d.E = reinterpret_cast<double2*>(base + size_t(i) * per);
      d.Tp = d.E + n * n;
      d.Z = d.E;                              // inverse in place, inside the CTA
      d.D = nullptr;
      d.n = nb;
    }
    rc = launch_dielectric<double2>(sys, s, ctx);
    if (rc) return rc;
  }
  return GW_OK;
}

}  // namespace gw
