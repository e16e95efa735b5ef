// a2 tensor-core path: P_IJ(q, i w_j) = sum_t w_tj M_tI conj(M_tJ) (Eq. polar_MB at
// w = i omega) on tcgen05 with split-precision operands.
//
// The complex rank-K update is one real weighted Gram matrix: with x the FP32
// interleaved view of M ([K][2 N_b]) and s_tj = |w_tj|,
//   G_j = x^T diag(s_j) x,   P_IJ = -(G[2I][2J] + G[2I+1][2J+1]) - i (G[2I+1][2J] - G[2I][2J+1]).
// A CTA tile is 128 rows (A: the s_tj-scaled columns of x) by 128 columns (B: the plain
// columns of x) of G_j for one frequency. Every operand y is split as y = hi + lo (TF32
// or BF16 pieces, each rounded to nearest) and each product is formed as
//   lo_A*hi_B + hi_A*lo_B + hi_A*hi_B
// by three MMAs into the same TMEM accumulator.
//
// Accuracy: the tensor core adds into its FP32 accumulator with truncation, which
// biases a long chain of additions toward zero (about 2e-8 of the running value per
// MMA). A round is two 64-byte K chunks (2 x 16 TF32 or 2 x 32 BF16 transitions, 12 MMAs);
// every drain period of PL rounds on one accumulator (PL = 1: one round) therefore starts a
// fresh accumulator; the epilogue adds each period's result into FP32 running sums held in
// its registers (round to nearest) and folds them into FP64 every 256 periods (FP64
// reductions performed at L2 into per-CTA sums), so no truncating chain is longer than 12 PL
// MMAs; the round-to-nearest FP32 sums add only unbiased errors that average out over the
// folds.
//
// Layout and roles (512 threads in four warpgroups, one persistent CTA per SM; 512 TMEM
// columns):
//   TMEM  cols [0,256): two accumulators (round g uses g mod 2, PL rounds per drain);
//         cols [256,512): four A slots of one round each (per chunk 16 columns hi + 16 lo);
//         round g uses slot g mod 4, so each A set owns two slots and can fill one while
//         the MMAs still read the other.
//   warps 0-7    A transform: scale x by s_tj, split, tcgen05.st into the A slot of their
//                lane quadrant; set g mod 2 (warps 4 (g mod 2) .. + 3) takes round g;
//   warp 8       one thread issues the bulk copies of a round's pre-split B tiles into a
//                4-stage shared-memory ring;
//   warps 9-10   one thread each issues the MMAs (A from TMEM, B from shared memory) of the
//                rounds of one accumulator, and tcgen05.commit;
//   warp 11      one thread issues the bulk copies of the rounds' weights into an 8-slot ring
//                of their own, so the A sets can run ahead of the B stages;
//   warps 12-15  epilogue, one per lane quadrant: tcgen05.ld of the finished accumulator
//                into FP32 running sums in registers (the warpgroup raises its register
//                budget with setmaxnreg, the producer/MMA warpgroup lowers its own), FP64
//                folding, the final complex combination and the Hermitian store.
// Every barrier is waited on only by threads that see each of its phases in order (a
// parity wait cannot tell phase p from phase p + 2): the stage, slot and weight-slot counts
// are even, so the A set and the MMA issuer of round g also handled rounds g - NSB, g - NSA
// and g - NWS.
// The same kernel forms the Sigma pair coefficients as a quadratic form (MODE 1: A = the pair
// projections, B = the real form of W^c, c_p = row sums of (X R) o X) and the real polarization
// of inversion-symmetric systems (MODE 2, real operand of width N_b).
// Only tiles that meet the upper triangle (complex I <= J) are computed. Every mbarrier
// wait is bounded; on expiry the CTA records a timeout in the status word and winds
// down, waiting for its own MMAs before releasing TMEM.
#include <vector>
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <cuda_bf16.h>

#include "gw_internal.cuh"
#include "tc_ptx.cuh"

namespace gw {

namespace {

constexpr int TM = 128;          // real Gram rows per tile (A operand, in TMEM)
constexpr int TN = 128;          // real Gram columns per tile (B operand, in shared memory)
constexpr int SWB = 64;          // bytes of K per B row per chunk (64-byte swizzle)
constexpr int SUB = 2;           // 64-byte K chunks per barrier round
// B stages (rounds) in shared memory: a template parameter of the kernel, 4 (default) or 6
constexpr int NSA = 4;           // A slots (rounds) in TMEM: two per A set
constexpr int NWS = 8;           // weight slots (rounds) in shared memory
constexpr int B_TILE = TN * SWB;                 // 8 KB: one chunk's hi (or lo) tile
constexpr int CHUNK_BYTES = 2 * B_TILE;          // hi + lo of one chunk (pre-split layout)
constexpr int STAGE_BYTES = SUB * CHUNK_BYTES;   // one round
constexpr int WSLOT_BYTES = 256;                 // one round's weights (SUB x 32 floats at most)
constexpr uint32_t ACC_COL = 0;                  // two accumulators: cols [0,128), [128,256)
constexpr uint32_t A_COL = 2 * TN;               // A slots: [256,512), 64 columns each
constexpr int A_WARPS = 8;       // warps 0-7: A transform, two sets of one warp per quadrant
constexpr int PROD_WARP = A_WARPS;       // one thread: bulk copies of B tiles
constexpr int MMA_WARP = A_WARPS + 1;    // two warps issue the MMAs of even and odd rounds
constexpr int WPROD_WARP = A_WARPS + 3;  // one thread: bulk copies of the weights
constexpr int EPI_WARP0 = A_WARPS + 4;   // four warps: epilogue, one per lane quadrant
constexpr int NEPI = 4;
constexpr int NWARPS = EPI_WARP0 + NEPI;
constexpr int NTHREADS = NWARPS * 32;
constexpr int REG_LOW = 40;      // registers per thread of the producer/MMA warpgroup
constexpr int REG_EPI = 216;     // ... of the epilogue warpgroup (128 + 128 - 40 at launch)
constexpr int PL = 1;                            // own rounds per drain period and accumulator
constexpr int FLUSH = 256;                       // periods per FP64 fold of the running sums
constexpr int TQ = 64;
constexpr uint64_t WAIT_LIMIT = 2000000000ull;   // ns: 2 s per bounded wait
static_assert(NTHREADS == 512 && REG_EPI + REG_LOW == 2 * 128, "register split");

// Wait profile, compiled in only with GW_HERK_WAIT_PROFILE defined: the SM cycles (clock64)
// that the issuing thread of each role spends in its barrier waits, in its drain and fold work
// and in total, summed over the CTAs into g_herk_prof (the order of include/gw.h's
// GW_HERK_WAIT_COUNTERS); in a normal build every counter is dead code.
#ifdef GW_HERK_WAIT_PROFILE
constexpr bool kWaitProfile = true;
#else
constexpr bool kWaitProfile = false;
#endif
enum HerkProf {
  HP_A_TOTAL, HP_A_WAIT_W, HP_A_WAIT_SLOT, HP_A_ROUNDS,
  HP_MMA_TOTAL, HP_MMA_WAIT_B, HP_MMA_WAIT_A, HP_MMA_WAIT_ACC, HP_MMA_ROUNDS,
  HP_EPI_TOTAL, HP_EPI_WAIT_ACC, HP_EPI_DRAIN, HP_EPI_FOLD, HP_EPI_PERIODS,
  HP_BP_TOTAL, HP_BP_WAIT, HP_WP_TOTAL, HP_WP_WAIT, HP_N
};
static_assert(HP_N == GW_HERK_WAIT_COUNTERS, "counter list of include/gw.h");
__device__ unsigned long long g_herk_prof[HP_N];

__device__ __forceinline__ uint64_t hp_now() {
  if constexpr (kWaitProfile) return clock64();
  return 0;
}
__device__ __forceinline__ void hp_flush(int i, uint64_t v) {
  if constexpr (kWaitProfile) atomicAdd(&g_herk_prof[i], static_cast<unsigned long long>(v));
}

struct TcLaunch {
  int accumulate;           // P += the tile's sum instead of P = (slices of K into one P)
  const float* xT[TQ];      // A side, chunk-major: float4 [row block][kpad / CH][CH / 4][128 rows]
  const char* bsp[TQ];      // [nbi][nch] pre-split B tiles: 8 KB hi + 8 KB lo, swizzled
  const float* s[TQ];       // [nw][kpad] |w_tj| in FP32 (zero padded)
  double2* P[TQ];           // polarization output (Hermitian store)
  double* cq[TQ];           // quadratic-form output c[nw][nrow] (accumulated with atomics)
  int64_t bsp_jstride[TQ];  // bytes between the B tiles of consecutive frequencies (0: shared)
  int64_t nrow[TQ];         // valid A rows (quadratic form)
  int64_t K[TQ];
  int64_t kpad[TQ];
  int nb[TQ];
  int nbi[TQ];
  int nbj[TQ];              // B column blocks (three-product layout: N_b blocks nbb)
  int ntile[TQ];
  int prod3[TQ];            // complex polarization in three real products (see k_prep_tc3)
  double* g3[TQ];           // their tiles: [nw][C, S][col][row], 128 nbj rows and columns
  int64_t item0[TQ + 1];
  int nq;
  int nw;
};

// Work item -> q, frequency j, A block bi and B block bj (data blocks of the chunk-major copy
// and of the pre-split tiles) and the tile kind: 0 an upper tile of the real Gram matrix of
// the interleaved projections (or of the real ones), 1 a tile of C = Mr^T diag(s) Mi, 2 an
// upper tile of S = (Mr + Mi)^T diag(s) (Mr + Mi) (three-product layout), 3 a tile of the
// quadratic form.
// the q of a work item only
__device__ __forceinline__ int item_q(const TcLaunch& L, int64_t item) {
  int q = 0;
  while (q + 1 < L.nq && item >= L.item0[q + 1]) ++q;
  return q;
}

template <bool QF>
__device__ __forceinline__ void decode_item(const TcLaunch& L, int64_t item, int& q, int& j,
                                            int& bi, int& bj, int& kind) {
  q = 0;
  while (q + 1 < L.nq && item >= L.item0[q + 1]) ++q;
  int64_t loc = item - L.item0[q];
  int u = int(loc % L.ntile[q]);
  j = int(loc / L.ntile[q]);
  if (QF) {             // full rectangular grid; consecutive items share the B column block
    bi = u % L.nbi[q];
    bj = u / L.nbi[q];
    kind = 3;
    return;
  }
  int off = 0;
  kind = 0;
  if (L.prod3[q]) {
    const int nbb = L.nbj[q];
    if (u < nbb * nbb) {  // C: every tile; consecutive items share the B column block
      bi = u % nbb;
      bj = u / nbb;
      kind = 1;
      return;
    }
    u -= nbb * nbb;
    off = nbb;
    kind = 2;
  }
  bj = 0;
  while (u > bj) {      // upper tiles bi <= bj, column by column
    u -= bj + 1;
    ++bj;
  }
  bi = u + off;
  bj += off;
}

// Rounds of a work item: the q's whole K range, except for the quadratic form, whose B operand
// is the upper triangle of the form (k <= c): column block bj needs the K blocks 0 .. bj only.
// nr_all: the rounds of the whole K range (the stride of the pre-split B tiles).
template <bool QF, int CH>
__device__ __forceinline__ int64_t item_rounds(const TcLaunch& L, int q, int bj, int64_t& nr_all) {
  nr_all = ((L.K[q] + CH - 1) / CH + SUB - 1) / SUB;
  if (!QF) return nr_all;
  const int64_t k = L.K[q] < int64_t(bj + 1) * TN ? L.K[q] : int64_t(bj + 1) * TN;
  return ((k + CH - 1) / CH + SUB - 1) / SUB;
}

// byte offset of (row n, 16-byte chunk kc) in a K-major, 64-byte-swizzled tile
__device__ __forceinline__ uint32_t sw64_off(int n, int kc) {
  return uint32_t((n >> 3) * 512 + (n & 7) * 64 + ((kc ^ ((n & 7) >> 1)) << 4));
}

// Round an FP32 value to TF32 (10 explicit mantissa bits), to nearest with ties away from
// zero, on the bit pattern: adding half a TF32 unit in the last place (bit 12) and clearing the
// 13 dropped bits rounds the magnitude up exactly when the dropped part is at least half a unit
// (a carry into the exponent is the correct result). Valid for every finite value below the
// FP32 maximum, which covers the scaled projections.
__device__ __forceinline__ uint32_t tf32_rna(float y) {
  return (__float_as_uint(y) + 0x1000u) & 0xFFFFE000u;
}

// y -> (hi, lo) pieces packed as 32-bit TMEM / shared-memory words.
// TF32: one value per word. BF16: two consecutive K values per word (low half first).
template <bool BF16>
__device__ __forceinline__ void split_words(const float* y, uint32_t* hi, uint32_t* lo, int nwords) {
  if (!BF16) {
    for (int i = 0; i < nwords; ++i) {
      uint32_t h = tf32_rna(y[i]);
      hi[i] = h;
      lo[i] = tf32_rna(y[i] - __uint_as_float(h));
    }
  } else {
    for (int i = 0; i < nwords; ++i) {
      const uint32_t h = tc::cvt_bf16x2(y[2 * i], y[2 * i + 1]);     // both hi pieces, RN
      const float h0 = __uint_as_float(h << 16), h1 = __uint_as_float(h & 0xFFFF0000u);
      hi[i] = h;
      lo[i] = tc::cvt_bf16x2(y[2 * i] - h0, y[2 * i + 1] - h1);
    }
  }
}

// TF32 pieces of packed pairs of values (pair i = values 2i, 2i + 1, low word first), the
// subtraction of the hi pieces by paired instructions: the same pieces as split_words<false>
// with fewer instructions (measured: TF32x3 polarization 14.7 -> 13.9 ms on one q of
// K = 102,400; the same for BF16 pieces brought nothing).
__device__ __forceinline__ void split_pairs_tf32(const uint64_t* yp, uint32_t* hi, uint32_t* lo,
                                                 int nwords) {
  for (int i = 0; i < nwords / 2; ++i) {
    float y0, y1;
    tc::f2_unpack(yp[i], y0, y1);
    const uint32_t h0 = tf32_rna(y0), h1 = tf32_rna(y1);
    float r0, r1;
    tc::f2_unpack(tc::f2_sub(yp[i], tc::f2_pack(h0, h1)), r0, r1);
    hi[2 * i] = h0;
    hi[2 * i + 1] = h1;
    lo[2 * i] = tf32_rna(r0);
    lo[2 * i + 1] = tf32_rna(r1);
  }
}

// One bounded wait by lane 0, broadcast to the warp; raises the abort flag on expiry.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          unsigned* status) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) {
    ok = (!*abort && tc::mbar_wait(bar, parity, abort, WAIT_LIMIT)) ? 1 : 0;
    if (!ok && !*abort) {
      *abort = 1;
      raise_status(status, ST_ETIMEOUT);
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// MODE: 0 complex polarization, 1 quadratic form (Sigma pair coefficients), 2 real
// polarization (real projections, inversion-symmetric systems: P = -G directly).
template <bool BF16, int MODE, int NSB>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_herk_tc(const __grid_constant__ TcLaunch L, double* __restrict__ acc64, unsigned* status) {
  constexpr bool QF = MODE == 1;
  constexpr int CH = BF16 ? 32 : 16;          // transitions per chunk (64 bytes of K)
  constexpr int CH4 = CH / 4;                 // float4 per chunk column
  constexpr uint32_t IDESC = tc::instr_desc(BF16 ? 1u : 2u, TM, TN);

  extern __shared__ __align__(1024) char dsmem[];
  char* ring = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
  char* wring = ring + NSB * STAGE_BYTES;     // weight slots
  __shared__ __align__(8) uint64_t fullB[NSB], emptyB[NSB], fullA[NSA], emptyA[NSA], fullW[NWS],
      emptyW[NWS], accf_bar[2], acce_bar[2], done_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSB; ++i) {
      tc::mbar_init(&fullB[i], 1);
      tc::mbar_init(&emptyB[i], 1);
    }
    for (int i = 0; i < NSA; ++i) {
      tc::mbar_init(&fullA[i], 4);         // the set's four warps
      tc::mbar_init(&emptyA[i], 1);
    }
    for (int i = 0; i < NWS; ++i) {
      tc::mbar_init(&fullW[i], 1);
      tc::mbar_init(&emptyW[i], 4);        // the set's four warps have read the weights
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&accf_bar[i], 1);
      tc::mbar_init(&acce_bar[i], NEPI);   // every epilogue warp drains every period
    }
    tc::mbar_init(&done_bar[0], 1);
    tc::mbar_init(&done_bar[1], 1);
    s_abort = 0;
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t nitems = L.item0[L.nq];

  if (warp < A_WARPS) {
    // ------------------------------------------------ A transform -> TMEM
    // A set par (warps 4 par .. 4 par + 3, one per lane quadrant) takes the rounds g with
    // g mod 2 == par (g counted over all items of this CTA); round g goes to A slot g mod 4.
    // Each lane reads its column's values from the chunk-major copy (each float4 read of a
    // warp is 512 contiguous bytes; a ring of register buffers keeps the reads of the next
    // chunks in flight while the current one is split) and the round's weights from the
    // weight ring.
    constexpr int RA = BF16 ? 2 : 4;            // chunks of column reads in flight
    const int qd = warp & 3, par = warp >> 2;
    const int m = qd * 32 + lane;
    uint64_t g0 = 0;                  // rounds of the previous items
    bool stop = false;
    const uint64_t hp0 = hp_now();
    uint64_t hp_ww = 0, hp_ws = 0, hp_n = 0;
    for (int64_t item = blockIdx.x; item < nitems && !stop; item += gridDim.x) {
      int q, j, bi, bj, kind;
      decode_item<QF>(L, item, q, j, bi, bj, kind);
      int64_t nr_all;
      const int64_t nr = item_rounds<QF, CH>(L, q, bj, nr_all);
      const float4* __restrict__ xc = reinterpret_cast<const float4*>(L.xT[q]) +
                                      size_t(bi) * size_t(L.kpad[q] / CH) * CH4 * TM + m;
      const int64_t r_first = int64_t((par + 2 - int(g0 & 1)) & 1);
      const int64_t nown = nr > r_first ? (nr - r_first + 1) / 2 : 0;
      // own chunk k (k = 0 .. SUB nown - 1) is chunk SUB (r_first + 2 (k / SUB)) + k % SUB
      auto load = [&](int64_t k, float4 (&rg)[CH4]) {
        const int64_t c = SUB * (r_first + 2 * (k / SUB)) + k % SUB;
#pragma unroll
        for (int e = 0; e < CH4; ++e) rg[e] = __ldg(xc + size_t(c * CH4 + e) * TM);
      };
      // chunk k of the own rounds: the first one of a round waits for the round's weights;
      // the chunk is scaled and split before the wait for the A slot, so that work overlaps
      // the MMAs still reading the slot; the last chunk releases the weights and signals the
      // slot full
      auto process = [&](int64_t k, const float4 (&xr)[CH4]) -> bool {
        const int u = int(k % SUB);
        const uint64_t gg = g0 + uint64_t(r_first + 2 * (k / SUB));
        const int slot = int(gg % NSA), ws = int(gg % NWS);
        uint64_t t = hp_now();
        if (!QF && u == 0 && !warp_wait(&fullW[ws], uint32_t(gg / NWS) & 1, &s_abort, status))
          return false;
        hp_ww += hp_now() - t;
        const float4* sw = reinterpret_cast<const float4*>(wring + ws * WSLOT_BYTES) + u * CH4;
        uint32_t hw[2][8], lw[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {               // halves of the chunk: 8 TMEM words each
          if constexpr (BF16) {
            float y[CH / 2];
#pragma unroll
            for (int e = 0; e < CH4 / 2; ++e) {
              const float4 xv = xr[h * (CH4 / 2) + e];
              const float4 wv = QF ? make_float4(1.f, 1.f, 1.f, 1.f) : sw[h * (CH4 / 2) + e];
              y[4 * e + 0] = wv.x * xv.x;
              y[4 * e + 1] = wv.y * xv.y;
              y[4 * e + 2] = wv.z * xv.z;
              y[4 * e + 3] = wv.w * xv.w;
            }
            split_words<true>(y, hw[h], lw[h], 8);
          } else {                                  // scaled values in packed pairs
            uint64_t yp[CH / 4];
#pragma unroll
            for (int e = 0; e < CH4 / 2; ++e) {
              const float4 xv = xr[h * (CH4 / 2) + e];
              const uint64_t x01 = tc::f2_pack(__float_as_uint(xv.x), __float_as_uint(xv.y));
              const uint64_t x23 = tc::f2_pack(__float_as_uint(xv.z), __float_as_uint(xv.w));
              if (QF) {
                yp[2 * e] = x01;
                yp[2 * e + 1] = x23;
              } else {
                const float4 wv = sw[h * (CH4 / 2) + e];
                yp[2 * e] = tc::f2_mul(tc::f2_pack(__float_as_uint(wv.x), __float_as_uint(wv.y)), x01);
                yp[2 * e + 1] =
                    tc::f2_mul(tc::f2_pack(__float_as_uint(wv.z), __float_as_uint(wv.w)), x23);
              }
            }
            split_pairs_tf32(yp, hw[h], lw[h], 8);
          }
        }
        if (!QF && u == SUB - 1) {                  // this warp is done with the weights
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&emptyW[ws]);
        }
        t = hp_now();
        if (u == 0 && !warp_wait(&emptyA[slot], (uint32_t(gg / NSA) & 1) ^ 1, &s_abort, status))
          return false;
        hp_ws += hp_now() - t;
        hp_n += u == 0;
        const uint32_t base = tmem + (uint32_t(qd * 32) << 16) + A_COL + slot * (SUB * 32) + u * 32;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tc::tmem_st8(base + h * 8, hw[h]);
          tc::tmem_st8(base + 16 + h * 8, lw[h]);
        }
        if (u == SUB - 1) {
          tc::tmem_wait_st();
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&fullA[slot]);
        }
        return true;
      };
      const int64_t nk = SUB * nown;
      // ring of RA register buffers: the reads of the next RA - 1 own chunks are in flight
      float4 X[RA][CH4];
#pragma unroll
      for (int v = 0; v < RA - 1; ++v)
        if (v < nk) load(v, X[v]);
      for (int64_t kb = 0; kb < nk && !stop; kb += RA) {
#pragma unroll
        for (int v = 0; v < RA; ++v) {
          const int64_t k = kb + v;
          if (k >= nk) break;
          if (k + RA - 1 < nk) load(k + RA - 1, X[(v + RA - 1) % RA]);
          if (!process(k, X[v])) {
            stop = true;
            break;
          }
        }
      }
      g0 += uint64_t(nr);
    }
    if (kWaitProfile && lane == 0) {
      hp_flush(HP_A_TOTAL, hp_now() - hp0);
      hp_flush(HP_A_WAIT_W, hp_ww);
      hp_flush(HP_A_WAIT_SLOT, hp_ws);
      hp_flush(HP_A_ROUNDS, hp_n);
    }
  } else if (warp < EPI_WARP0) {
    tc::setmaxnreg_dec<REG_LOW>();
    if (warp == PROD_WARP) {
      // ---------------------------------------------- B tiles: bulk copies
      // One round per stage: the SUB consecutive pre-split chunk tiles (contiguous).
      if (lane == 0) {
        uint64_t g = 0;
        bool ok = true;
        const uint64_t hp0 = hp_now();
        uint64_t hp_w = 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
          int q, j, bi, bj, kind;
          decode_item<QF>(L, item, q, j, bi, bj, kind);
          int64_t nr_all;
          const int64_t nr = item_rounds<QF, CH>(L, q, bj, nr_all);
          const char* src = L.bsp[q] + size_t(j) * L.bsp_jstride[q] +
                            size_t(bj) * size_t(nr_all * SUB) * CHUNK_BYTES;
          for (int64_t r = 0; r < nr; ++r, ++g) {
            const int st = int(g % NSB);
            const uint64_t t = hp_now();
            if (!tc::mbar_wait(&emptyB[st], (uint32_t(g / NSB) & 1) ^ 1, &s_abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            hp_w += hp_now() - t;
            char* dst = ring + st * STAGE_BYTES;
            tc::mbar_arrive_expect_tx(&fullB[st], STAGE_BYTES);
            tc::bulk_g2s(dst, src + size_t(r) * STAGE_BYTES, STAGE_BYTES, &fullB[st]);
          }
        }
        if (!ok && !s_abort) {
          s_abort = 1;
          raise_status(status, ST_ETIMEOUT);
        }
        if (kWaitProfile) {
          hp_flush(HP_BP_TOTAL, hp_now() - hp0);
          hp_flush(HP_BP_WAIT, hp_w);
        }
      }
      __syncwarp();
    } else if (warp == WPROD_WARP) {
      // ---------------------------------------------- weights: bulk copies
      // One round per weight slot: the round's SUB CH weights (SUB CH 4 bytes, 16-byte
      // aligned). With BF16 pieces this thread also asks L2 to prefetch the A columns
      // (contiguous, 16-byte aligned) of the round PD rounds behind the one whose weights it
      // copies, i.e. about three rounds ahead of the A sets (it runs at most NWS ahead of them),
      // so that their loads find the columns in L2 (measured on one q of K = 102,400: BF16x3
      // 9.65 -> 7.84 ms; the same for TF32 pieces, or a prefetch eight rounds ahead, or of the
      // B tiles as well, raised the DRAM reads and slowed TF32x3 down: 14.8 -> 16.7 ms).
      // The quadratic form has no weights (its operands are small and stay in L2).
      if (!QF && lane == 0) {
        uint64_t g = 0;
        bool ok = true;
        const uint64_t hp0 = hp_now();
        uint64_t hp_w = 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
          int q, j, bi, bj, kind;
          decode_item<QF>(L, item, q, j, bi, bj, kind);
          int64_t nr_all;
          const int64_t nr = item_rounds<QF, CH>(L, q, bj, nr_all);
          const float* wsrc = L.s[q] + size_t(j) * L.kpad[q];
          const char* xsrc = reinterpret_cast<const char*>(L.xT[q]) +
                             size_t(bi) * size_t(L.kpad[q] / CH) * CH4 * TM * 16;
          for (int64_t r = 0; r < nr; ++r, ++g) {
            const int ws = int(g % NWS);
            const uint64_t t = hp_now();
            if (!tc::mbar_wait(&emptyW[ws], (uint32_t(g / NWS) & 1) ^ 1, &s_abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            hp_w += hp_now() - t;
            tc::mbar_arrive_expect_tx(&fullW[ws], SUB * CH * 4);
            tc::bulk_g2s(wring + ws * WSLOT_BYTES, wsrc + r * SUB * CH, SUB * CH * 4, &fullW[ws]);
            if (BF16) {
              constexpr int64_t PD = NWS - 3;
              const uint32_t xb = SUB * CH4 * TM * 16;           // one round of A columns
              if (r == 0)                                         // the item's first rounds
                for (int64_t r2 = 0; r2 < PD && r2 < nr; ++r2)
                  tc::bulk_prefetch_l2(xsrc + size_t(r2) * xb, xb);
              if (r >= PD) tc::bulk_prefetch_l2(xsrc + size_t(r - PD) * xb, xb);
            }
          }
        }
        if (!ok && !s_abort) {
          s_abort = 1;
          raise_status(status, ST_ETIMEOUT);
        }
        if (kWaitProfile) {
          hp_flush(HP_WP_TOTAL, hp_now() - hp0);
          hp_flush(HP_WP_WAIT, hp_w);
        }
      }
      __syncwarp();
    } else {
      // ---------------------------------------------- MMA issue (two threads, alternate rounds)
      // Round g goes to accumulator g mod 2 and is issued by MMA warp g mod 2 (g counted over
      // all items), so the barrier waits of one issuing thread overlap the tensor-core work of
      // the other. Each round is one drain period: SUB chunks x 2 K steps x 3 MMAs into a
      // fresh accumulator.
      const uint32_t mpar = uint32_t(warp - MMA_WARP);
      if (lane == 0) {
        uint64_t g = 0;
        uint32_t kb = 0;              // periods issued on this warp's accumulator
        const uint64_t desc0 = tc::smem_desc(tc::smem_u32(ring), 512, 4);
        const uint32_t d = tmem + ACC_COL + mpar * TN;
        bool ok = true;
        const uint64_t hp0 = hp_now();
        uint64_t hp_wb = 0, hp_wa = 0, hp_wc = 0, hp_n = 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
          int q, bj = 0;
          if (QF) {
            int j, bi, kind;
            decode_item<QF>(L, item, q, j, bi, bj, kind);
          } else {
            q = item_q(L, item);
          }
          int64_t nr_all;
          const int64_t nr = item_rounds<QF, CH>(L, q, bj, nr_all);
          const int64_t first = int64_t((mpar + 2 - uint32_t(g & 1)) & 1);
          const int64_t nown = nr > first ? (nr - first + 1) / 2 : 0;   // own rounds of the item
          for (int64_t i = 0; i < nown; ++i) {
            const int64_t r = first + 2 * i;
            // a drain period is PL own rounds (fewer at the end of the item)
            const bool pstart = i % PL == 0, pend = i % PL == PL - 1 || i == nown - 1;
            const uint64_t gg = g + uint64_t(r);
            const int st = int(gg % NSB), slot = int(gg % NSA);
            const uint64_t t0 = hp_now();
            if (!tc::mbar_wait(&fullB[st], uint32_t(gg / NSB) & 1, &s_abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            const uint64_t t1 = hp_now();
            if (!tc::mbar_wait(&fullA[slot], uint32_t(gg / NSA) & 1, &s_abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            const uint64_t t2 = hp_now();
            if (pstart && !tc::mbar_wait(&acce_bar[mpar], (kb & 1) ^ 1, &s_abort, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            hp_wb += t1 - t0;
            hp_wa += t2 - t1;
            hp_wc += hp_now() - t2;
            ++hp_n;
            tc::tc_fence_after();
            const uint32_t a0 = tmem + A_COL + slot * (SUB * 32);
            // descriptor address field is (addr >> 4): advancing the address adds to the low bits
            const uint64_t dst = desc0 + uint64_t((st * STAGE_BYTES) >> 4);
#pragma unroll
            for (int u = 0; u < SUB; ++u) {
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t dBh = dst + uint64_t((u * CHUNK_BYTES + ks * 32) >> 4);
                const uint64_t dBl = dst + uint64_t((u * CHUNK_BYTES + B_TILE + ks * 32) >> 4);
                const uint32_t ah = a0 + u * 32 + ks * 8, al = a0 + u * 32 + 16 + ks * 8;
                const uint32_t acc0 = (pstart && u == 0 && ks == 0) ? 0u : 1u;
                if (BF16) {
                  tc::mma_f16_ta(d, al, dBh, IDESC, acc0);
                  tc::mma_f16_ta(d, ah, dBl, IDESC, 1u);
                  tc::mma_f16_ta(d, ah, dBh, IDESC, 1u);
                } else {
                  tc::mma_tf32_ta(d, al, dBh, IDESC, acc0);
                  tc::mma_tf32_ta(d, ah, dBl, IDESC, 1u);
                  tc::mma_tf32_ta(d, ah, dBh, IDESC, 1u);
                }
              }
            }
            tc::mma_commit(&emptyB[st]);
            tc::mma_commit(&emptyA[slot]);
            if (pend) {
              tc::mma_commit(&accf_bar[mpar]);
              ++kb;
            }
          }
          g += uint64_t(nr);
        }
        if (!ok && !s_abort) {
          s_abort = 1;
          raise_status(status, ST_ETIMEOUT);
        }
        if (kWaitProfile) {
          hp_flush(HP_MMA_TOTAL, hp_now() - hp0);
          hp_flush(HP_MMA_WAIT_B, hp_wb);
          hp_flush(HP_MMA_WAIT_A, hp_wa);
          hp_flush(HP_MMA_WAIT_ACC, hp_wc);
          hp_flush(HP_MMA_ROUNDS, hp_n);
        }
        tc::mma_commit(&done_bar[mpar]);
        int never = 0;
        tc::mbar_wait(&done_bar[mpar], 0, reinterpret_cast<volatile int*>(&never), WAIT_LIMIT);
      }
      __syncwarp();
    }
  } else {
    tc::setmaxnreg_inc<REG_EPI>();
    // ------------------------------------------------ drain / epilogue
    // Each period's accumulator is added into FP32 running sums in registers (round to
    // nearest): one read of the accumulator per period, no TMEM write. Every FLUSH periods
    // (staggered over the warps) the sums are folded into FP64 with L2 reductions.
    const int qd = warp & 3;
    const int r = qd * 32 + lane;               // tile row
    const uint32_t lane_base = tmem + (uint32_t(qd * 32) << 16);
    double* acc = acc64 + size_t(blockIdx.x) * TN * TM + r;   // [col][row]
    uint32_t kb0 = 0, kb1 = 0;      // periods drained per accumulator
    uint32_t gp = 0;                // periods drained in total (flush schedule)
    uint64_t g0 = 0;                // rounds of the previous items
    bool stop = false;
    const uint64_t hp0 = hp_now();
    uint64_t hp_wc = 0, hp_dr = 0, hp_fo = 0, hp_n = 0;
    float rs[TN];
    // the conversions go through volatile asm so that they stay next to their reductions
    // (converted all at once, 128 doubles would not fit beside the running sums)
    // quadratic form: this row's c_p part of the item, x_p . (sums), compensated in FP32
    // (the exact FP32 product as p + e by FMA, added by two-sum); qx: the item's x_p columns
    float qs = 0.0f, qc = 0.0f;
    const float4* qx = nullptr;
    auto fold = [&]() {
      if constexpr (QF) {
        // columns bj TN + i of row p in the chunk-major copy: float4 group i / 4 of the block
        // sits at ((i / CH) (CH / 4) + (i % CH) / 4) TM float4 from the block's first one;
        // eight loads in flight, then their 32 terms (the volatile adds keep the groups apart)
#pragma unroll
        for (int g8 = 0; g8 < TN / 32; ++g8) {
          float4 xv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int i = g8 * 32 + e * 4;
            const float4* ptr = qx + size_t((i / CH) * (CH / 4) + (i % CH) / 4) * TM;
            asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(xv[e].x), "=f"(xv[e].y), "=f"(xv[e].z), "=f"(xv[e].w)
                         : "l"(ptr));
          }
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float xs[4] = {xv[e].x, xv[e].y, xv[e].z, xv[e].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float a = rs[g8 * 32 + e * 4 + t], b = xs[t];
              const float pr = __fmul_rn(a, b);
              const float er = __fmaf_rn(a, b, -pr);
              float sn;
              asm volatile("add.rn.f32 %0, %1, %2;" : "=f"(sn) : "f"(qs), "f"(pr));
              const float bp = __fsub_rn(sn, qs);
              const float ds = __fadd_rn(__fsub_rn(qs, __fsub_rn(sn, bp)), __fsub_rn(pr, bp));
              qc = __fadd_rn(qc, __fadd_rn(ds, er));
              qs = sn;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < TN; ++i) rs[i] = 0.0f;
      } else {
#pragma unroll
        for (int i = 0; i < TN; ++i) {
          double d;
          asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(rs[i]));
          atomicAdd(acc + size_t(i) * TM, d);
          rs[i] = 0.0f;
        }
      }
    };
    for (int64_t item = blockIdx.x; item < nitems && !stop; item += gridDim.x) {
      int q, j, bi, bj, kind;
      decode_item<QF>(L, item, q, j, bi, bj, kind);
      int64_t nr_all;
      const int64_t nr = item_rounds<QF, CH>(L, q, bj, nr_all);
      const int nb = L.nb[q];
      if (QF) {
        qs = 0.0f;
        qc = 0.0f;
        qx = reinterpret_cast<const float4*>(L.xT[q] + size_t(bi) * size_t(L.kpad[q] / CH) * CH * TM) +
             size_t(bj) * (TN / 4) * TM + r;
      } else {
#pragma unroll 8
        for (int i = 0; i < TN; ++i) acc[size_t(i) * TM] = 0.0;
      }
#pragma unroll
      for (int i = 0; i < TN; ++i) rs[i] = 0.0f;
      bool sum_empty = true;
      // drain periods in completion order: the accumulators alternate, starting with the one
      // of the item's first round (its own-round count, and so its period count, is the larger)
      const int buf0 = int(g0 & 1);
      const int64_t np0 = ((nr + 1) / 2 + PL - 1) / PL, np1 = (nr / 2 + PL - 1) / PL;
      for (int64_t k = 0; k < np0 + np1; ++k, ++gp) {
        const int buf = (k & 1) ? buf0 ^ 1 : buf0;
        const uint32_t kbb = buf ? kb1 : kb0;
        const uint64_t t0 = hp_now();
        if (!warp_wait(&accf_bar[buf], kbb & 1, &s_abort, status)) {
          stop = true;
          break;
        }
        const uint64_t t1 = hp_now();
        hp_wc += t1 - t0;
        if (buf) ++kb1; else ++kb0;
        tc::tc_fence_after();
        const uint32_t src = lane_base + ACC_COL + buf * TN;
#pragma unroll
        for (int hb = 0; hb < TN / 64; ++hb) {      // two loads in flight, then the sums
          uint32_t va[32], vb[32];
          tc::tmem_ld32_nowait(src + hb * 64, va);
          tc::tmem_ld32_nowait(src + hb * 64 + 32, vb);
          tc::tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            rs[hb * 64 + i] += __uint_as_float(va[i]);
            rs[hb * 64 + 32 + i] += __uint_as_float(vb[i]);
          }
        }
        sum_empty = false;
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce_bar[buf]);
        const uint64_t t2 = hp_now();
        hp_dr += t2 - t1;
        ++hp_n;
        if (int((gp + qd * (FLUSH / 4)) % FLUSH) == FLUSH - 1) {
          fold();
          sum_empty = true;
          hp_fo += hp_now() - t2;
        }
      }
      if (stop) break;
      g0 += uint64_t(nr);
      if (!sum_empty) fold();
      if (QF) {
        // c_p += sum_c x_pc (x U)_pc over this tile's columns c (U: the upper triangle of the
        // form, so that x U x^T is the whole form)
        const int64_t p = int64_t(bi) * TM + r;
        if (p < L.nrow[q]) atomicAdd(L.cq[q] + size_t(j) * L.nrow[q] + p, double(qs) + double(qc));
        continue;
      }
      __threadfence();
      if (MODE == 2) {
        // real projections: P_IJ = -G_IJ (real symmetric)
        const int I = bi * TM + r;
        double2* P = L.P[q] + size_t(j) * nb * nb;
#pragma unroll 4
        for (int i = 0; i < TN; ++i) {
          const int J = bj * TN + i;
          if (I < nb && J < nb && I <= J) {
            double g = -acc[size_t(i) * TM];
            if (L.accumulate) g += P[size_t(I) * nb + J].x;     // written by this thread only
            P[size_t(I) * nb + J] = make_double2(g, 0.0);
            if (I != J) P[size_t(J) * nb + I] = make_double2(g, 0.0);
          }
        }
      } else if (kind != 0) {
        // three-product layout: the tile of C or S, transposed ([col][row], rows coalesced),
        // into the q's scratch; k_prod3_combine forms P after the launch
        const size_t nbp = size_t(L.nbj[q]) * TM;
        const int a = (kind == 2 ? bi - L.nbj[q] : bi) * TM + r;
        const int b0 = (kind == 2 ? bj - L.nbj[q] : bj) * TN;
        double* gt = L.g3[q] + (size_t(j) * 2 + (kind == 2 ? 1 : 0)) * nbp * nbp + size_t(b0) * nbp + a;
#pragma unroll 8
        for (int i = 0; i < TN; ++i) gt[size_t(i) * nbp] = acc[size_t(i) * TM];
      } else {
        // complex combination of rows (2I, 2I+1) held by lanes (2l, 2l+1)
        const int R = bi * TM + r;
        const int I = R >> 1;
        const bool odd = R & 1;
        double2* P = L.P[q] + size_t(j) * nb * nb;
#pragma unroll 4
        for (int jj = 0; jj < TN / 2; ++jj) {
          double e0 = acc[size_t(2 * jj) * TM];
          double e1 = acc[size_t(2 * jj + 1) * TM];
          double o0 = __shfl_xor_sync(0xffffffffu, e0, 1);
          double o1 = __shfl_xor_sync(0xffffffffu, e1, 1);
          if (!odd) {
            const int J = (bj * TN) / 2 + jj;
            if (I < nb && J < nb && I <= J) {
              double re = -(e0 + o1);
              double im = (I == J) ? 0.0 : -(o0 - e1);
              if (L.accumulate) {               // written by this thread only
                const double2 old = P[size_t(I) * nb + J];
                re += old.x;
                if (I != J) im += old.y;
              }
              P[size_t(I) * nb + J] = make_double2(re, im);
              if (I != J) P[size_t(J) * nb + I] = make_double2(re, -im);
            }
          }
        }
      }
    }
    if (kWaitProfile && lane == 0) {
      hp_flush(HP_EPI_TOTAL, hp_now() - hp0);
      hp_flush(HP_EPI_WAIT_ACC, hp_wc);
      hp_flush(HP_EPI_DRAIN, hp_dr);
      hp_flush(HP_EPI_FOLD, hp_fo);
      hp_flush(HP_EPI_PERIODS, hp_n);
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Per q, once: the chunk-major copy xT (A side: for each 128-column block and chunk, CH/4
// float4 groups of 128 consecutive columns, so a warp's reads of one group are contiguous)
// and the pre-split, pre-swizzled B tiles (frequency independent). One CTA per (128-column
// block, chunk); the chunk of x is staged through shared memory with coalesced float4 loads.
template <bool BF16>
__global__ void __launch_bounds__(128) k_prep_tc(const float* __restrict__ x, int64_t K, int ncol,
                                                 int64_t kpad, int64_t nch, float* __restrict__ xT,
                                                 char* __restrict__ bsp) {
  constexpr int CH = BF16 ? 32 : 16;
  constexpr int EPC = CH / 4;
  __shared__ __align__(16) float tile[CH][TM + 4];
  const int cb = blockIdx.y;               // column block (grid.y <= 65535)
  const int64_t c = blockIdx.x;             // chunk (grid.x: up to 2^31 - 1)
  const int tid = threadIdx.x;
  // pairs of columns: one 8-byte load when the row length ncol is even (the FP32 view of
  // complex projections: 2 N_b floats per row), two 4-byte loads when it is odd (real
  // projections with odd N_b, rows only 4-byte aligned)
  for (int idx = tid; idx < CH * (TM / 2); idx += 128) {
    const int t = idx / (TM / 2), c2 = idx % (TM / 2);
    const int64_t row = c * CH + t;
    const int col = cb * TM + 2 * c2;
    float2 v = make_float2(0.f, 0.f);
    if (row < K && col < ncol) {
      if ((ncol & 1) == 0) {
        v = __ldg(reinterpret_cast<const float2*>(x + row * ncol + col));
      } else {
        v.x = __ldg(x + row * ncol + col);
        if (col + 1 < ncol) v.y = __ldg(x + row * ncol + col + 1);
      }
    }
    *reinterpret_cast<float2*>(&tile[t][2 * c2]) = v;
  }
  __syncthreads();
  const int n = tid;
  float v[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t) v[t] = tile[t][n];
  float4* dst = reinterpret_cast<float4*>(xT) + (size_t(cb) * (kpad / CH) + c) * (CH / 4) * TM + n;
#pragma unroll
  for (int t = 0; t < CH / 4; ++t)
    dst[size_t(t) * TM] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
  char* hi = bsp + (size_t(cb) * nch + c) * CHUNK_BYTES;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    uint32_t hw[4], lw[4];
    split_words<BF16>(v + kc * EPC, hw, lw, 4);
    const uint32_t off = sw64_off(n, kc);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(hi + B_TILE + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// The same per-q preparation for the complex polarization in three real products. With
// M = Mr + i Mi and s_tj = |w_tj|, P_IJ = -sum_t s_tj conj(M_tI) M_tJ splits as
//   P_IJ = -S_IJ + (1 + i) C_IJ + (1 - i) C_JI,
//   C = Mr^T diag(s) Mi,   S = (Mr + Mi)^T diag(s) (Mr + Mi)
// (the real part -(Mr^T D Mr + Mi^T D Mi) = -S + C + C^T, the imaginary part C - C^T): S is
// symmetric, so the HERK computes its upper tiles and all tiles of C, N_b^2 (3/2) instead of
// (2 N_b)^2 / 2 tile elements, 3/4 of the multiply-adds of the real Gram matrix of the
// interleaved projections. A side (scaled later by the weights): column blocks [0, nbb) hold
// Mr, [nbb, 2 nbb) Mr + Mi; B side: [0, nbb) Mi, [nbb, 2 nbb) Mr + Mi (nbb = ceil(N_b / 128),
// zero padded). One CTA per (128 basis functions, chunk).
template <bool BF16>
__global__ void __launch_bounds__(128) k_prep_tc3(const float* __restrict__ x, int64_t K, int nb,
                                                  int nbb, int64_t kpad, int64_t nch,
                                                  float* __restrict__ xT, char* __restrict__ bsp) {
  constexpr int CH = BF16 ? 32 : 16;
  constexpr int EPC = CH / 4;
  __shared__ __align__(16) float tile[CH][2 * TM + 4];
  const int cb = blockIdx.y;
  const int64_t c = blockIdx.x;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < CH * TM; idx += 128) {     // (re, im) of 128 basis functions
    const int t = idx / TM, n2 = idx % TM;
    const int64_t row = c * CH + t;
    const int a = cb * TM + n2;
    float2 v = make_float2(0.f, 0.f);
    if (row < K && a < nb) v = __ldg(reinterpret_cast<const float2*>(x + row * (2 * int64_t(nb)) + 2 * a));
    *reinterpret_cast<float2*>(&tile[t][2 * n2]) = v;
  }
  __syncthreads();
  const int n = tid;
  float vr[CH], vi[CH], vs[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    const float2 v = *reinterpret_cast<const float2*>(&tile[t][2 * n]);
    vr[t] = v.x;
    vi[t] = v.y;
    vs[t] = v.x + v.y;
  }
  const int blk[2] = {cb, nbb + cb};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float* va = h ? vs : vr;                 // A side: Mr, Mr + Mi
    const float* vb = h ? vs : vi;                 // B side: Mi, Mr + Mi
    float4* dst = reinterpret_cast<float4*>(xT) + (size_t(blk[h]) * (kpad / CH) + c) * (CH / 4) * TM + n;
#pragma unroll
    for (int t = 0; t < CH / 4; ++t)
      dst[size_t(t) * TM] = make_float4(va[4 * t], va[4 * t + 1], va[4 * t + 2], va[4 * t + 3]);
    char* hi = bsp + (size_t(blk[h]) * nch + c) * CHUNK_BYTES;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t hw[4], lw[4];
      split_words<BF16>(vb + kc * EPC, hw, lw, 4);
      const uint32_t off = sw64_off(n, kc);
      *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(hi + B_TILE + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
}

// P (or P += with accumulate) from the three-product tiles: P_ab = -S_ab + C_ab + C_ba
// + i (C_ab - C_ba) for every a, b (Hermitian, since S is symmetric); the tiles are stored
// transposed (G[a][b] at [b][a]) with nbp rows and columns, S only in its upper tiles.
__global__ void k_prod3_combine(double2* __restrict__ P, const double* __restrict__ g3, int nb,
                                int nbp, int nw, int accumulate) {
  const int64_t n2 = int64_t(nb) * nb;
  const int64_t total = n2 * nw;
  const size_t p2 = size_t(nbp) * nbp;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = e / n2, rem = e % n2;
    const int a = int(rem / nb), b = int(rem % nb);
    const double* C = g3 + size_t(j) * 2 * p2;
    const double* S = C + p2;
    const double cab = C[size_t(b) * nbp + a], cba = C[size_t(a) * nbp + b];
    // S_ab from its upper element (row <= column), and (C_ab + C_ba) summed in an order-free
    // way, so that P_ba is exactly conj(P_ab)
    const double sab = (a <= b) ? S[size_t(b) * nbp + a] : S[size_t(a) * nbp + b];
    double re = (cab + cba) - sab, im = cab - cba;
    if (accumulate) {
      const double2 old = P[e];
      re += old.x;
      im += old.y;
    }
    P[e] = make_double2(re, im);
  }
}

// Quadratic form c_p = x_p^T R x_p (pair coefficients of the self-energy): the A operand is
// the real view X of the pair projections, row-padded to 128 and column-padded to kpad, in
// the chunk-major layout of the polarization's A side (rows = pairs, K = basis columns).
template <int CH>
__global__ void k_prep_xpad(const float* __restrict__ x, int64_t nrow, int ncol, int64_t nrowp,
                            int64_t kpad, float* __restrict__ xp) {
  const int64_t n4 = nrowp * (kpad / 4);
  const int64_t nchp = kpad / CH;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n4;
       e += int64_t(gridDim.x) * blockDim.x) {
    // destination order: [row block][chunk][group of 4 columns][row in block]
    const int64_t r = e % TM;
    const int64_t g = (e / TM) % (CH / 4);
    const int64_t ch = (e / (TM * (CH / 4))) % nchp;
    const int64_t blk = e / (TM * (CH / 4) * nchp);
    const int64_t row = blk * TM + r;
    const int64_t c = ch * CH + g * 4;
    // two float2 loads when ncol is even (complex projections: 8-byte aligned for any N_b),
    // four scalar loads when it is odd (real projections of an odd basis size)
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < nrow && c < ncol) {
      const float* src = x + row * ncol + c;
      if ((ncol & 1) == 0) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(src));
        v.x = a.x;
        v.y = a.y;
        if (c + 2 < ncol) {
          const float2 b = __ldg(reinterpret_cast<const float2*>(src + 2));
          v.z = b.x;
          v.w = b.y;
        }
      } else {
        v.x = __ldg(src);
        if (c + 1 < ncol) v.y = __ldg(src + 1);
        if (c + 2 < ncol) v.z = __ldg(src + 2);
        if (c + 3 < ncol) v.w = __ldg(src + 3);
      }
    }
    reinterpret_cast<float4*>(xp)[e] = v;
  }
}

// B operand of the quadratic form for one frequency: the upper triangle U of the real form R
// of W^c (R[2I+a][2J+b] = Re W_IJ for a = b, -Im W_IJ for (a,b) = (0,1), Im W_IJ for (1,0)), or
// of R = Re W^c for real projections (REAL): U_kk = R_kk, U_kc = R_kc + R_ck for k < c, 0 below
// the diagonal, so that x U x^T = x R x^T for every real row x (the form sees only the
// symmetric part of R) with about half the products. Split and swizzled like the
// polarization's B tiles, [c block][k chunk]; chunks below the diagonal block are zero.
template <bool BF16, bool REAL>
__global__ void __launch_bounds__(128) k_prep_quad(const double2* __restrict__ W0, int nb,
                                                   int64_t nch, char* __restrict__ bsp0,
                                                   int64_t jstride) {
  constexpr int CH = BF16 ? 32 : 16;
  constexpr int EPC = CH / 4;
  // frequency j = blockIdx.z: its W^c and its own B tiles
  const double2* __restrict__ W = W0 + size_t(blockIdx.z) * nb * nb;
  char* __restrict__ bsp = bsp0 + size_t(blockIdx.z) * size_t(jstride);
  const int cb = blockIdx.y;
  const int64_t ch = blockIdx.x;
  const int n = threadIdx.x;
  const int c = cb * TN + n;
  const int ncol = REAL ? nb : 2 * nb;
  const int J = REAL ? c : c >> 1, b = c & 1;
  char* hi = bsp + (size_t(cb) * nch + ch) * CHUNK_BYTES;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    float v[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      const int64_t k = ch * CH + kc * EPC + e;
      float r = 0.0f;
      if (c < ncol && k <= c) {
        if (REAL) {
          double u = W[size_t(k) * nb + J].x;
          if (k < c) u += W[size_t(J) * nb + k].x;
          r = float(u);
        } else {
          const int I = int(k >> 1), a = int(k & 1);
          const double2 w = W[size_t(I) * nb + J];
          double u = a == b ? w.x : (a == 0 ? -w.y : w.y);
          if (k < c) {                                  // R_ck = R[2J+b][2I+a]
            const double2 wt = W[size_t(J) * nb + I];
            u += a == b ? wt.x : (b == 0 ? -wt.y : wt.y);
          }
          r = float(u);
        }
      }
      v[e] = r;
    }
    uint32_t hw[4], lw[4];
    split_words<BF16>(v, hw, lw, 4);
    const uint32_t off = sw64_off(n, kc);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(hi + B_TILE + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// s_tj = -w_tj = prefactor f_t 2 Delta_t / (Delta_t^2 + omega_j^2), stored in FP32; with the
// extrapolar correction the same transition at Delta_bar_t is subtracted (s may then change sign)
__global__ void k_abs_weights_f32(int64_t K, int64_t kpad, const double* __restrict__ delta,
                                  const double* __restrict__ dbar, const double* __restrict__ f,
                                  double pref, int nw, OmegaArr om, float* __restrict__ s,
                                  unsigned* status) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (; t < kpad; t += stride) {
    if (t >= K) {
      for (int j = 0; j < nw; ++j) s[size_t(j) * kpad + t] = 0.0f;
      continue;
    }
    double d = delta[t];
    if (!(d > 0.0)) raise_status(status, ST_EINVAL);
    const double ft = 2.0 * pref * (f ? f[t] : 1.0);
    if (dbar == nullptr) {
      for (int j = 0; j < nw; ++j) s[size_t(j) * kpad + t] = float(ft * d / (d * d + om.v[j] * om.v[j]));
    } else {
      const double db = dbar[t];
      if (!(db > 0.0)) raise_status(status, ST_EINVAL);
      for (int j = 0; j < nw; ++j) {
        const double w2 = om.v[j] * om.v[j];
        s[size_t(j) * kpad + t] = float(ft * (d / (d * d + w2) - db / (db * db + w2)));
      }
    }
  }
}

// ncol: columns of the real operand x (2 N_b for complex projections, N_b for real ones)
int tile_count(int ncol, int* nbi_out) {
  int nbi = (ncol + TM - 1) / TM;     // TM == TN: square tiles, upper triangle
  if (nbi_out) *nbi_out = nbi;
  return nbi * (nbi + 1) / 2;
}

// Tiles of the complex polarization of one q: the three-product layout (C and the upper half
// of S over nbb = ceil(N_b / 128) blocks) where it has fewer tiles than the upper half of the
// real Gram matrix of the interleaved projections (N_b = 600: 40 against 55; N_b <= 64 and a
// few sizes such as 150 keep the interleaved layout). nbi: data blocks of each side.
struct CplxLayout {
  bool prod3;
  int nbb;
  int nbi;
  int ntile;
};
CplxLayout cplx_layout(int nb) {
  int nbi4;
  const int t4 = tile_count(2 * nb, &nbi4);
  const int nbb = (nb + TM - 1) / TM;
  const int t3 = nbb * nbb + nbb * (nbb + 1) / 2;
  if (t3 < t4) return CplxLayout{true, nbb, 2 * nbb, t3};
  return CplxLayout{false, nbb, nbi4, t4};
}

}  // namespace

static int64_t chunk_rows(int precision) { return precision == GW_BF16X3 ? 32 : 16; }

static void q_sizes(int64_t K, int precision, int64_t* nch, int64_t* kpad) {
  const int64_t ch = chunk_rows(precision);
  *nch = ((K + ch - 1) / ch + SUB - 1) / SUB * SUB;   // whole rounds (padding chunks are zero)
  *kpad = *nch * ch;
}

// q points are processed in groups: preparation of the group's q, then one HERK launch over
// them. A group closes once it holds GROUP_ITEMS_PER_SM work items per SM (or TQ q points), so
// large q run one at a time (measured faster than one launch over many large q) and small q
// share a launch; the workspace holds one group at a time. The grouping uses the complex tile
// count for real and complex projections alike, so the workspace query and the call agree.

// the tiles of C and S of the three-product layout, [nw][2][nbp][nbp] doubles
static size_t g3_bytes(const CplxLayout& lay, int nw) {
  const size_t nbp = size_t(lay.nbb) * TM;
  return lay.prod3 ? ws_round(size_t(nw) * 2 * nbp * nbp * sizeof(double)) : 0;
}

// nbi: data blocks of each side (the complex layout's, which is at least the real one's)
static size_t q_bytes(int64_t K, int nbi, int nw, int precision) {
  int64_t nch, kpad;
  q_sizes(K, precision, &nch, &kpad);
  return ws_round(size_t(nw) * size_t(kpad) * sizeof(float))          // weights
         + ws_round(size_t(nbi) * TM * size_t(kpad) * sizeof(float))  // chunk-major copy
         + ws_round(size_t(nbi) * size_t(nch) * CHUNK_BYTES);         // pre-split B tiles
}

// first q of every group, and the end (nq)
static void tc_groups(int nq, const int64_t* K, const int* nb, int nw, int sm,
                      int64_t items_per_sm, std::vector<int>& start) {
  start.clear();
  int64_t items = 0;
  int n = 0;
  for (int q = 0; q < nq; ++q) {
    if (n == 0 || items >= items_per_sm * sm || n == TQ) {
      start.push_back(q);
      items = 0;
      n = 0;
    }
    items += K[q] > 0 ? int64_t(cplx_layout(nb[q]).ntile) * nw : 0;
    ++n;
  }
  start.push_back(nq);
}

// the workspace of the largest group (the order of pol_tc's slices: per q the weights, the
// chunk-major copy, the pre-split tiles and the three-product tiles)
static size_t group_max_bytes(const std::vector<int>& start, const int64_t* K, const int* nb,
                              int nw, int precision) {
  size_t group_max = 0;
  for (size_t g = 0; g + 1 < start.size(); ++g) {
    size_t b = 0;
    for (int q = start[g]; q < start[g + 1]; ++q) {
      const CplxLayout lay = cplx_layout(nb[q]);
      b += q_bytes(K[q], lay.nbi, nw, precision) + (K[q] > 0 ? g3_bytes(lay, nw) : 0);
    }
    group_max = std::max(group_max, b);
  }
  return group_max;
}

// the preparation of the next group overlaps the HERK of the current one (two slots)
static bool overlapped(const std::vector<int>& start, const PolOpts& o) {
  return start.size() > 2 && !o.serial_prep;
}

size_t pol_tc_workspace(int nq, const int64_t* K, const int* nb, int nw, int precision,
                        const PolOpts& o) {
  int sm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  std::vector<int> start;
  tc_groups(nq, K, nb, nw, sm, o.group_items_per_sm, start);
  const size_t group_max = group_max_bytes(start, K, nb, nw, precision);
  return ws_round(size_t(sm) * TN * TM * sizeof(double)) + (overlapped(start, o) ? 2 : 1) * group_max;
}

// Streams of the overlapped preparation. A q of the mesh workload is one group of 640 work
// items, 4.2 waves on 152 SMs: during the HERK's last, partial wave most SMs are idle. With
// more than one group, the weights and operand copies of group g + 1 (bound by HBM) therefore
// run on a low-priority stream while the HERK of group g runs on a high-priority one; the
// priorities make the HERK's CTAs (one per SM, each holding the whole register file) take the
// SMs first whenever both are ready, and the copies fill the SMs the HERK has left. Two
// workspace slots alternate between groups; the preparation of group g waits for the HERK of
// group g - 2, the last reader of its slot. The call's stream is forked to the two streams at
// entry and joined again at exit, so the call keeps the ordering of one stream.
struct PolStreams {
  cudaStream_t herk = nullptr, prep = nullptr;
  cudaEvent_t entry = nullptr, exit_h = nullptr, exit_p = nullptr;
  cudaEvent_t prep_done[2] = {nullptr, nullptr}, herk_done[2] = {nullptr, nullptr};
};
static std::mutex g_ps_mu;           // held while a call enqueues its work on the streams
static PolStreams g_ps[64];
static bool g_ps_ok[64];

static int pol_streams(int dev, PolStreams** out) {   // with g_ps_mu held
  if (dev < 0 || dev >= 64) return set_error(GW_EINVAL, "device id %d out of range", dev);
  if (!g_ps_ok[dev]) {
    PolStreams p;
    int least = 0, greatest = 0;
    GW_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GW_CUDA_TRY(cudaStreamCreateWithPriority(&p.herk, cudaStreamNonBlocking, greatest));
    GW_CUDA_TRY(cudaStreamCreateWithPriority(&p.prep, cudaStreamNonBlocking, least));
    cudaEvent_t* evs[] = {&p.entry,        &p.exit_h,       &p.exit_p,      &p.prep_done[0],
                          &p.prep_done[1], &p.herk_done[0], &p.herk_done[1]};
    for (cudaEvent_t* e : evs) GW_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    g_ps[dev] = p;
    g_ps_ok[dev] = true;
  }
  *out = &g_ps[dev];
  return GW_OK;
}

static size_t herk_smem(int nsb) { return size_t(nsb) * STAGE_BYTES + NWS * WSLOT_BYTES + 1024; }

template <bool BF16, int MODE, int NSB>
static int launch_tc_k(const TcLaunch& L, unsigned grid, double* acc64, cudaStream_t s,
                       const DeviceCtx& ctx) {
  const size_t smem = herk_smem(NSB);
  int rc = set_max_dyn_smem(reinterpret_cast<const void*>(k_herk_tc<BF16, MODE, NSB>), smem,
                            ctx.device);
  if (rc) return rc;
  k_herk_tc<BF16, MODE, NSB><<<grid, NTHREADS, smem, s>>>(L, acc64, ctx.status);
  GW_LAUNCH_CHECK("k_herk_tc");
  return GW_OK;
}

// the quadratic form always runs with 4 stages; the polarization with o.b_stages
template <int MODE>
static int launch_tc(const TcLaunch& L, bool bf, int nsb, unsigned grid, double* acc64,
                     cudaStream_t s, const DeviceCtx& ctx) {
  if constexpr (MODE != 1) {
    if (nsb == 6)
      return bf ? launch_tc_k<true, MODE, 6>(L, grid, acc64, s, ctx)
                : launch_tc_k<false, MODE, 6>(L, grid, acc64, s, ctx);
  }
  return bf ? launch_tc_k<true, MODE, 4>(L, grid, acc64, s, ctx)
            : launch_tc_k<false, MODE, 4>(L, grid, acc64, s, ctx);
}

// the groups of pol_tc: preparation on sp, HERK and combination on sh (the same stream unless
// ps is given: then slot g mod 2 of the workspace and the events of ps order the two)
static int pol_tc_groups(const std::vector<int>& start, const PolQ* qs, double pref, int nw,
                         const OmegaArr& om, int precision, bool real, WsCursor& cur,
                         size_t group_base, size_t group_max, double* acc64, PolStreams* ps,
                         cudaStream_t sp, cudaStream_t sh, const DeviceCtx& ctx, PolOpts& o) {
  const bool bf = precision == GW_BF16X3;
  const int cpb = real ? 1 : 2;          // real operand columns per basis function
  for (size_t g = 0; g + 1 < start.size(); ++g) {
    const int q0 = start[g], n = start[g + 1] - start[g];
    const int slot = ps ? int(g % 2) : 0;
    // one slot: the previous group's launch is ordered before this group's preparation
    cur.used = group_base + size_t(slot) * group_max;
    if (ps && g >= 2) GW_CUDA_TRY(cudaStreamWaitEvent(sp, ps->herk_done[slot], 0));
    TcLaunch L{};
    L.nq = n;
    L.nw = nw;
    L.accumulate = o.accumulate ? 1 : 0;
    int64_t item = 0;
    for (int i = 0; i < n; ++i) {
      const PolQ& Q = qs[q0 + i];
      int64_t nch, kpad;
      q_sizes(Q.K, precision, &nch, &kpad);
      const CplxLayout lay = cplx_layout(Q.nb);
      const bool p3 = !real && lay.prod3 && Q.K > 0;     // K = 0: the zero P of the plain tiles
      int nbi;
      const int ntile = real ? tile_count(Q.nb, &nbi)
                        : p3 ? (nbi = lay.nbi, lay.ntile) : tile_count(2 * Q.nb, &nbi);
      float* sw = static_cast<float*>(cur.take(size_t(nw) * size_t(kpad) * sizeof(float)));
      float* xT = static_cast<float*>(cur.take(size_t(nbi) * TM * size_t(kpad) * sizeof(float)));
      char* bsp = static_cast<char*>(cur.take(size_t(nbi) * size_t(nch) * CHUNK_BYTES));
      double* g3 = nullptr;
      if (p3) {
        g3 = static_cast<double*>(cur.take(g3_bytes(lay, nw)));
        if (!g3) return set_error(GW_EWORKSPACE, "internal: three-product tile buffers");
      }
      if (kpad > 0) {
        if (!sw || !xT || !bsp) return set_error(GW_EWORKSPACE, "internal: tensor-core buffers");
        // the q's inputs (projections, energies) are read only by its weights and copies
        if (o.input_events && o.input_events[q0 + i])
          GW_CUDA_TRY(cudaStreamWaitEvent(sp, static_cast<cudaEvent_t>(o.input_events[q0 + i]), 0));
        int64_t blocks = std::min<int64_t>((kpad + 255) / 256, int64_t(ctx.sm_count) * 8);
        k_abs_weights_f32<<<unsigned(blocks), 256, 0, sp>>>(Q.K, kpad, Q.delta, Q.dbar, Q.f, pref,
                                                           nw, om, sw, ctx.status);
        GW_LAUNCH_CHECK("k_abs_weights_f32");
        const dim3 pg(static_cast<unsigned>(nch), static_cast<unsigned>(nbi));
        if (nch > 2147483647LL) return set_error(GW_EINVAL, "too many transitions for one q");
        if (p3) {
          const dim3 pg3(static_cast<unsigned>(nch), static_cast<unsigned>(lay.nbb));
          if (bf)
            k_prep_tc3<true><<<pg3, 128, 0, sp>>>(static_cast<const float*>(Q.M), Q.K, Q.nb,
                                                 lay.nbb, kpad, nch, xT, bsp);
          else
            k_prep_tc3<false><<<pg3, 128, 0, sp>>>(static_cast<const float*>(Q.M), Q.K, Q.nb,
                                                  lay.nbb, kpad, nch, xT, bsp);
          GW_LAUNCH_CHECK("k_prep_tc3");
        } else {
          if (bf)
            k_prep_tc<true><<<pg, 128, 0, sp>>>(static_cast<const float*>(Q.M), Q.K, cpb * Q.nb,
                                               kpad, nch, xT, bsp);
          else
            k_prep_tc<false><<<pg, 128, 0, sp>>>(static_cast<const float*>(Q.M), Q.K, cpb * Q.nb,
                                                kpad, nch, xT, bsp);
          GW_LAUNCH_CHECK("k_prep_tc");
        }
      }
      L.xT[i] = xT;
      L.bsp[i] = bsp;
      L.s[i] = sw;
      L.P[i] = reinterpret_cast<double2*>(Q.P);
      L.K[i] = Q.K;
      L.kpad[i] = kpad;
      L.nb[i] = Q.nb;
      L.ntile[i] = ntile;
      L.nbi[i] = nbi;
      L.nbj[i] = p3 ? lay.nbb : nbi;
      L.prod3[i] = p3 ? 1 : 0;
      L.g3[i] = g3;
      L.item0[i] = item;
      item += int64_t(L.ntile[i]) * nw;
    }
    L.item0[n] = item;
    if (ps) {                            // the HERK of this group after its preparation
      GW_CUDA_TRY(cudaEventRecord(ps->prep_done[slot], sp));
      GW_CUDA_TRY(cudaStreamWaitEvent(sh, ps->prep_done[slot], 0));
    }
    if (item > 0) {
      unsigned grid = unsigned(std::min<int64_t>(item, ctx.sm_count));
      int rc = record_herk_event(o, o.launches, false, sh);
      if (rc) return rc;
      rc = real ? launch_tc<2>(L, bf, o.b_stages, grid, acc64, sh, ctx)
                : launch_tc<0>(L, bf, o.b_stages, grid, acc64, sh, ctx);
      if (rc) return rc;
      if ((rc = record_herk_event(o, o.launches, true, sh))) return rc;
      ++o.launches;
    }
    for (int i = 0; i < n; ++i) {
      const int64_t tot = int64_t(nw) * L.nb[i] * L.nb[i];
      if (!L.prod3[i] || tot == 0) continue;
      const unsigned blocks = unsigned(std::min<int64_t>((tot + 255) / 256, int64_t(ctx.sm_count) * 8));
      k_prod3_combine<<<blocks, 256, 0, sh>>>(L.P[i], L.g3[i], L.nb[i], L.nbj[i] * TM, nw,
                                             L.accumulate);
      GW_LAUNCH_CHECK("k_prod3_combine");
    }
    if (ps) GW_CUDA_TRY(cudaEventRecord(ps->herk_done[slot], sh));   // the slot is free again
  }
  return GW_OK;
}


int pol_tc(int nq, const PolQ* qs, double pref, int nw, const OmegaArr& om, int precision,
           bool real, void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx,
           PolOpts& o) {
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  double* acc64 = static_cast<double*>(cur.take(size_t(ctx.sm_count) * TN * TM * sizeof(double)));
  if (!acc64) return set_error(GW_EWORKSPACE, "internal: tensor-core workspace too small");
  const size_t group_base = cur.used;
  std::vector<int64_t> Ks(nq);
  std::vector<int> nbs(nq);
  for (int q = 0; q < nq; ++q) {
    Ks[q] = qs[q].K;
    nbs[q] = qs[q].nb;
  }
  std::vector<int> start;
  tc_groups(nq, Ks.data(), nbs.data(), nw, ctx.sm_count, o.group_items_per_sm, start);
  const size_t group_max = group_max_bytes(start, Ks.data(), nbs.data(), nw, precision);
  cudaStream_t sp = s, sh = s;         // preparation and HERK streams
  std::unique_lock<std::mutex> lk(g_ps_mu);
  PolStreams* ps = nullptr;
  // The streams and events are created by the first call that runs outside a stream capture
  // (single group or not); a call captured before that runs on the caller's stream alone.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  GW_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  const bool known = ctx.device >= 0 && ctx.device < 64 && g_ps_ok[ctx.device];
  if (known || cs == cudaStreamCaptureStatusNone) {
    int rc = pol_streams(ctx.device, &ps);
    if (rc) return rc;
  }
  const bool ovl = overlapped(start, o) && ps != nullptr;
  if (ovl) {
    GW_CUDA_TRY(cudaEventRecord(ps->entry, s));
    GW_CUDA_TRY(cudaStreamWaitEvent(ps->herk, ps->entry, 0));
    GW_CUDA_TRY(cudaStreamWaitEvent(ps->prep, ps->entry, 0));
    sp = ps->prep;
    sh = ps->herk;
  }
  int rc = pol_tc_groups(start, qs, pref, nw, om, precision, real, cur, group_base, group_max,
                         acc64, ovl ? ps : nullptr, sp, sh, ctx, o);
  if (ovl) {                           // join both streams into the call's stream (errors too)
    cudaError_t e = cudaEventRecord(ps->exit_h, sh);
    if (e == cudaSuccess) e = cudaEventRecord(ps->exit_p, sp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ps->exit_h, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ps->exit_p, 0);
    if (e != cudaSuccess && rc == GW_OK) rc = cuda_error(e, "joining the polarization streams");
  }
  return rc;
}

// ------------------------------------------------------------ pair coefficients
// ncol: columns of the real pair operand x (2 N_b for complex projections, N_b for real ones)
static void quad_sizes(int64_t npair, int ncol, int precision, int64_t* nch, int64_t* kpad,
                       int64_t* nrowp, int* nbi, int* nbj) {
  const int64_t ch = chunk_rows(precision);
  *nch = ((int64_t(ncol) + ch - 1) / ch + SUB - 1) / SUB * SUB;   // whole rounds
  *nbj = (ncol + TN - 1) / TN;
  *kpad = int64_t(*nbj) * TN;                 // multiple of 128 (>= every chunk end)
  *nbi = int((npair + TM - 1) / TM);
  *nrowp = int64_t(*nbi) * TM;
}

size_t quad_tc_workspace(int nq, const int64_t* npair, const int* nb, int nw, int precision) {
  int sm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  size_t b = ws_round(size_t(sm) * TN * TM * sizeof(double));
  for (int q = 0; q < nq; ++q) {
    int64_t nch, kpad, nrowp;
    int nbi, nbj;
    quad_sizes(npair[q], 2 * nb[q], precision, &nch, &kpad, &nrowp, &nbi, &nbj);   // complex: a bound
    b += ws_round(size_t(nrowp) * size_t(kpad) * sizeof(float));
    b += ws_round(size_t(nw) * size_t(nbj) * size_t(nch) * CHUNK_BYTES);
  }
  return b;
}

int quad_tc(int nq, const int64_t* npair, const int* nb, const void* const* Msig, int nw,
            const double* const* Wc, double* const* c, int precision, bool real, void* ws,
            size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx) {
  const bool bf = precision == GW_BF16X3;
  const int cpb = real ? 1 : 2;          // real operand columns per basis function
  WsCursor cur{static_cast<char*>(ws), ws_bytes, 0};
  double* acc64 = static_cast<double*>(cur.take(size_t(ctx.sm_count) * TN * TM * sizeof(double)));
  if (!acc64) return set_error(GW_EWORKSPACE, "internal: tensor-core workspace too small");
  std::vector<float*> xp(nq);
  std::vector<char*> bsp(nq);
  std::vector<int64_t> kp(nq), nchv(nq);
  std::vector<int> nbiv(nq), nbjv(nq);
  for (int q = 0; q < nq; ++q) {
    int64_t nch, kpad, nrowp;
    int nbi, nbj;
    quad_sizes(npair[q], cpb * nb[q], precision, &nch, &kpad, &nrowp, &nbi, &nbj);
    kp[q] = kpad;
    nchv[q] = nch;
    nbiv[q] = nbi;
    nbjv[q] = nbj;
    xp[q] = static_cast<float*>(cur.take(size_t(nrowp) * size_t(kpad) * sizeof(float)));
    bsp[q] = static_cast<char*>(cur.take(size_t(nw) * size_t(nbj) * size_t(nch) * CHUNK_BYTES));
    if (npair[q] == 0) continue;
    if (!xp[q] || !bsp[q]) return set_error(GW_EWORKSPACE, "internal: tensor-core buffers");
    GW_CUDA_TRY(cudaMemsetAsync(c[q], 0, sizeof(double) * size_t(nw) * size_t(npair[q]), s));
    const int64_t n4 = nrowp * (kpad / 4);
    const unsigned xg = unsigned(std::min<int64_t>((n4 + 255) / 256, int64_t(ctx.sm_count) * 16));
    if (bf)
      k_prep_xpad<32><<<xg, 256, 0, s>>>(static_cast<const float*>(Msig[q]), npair[q],
                                         cpb * nb[q], nrowp, kpad, xp[q]);
    else
      k_prep_xpad<16><<<xg, 256, 0, s>>>(static_cast<const float*>(Msig[q]), npair[q],
                                         cpb * nb[q], nrowp, kpad, xp[q]);
    GW_LAUNCH_CHECK("k_prep_xpad");
    const dim3 pg(static_cast<unsigned>(nch), static_cast<unsigned>(nbj), static_cast<unsigned>(nw));
    const double2* W = reinterpret_cast<const double2*>(Wc[q]);
    const int64_t jstride = int64_t(nbj) * nch * CHUNK_BYTES;
    if (bf && real)
      k_prep_quad<true, true><<<pg, 128, 0, s>>>(W, nb[q], nch, bsp[q], jstride);
    else if (bf)
      k_prep_quad<true, false><<<pg, 128, 0, s>>>(W, nb[q], nch, bsp[q], jstride);
    else if (real)
      k_prep_quad<false, true><<<pg, 128, 0, s>>>(W, nb[q], nch, bsp[q], jstride);
    else
      k_prep_quad<false, false><<<pg, 128, 0, s>>>(W, nb[q], nch, bsp[q], jstride);
    GW_LAUNCH_CHECK("k_prep_quad");
  }
  for (int q0 = 0; q0 < nq; q0 += TQ) {
    int n = std::min(TQ, nq - q0);
    TcLaunch L{};
    L.nq = n;
    L.nw = nw;
    int64_t item = 0;
    for (int q = 0; q < n; ++q) {
      const int Q = q0 + q;
      L.xT[q] = xp[Q];
      L.bsp[q] = bsp[Q];
      L.s[q] = nullptr;
      L.cq[q] = c[Q];
      L.bsp_jstride[q] = int64_t(nbjv[Q]) * nchv[Q] * CHUNK_BYTES;
      L.nrow[q] = npair[Q];
      L.K[q] = npair[Q] > 0 ? int64_t(cpb) * nb[Q] : 0;
      L.kpad[q] = kp[Q];
      L.nb[q] = nb[Q];
      L.nbi[q] = nbiv[Q];
      L.nbj[q] = nbjv[Q];
      L.ntile[q] = npair[Q] > 0 ? nbiv[Q] * nbjv[Q] : 0;
      L.item0[q] = item;
      item += int64_t(L.ntile[q]) * nw;
    }
    L.item0[n] = item;
    if (item == 0) continue;
    unsigned grid = unsigned(std::min<int64_t>(item, ctx.sm_count));
    int rc = launch_tc<1>(L, bf, 4, grid, acc64, s, ctx);
    if (rc) return rc;
  }
  return GW_OK;
}

int herk_wait_profile(unsigned long long* counters, int n, int reset) {
  if (!kWaitProfile)
    return set_error(GW_EUNSUPPORTED, "the library was built without GW_HERK_WAIT_PROFILE");
  if (n < 0 || (n > 0 && !counters))
    return set_error(GW_EINVAL, "n=%d with counters=%p", n, static_cast<void*>(counters));
  GW_CUDA_TRY(cudaDeviceSynchronize());
  if (n > 0)
    GW_CUDA_TRY(cudaMemcpyFromSymbol(counters, g_herk_prof,
                                     sizeof(unsigned long long) * std::min(n, int(HP_N))));
  if (reset) {
    const unsigned long long zero[HP_N] = {};
    GW_CUDA_TRY(cudaMemcpyToSymbol(g_herk_prof, zero, sizeof(zero)));
  }
  return GW_OK;
}

}  // namespace gw
