// Diagnostic (no counterpart in the paper): the issue rate of the split-precision HERK's
// tcgen05.mma sequence under the conditions the HERK runs it in. One CTA per SM; lane 0 of
// warp 0 issues rounds of 12 MMAs of 128 x 128 x 16 BF16 (A from TMEM, B from a 4-stage
// 64-byte-swizzled shared-memory ring, 3 commits per round, accumulators alternating by
// round) on fixed random operands; other warps of the CTA load the SM sub-partitions
// (warp w runs on sub-partition w mod 4) with independent FMA chains. The result is the
// average number of SM cycles per MMA (64 is the tensor pipe's rate for this shape).
// Variants:
//   0  the issuer alone
//   1  the issuer with a branch on a shared-memory value before each round
//   2  three warps of FMA chains on the issuer's sub-partition
//   3  three warps of FMA chains on the other three sub-partitions
//   4  as 2, with MMAs of 128 x 256 x 16 (counted as two 128 x 128 x 16)
//   5  two issuers on two sub-partitions, rounds concurrent, three FMA warps beside each
// Every wait is bounded; the FMA warps stop when the issuers are done (or after a fixed count).
#include "gw_internal.cuh"
#include "tc_ptx.cuh"

namespace gw {

namespace {

constexpr int PR_THREADS = 512;
constexpr int PR_RING = 160 * 1024;     // B ring (4 x 32 KB) and the 256-row tiles of variant 4

__device__ __forceinline__ uint32_t pr_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
// two BF16 values in +-[1, 2)
__device__ __forceinline__ uint32_t pr_bf16x2(uint32_t h) {
  const uint32_t lo = 0x3F80u | (h & 0x7Fu) | (((h >> 7) & 1u) << 15);
  const uint32_t hi = 0x3F80u | ((h >> 8) & 0x7Fu) | (((h >> 15) & 1u) << 15);
  return lo | (hi << 16);
}

// one round as the HERK issues it: 2 chunks x 2 K steps x (lo*hi, hi*lo, hi*hi)
__device__ __forceinline__ void pr_round(uint32_t tmem, uint64_t desc0, uint32_t g, uint32_t d,
                                         uint32_t idesc) {
  const uint32_t st = g % 4, slot = g % 4;
  const uint32_t a0 = tmem + 256 + slot * 64;
  const uint64_t dst = desc0 + uint64_t((st * 32768u) >> 4);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint64_t dBh = dst + uint64_t((u * 16384 + ks * 32) >> 4);
      const uint64_t dBl = dst + uint64_t((u * 16384 + 8192 + ks * 32) >> 4);
      const uint32_t ah = a0 + u * 32 + ks * 8, al = ah + 16;
      tc::mma_f16_ta(d, al, dBh, idesc, (u == 0 && ks == 0) ? 0u : 1u);
      tc::mma_f16_ta(d, ah, dBl, idesc, 1u);
      tc::mma_f16_ta(d, ah, dBh, idesc, 1u);
    }
  }
}

template <int VAR>
__global__ void __launch_bounds__(PR_THREADS, 1)
    k_probe_mma(int rounds, unsigned long long* cycles, float* sink, unsigned* status) {
  extern __shared__ __align__(1024) char dsmem[];
  char* ring = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar[2], done_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_done;
  __shared__ volatile int s_zero;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < PR_RING / 4; i += PR_THREADS)
    reinterpret_cast<uint32_t*>(ring)[i] = pr_bf16x2(pr_hash(uint32_t(i) * 2654435761u + blockIdx.x));
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&bar[i], 1);        // per-round commits (nothing waits on them)
      tc::mbar_init(&done_bar[i], 1);   // one commit after an issuer's last round
    }
    tc::mbar_fence_init();
    s_done = 0;
    s_zero = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 512);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (warp < 4) {                 // random A operands in columns [256, 512) of every lane
    const uint32_t lb = tmem + (uint32_t(warp * 32) << 16);
    for (int c = 256; c < 512; c += 8) {
      uint32_t z[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) z[e] = pr_bf16x2(pr_hash(uint32_t(threadIdx.x * 512 + c + e) * 97u + 5u));
      tc::tmem_st8(lb + c, z);
    }
    tc::tmem_wait_st();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();

  constexpr bool TWO = VAR == 5;
  const uint32_t idesc = tc::instr_desc(1u, 128, VAR == 4 ? 256 : 128);
  const uint64_t desc0 = tc::smem_desc(tc::smem_u32(ring), 512, 4);
  const bool issuer = lane == 0 && (warp == 0 || (TWO && warp == 1));
  if (issuer) {
    const uint32_t p = uint32_t(warp);
    const uint64_t t0 = clock64();
    const int nr = TWO ? rounds / 2 : rounds;
    for (int g = 0; g < nr; ++g) {
      if (VAR == 1 && s_zero) break;                       // a branch on a shared value
      const uint32_t d = tmem + (VAR == 4 ? 0u : TWO ? p * 128u : uint32_t(g & 1) * 128u);
      pr_round(tmem, desc0, uint32_t(g), d, idesc);
      tc::mma_commit(&bar[p]);
      tc::mma_commit(&bar[p]);
      tc::mma_commit(&bar[p]);
    }
    // until every MMA of this thread has completed
    tc::mma_commit(&done_bar[p]);
    int never = 0;
    if (!tc::mbar_wait(&done_bar[p], 0, reinterpret_cast<volatile int*>(&never), 2000000000ull))
      raise_status(status, ST_ETIMEOUT);
    const uint64_t t1 = clock64();
    if (p == 0) {
      s_done = 1;
      atomicAdd(cycles, static_cast<unsigned long long>(t1 - t0));
    }
  } else {
    const int sp = warp & 3;
    const bool busy = (VAR == 2 || VAR == 4) ? (sp == 0 && warp >= 4)
                      : (VAR == 3)           ? (warp >= 1 && warp <= 3)
                      : (VAR == 5)           ? ((sp == 0 || sp == 1) && warp >= 4)
                                             : false;
    if (busy) {
      float x[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = float(threadIdx.x + e);
      for (int it = 0; it < 4000000 && !s_done; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
          for (int e = 0; e < 8; ++e) x[e] = fmaf(x[e], 0.999f, 0.5f);
        }
      }
      float t = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) t += x[e];
      if (t == 1234.5f) sink[0] = t;                     // keeps the chains live
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  __syncwarp();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int VAR>
int launch_probe(int rounds, unsigned long long* cycles, float* sink, cudaStream_t s,
                 const DeviceCtx& ctx) {
  const int smem = PR_RING + 1024;
  int rc = set_max_dyn_smem(reinterpret_cast<const void*>(&k_probe_mma<VAR>), smem, ctx.device);
  if (rc) return rc;
  k_probe_mma<VAR><<<ctx.sm_count, PR_THREADS, smem, s>>>(rounds, cycles, sink, ctx.status);
  GW_LAUNCH_CHECK("k_probe_mma");
  return GW_OK;
}

}  // namespace

int probe_mma_issue(int variant, int rounds, double* cycles_per_mma, cudaStream_t s,
                    const DeviceCtx& ctx) {
  unsigned long long* d_cyc = nullptr;
  float* d_sink = nullptr;
  GW_CUDA_TRY(cudaMallocAsync(&d_cyc, sizeof(unsigned long long), s));
  GW_CUDA_TRY(cudaMallocAsync(&d_sink, sizeof(float), s));
  GW_CUDA_TRY(cudaMemsetAsync(d_cyc, 0, sizeof(unsigned long long), s));
  int rc = GW_OK;
  switch (variant) {
    case 0: rc = launch_probe<0>(rounds, d_cyc, d_sink, s, ctx); break;
    case 1: rc = launch_probe<1>(rounds, d_cyc, d_sink, s, ctx); break;
    case 2: rc = launch_probe<2>(rounds, d_cyc, d_sink, s, ctx); break;
    case 3: rc = launch_probe<3>(rounds, d_cyc, d_sink, s, ctx); break;
    case 4: rc = launch_probe<4>(rounds, d_cyc, d_sink, s, ctx); break;
    default: rc = launch_probe<5>(rounds, d_cyc, d_sink, s, ctx); break;
  }
  unsigned long long h = 0;
  if (rc == GW_OK) {
    GW_CUDA_TRY(cudaMemcpyAsync(&h, d_cyc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GW_CUDA_TRY(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(d_cyc, s);
  cudaFreeAsync(d_sink, s);
  if (rc) return rc;
  // cycles of issuer 0 per CTA, over the MMAs issued in that time (both issuers' for
  // variant 5), in units of 128 x 128 x 16
  const double units = 12.0 * (variant == 5 ? 2 * (rounds / 2) : rounds) * (variant == 4 ? 2 : 1);
  *cycles_per_mma = double(h) / double(ctx.sm_count) / units;
  return GW_OK;
}

}  // namespace gw
