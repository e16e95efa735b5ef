// Synthetic projections on the device (input generation, not part of the method).
// Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, counter
// (element index low, element index high, q, tensor id); Box-Muller on the four
// output words gives one complex normal per element, scaled by 1/(1 + I/16).
#include "gw_internal.cuh"

namespace gw {

__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                             uint32_t& x3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, x0), lo0 = M0 * x0;
  uint32_t hi1 = __umulhi(M1, x2), lo1 = M1 * x2;
  uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
  x0 = y0;
  x1 = y1;
  x2 = y2;
  x3 = y3;
}

__device__ __forceinline__ void philox10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(x0, x1, x2, x3, k0, k1);
  }
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return (double(a >> 5) * 67108864.0 + double(b >> 6)) * (1.0 / 9007199254740992.0);
}

template <typename T>
__global__ void k_synth(uint64_t seed, uint32_t tid, uint32_t q, int64_t row0, int64_t rows,
                        int nb, T* __restrict__ out) {
  int64_t n = rows * nb;
  int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (; e < n; e += stride) {
    int64_t r = e / nb;
    int I = int(e - r * nb);
    uint64_t idx = uint64_t(row0 + r) * uint64_t(nb) + uint64_t(I);
    uint32_t x0 = uint32_t(idx), x1 = uint32_t(idx >> 32), x2 = q, x3 = tid;
    philox10(x0, x1, x2, x3, uint32_t(seed), uint32_t(seed >> 32));
    double u1 = 1.0 - u53(x0, x1);
    double u2 = u53(x2, x3);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 2.0 * 3.141592653589793 * u2;
    double sc = 1.0 + double(I) / 16.0;
    double re = rad * cos(ang) / sc, im = rad * sin(ang) / sc;
    out[2 * e] = T(re);
    out[2 * e + 1] = T(im);
  }
}

int synth_projections(uint64_t seed, uint32_t tid, uint32_t q, int64_t row0, int64_t rows, int nb,
                      int dtype, void* out, cudaStream_t s, const DeviceCtx& ctx) {
  int64_t n = rows * nb;
  if (n == 0) return GW_OK;
  int64_t blocks = (n + 255) / 256;
  int64_t cap = int64_t(ctx.sm_count) * 16;
  if (blocks > cap) blocks = cap;
  if (dtype == GW_C128)
    k_synth<double><<<unsigned(blocks), 256, 0, s>>>(seed, tid, q, row0, rows, nb,
                                                     static_cast<double*>(out));
  else
    k_synth<float><<<unsigned(blocks), 256, 0, s>>>(seed, tid, q, row0, rows, nb,
                                                    static_cast<float*>(out));
  GW_LAUNCH_CHECK("k_synth");
  return GW_OK;
}

}  // namespace gw
