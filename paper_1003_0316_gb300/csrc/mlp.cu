// a7: learned initialiser of the multipole fit (Eq. modelf, N_p = 2): a multilayer
// perceptron 48 -> 128 -> 128 -> 8 with SiLU activations proposes (a_p, w_p) from the
// curve Sigma(i w_j) on 24 nodes; the FP64 Levenberg-Marquardt fit then starts there.
//
// Input: x = (Re y_j / s, Im y_j / s) interleaved per node, s = max_j |y_j| (1 if 0).
// Output o (8 values): a_p = s (o_{4p} + i o_{4p+1}), w_p = o_{4p+2} + i o_{4p+3}.
// Packed parameters (FP32): W1[128][48], b1[128], W2[128][128], b2[128], W3[8][128], b3[8].
//
// Inference (k_mlp_forward, k_mlp_start): BF16 storage arithmetic: the input, every weight
// and bias and both hidden activations are rounded to BF16 (round to nearest even), the
// dot products accumulate in FP32, SiLU is evaluated in FP32.
// Training (k_mlp_train): FP32 forward, the fit loss of the proposed parameters
//   L = (1/B) sum_b (1/24) sum_j |f_b(i w_j) - y_bj|^2 / s_b^2,
// its gradient by back-propagation (accumulated over the batch with FP32 atomics), and
// an optional Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8).
//
// One CTA of 128 threads takes CPB curves; weights live in shared memory with padded
// row strides (49, 129) so that both row-wise and column-wise sweeps are free of bank
// conflicts; thread t owns hidden unit t for every curve of the CTA.
#include <cuda_bf16.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int NIN = MLP_NIN, NH = MLP_NH, NOUT = MLP_NOUT, NW = 24;
constexpr int S1 = NIN + 1;     // padded row stride of W1 in shared memory
constexpr int S2 = NH + 1;      // padded row stride of W2
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH;
static_assert(OFF_B3 + NOUT == MLP_NPARAM, "packed layout");
constexpr int CPB = 16;         // curves per CTA

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float sg = 1.0f / (1.0f + expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}

struct MlpSmem {
  float W1[NH * S1];
  float W2[NH * S2];
  float W3[NOUT * NH];
  float b1[NH], b2[NH], b3[NOUT];
  float x[CPB][NIN];
  float z1[CPB][NH], h1[CPB][NH];
  float z2[CPB][NH], h2[CPB][NH];
  float o[CPB][NOUT];
  double s[CPB];
};

// Weights into shared memory (rounded to BF16 when BF is set).
template <bool BF>
__device__ void load_weights(MlpSmem& S, const float* __restrict__ w) {
  for (int i = threadIdx.x; i < NH * NIN; i += blockDim.x) {
    const float v = w[OFF_W1 + i];
    S.W1[(i / NIN) * S1 + i % NIN] = BF ? bf16r(v) : v;
  }
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
    const float v = w[OFF_W2 + i];
    S.W2[(i / NH) * S2 + i % NH] = BF ? bf16r(v) : v;
  }
  for (int i = threadIdx.x; i < NOUT * NH; i += blockDim.x) {
    const float v = w[OFF_W3 + i];
    S.W3[i] = BF ? bf16r(v) : v;
  }
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    S.b1[i] = BF ? bf16r(w[OFF_B1 + i]) : w[OFF_B1 + i];
    S.b2[i] = BF ? bf16r(w[OFF_B2 + i]) : w[OFF_B2 + i];
  }
  if (threadIdx.x < NOUT) S.b3[threadIdx.x] = BF ? bf16r(w[OFF_B3 + threadIdx.x]) : w[OFF_B3 + threadIdx.x];
}

// Features of curves [c0, c0 + nc) into S.x and S.s (FP64 data, FP32 features).
template <bool BF>
__device__ void load_features(MlpSmem& S, const double2* __restrict__ sig, int c0, int nc) {
  if (threadIdx.x < CPB) {
    const int c = threadIdx.x;
    double m = 0.0;
    if (c < nc)
      for (int j = 0; j < NW; ++j) {
        const double2 y = sig[size_t(c0 + c) * NW + j];
        m = fmax(m, hypot(y.x, y.y));
      }
    S.s[c] = m > 0.0 ? m : 1.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CPB * NW; i += blockDim.x) {
    const int c = i / NW, j = i % NW;
    float re = 0.f, im = 0.f;
    if (c < nc) {
      const double2 y = sig[size_t(c0 + c) * NW + j];
      const double inv = 1.0 / S.s[c];
      re = float(y.x * inv);
      im = float(y.y * inv);
    }
    S.x[c][2 * j] = BF ? bf16r(re) : re;
    S.x[c][2 * j + 1] = BF ? bf16r(im) : im;
  }
  __syncthreads();
}

// Forward pass of the CTA's curves; outputs in S.o (keeps z and h for back-propagation).
template <bool BF>
__device__ void forward(MlpSmem& S) {
  const int t = threadIdx.x;     // hidden unit
  float acc[CPB];
#pragma unroll
  for (int c = 0; c < CPB; ++c) acc[c] = S.b1[t];
  for (int k = 0; k < NIN; ++k) {
    const float w = S.W1[t * S1 + k];
#pragma unroll
    for (int c = 0; c < CPB; ++c) acc[c] = fmaf(w, S.x[c][k], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < CPB; ++c) {
    S.z1[c][t] = acc[c];
    const float h = silu_f(acc[c]);
    S.h1[c][t] = BF ? bf16r(h) : h;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CPB; ++c) acc[c] = S.b2[t];
  for (int k = 0; k < NH; ++k) {
    const float w = S.W2[t * S2 + k];
#pragma unroll
    for (int c = 0; c < CPB; ++c) acc[c] = fmaf(w, S.h1[c][k], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < CPB; ++c) {
    S.z2[c][t] = acc[c];
    const float h = silu_f(acc[c]);
    S.h2[c][t] = BF ? bf16r(h) : h;
  }
  __syncthreads();
  {
    const int c = t / NOUT, o = t % NOUT;      // 128 threads = CPB x NOUT outputs
    float a = S.b3[o];
    for (int k = 0; k < NH; ++k) a = fmaf(S.W3[o * NH + k], S.h2[c][k], a);
    S.o[c][o] = a;
  }
  __syncthreads();
}
static_assert(CPB * NOUT == NH, "one output per thread in the last layer");

__global__ void __launch_bounds__(NH) k_mlp_forward(int n, const double2* __restrict__ sig,
                                                    const float* __restrict__ w,
                                                    float* __restrict__ out) {
  extern __shared__ __align__(16) char smraw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smraw);
  load_weights<true>(S, w);
  for (int c0 = blockIdx.x * CPB; c0 < n; c0 += gridDim.x * CPB) {
    const int nc = min(CPB, n - c0);
    load_features<true>(S, sig, c0, nc);
    forward<true>(S);
    const int c = threadIdx.x / NOUT, o = threadIdx.x % NOUT;
    if (c < nc) out[size_t(c0 + c) * NOUT + o] = S.o[c][o];
    __syncthreads();
  }
}

// Learned start of the fit: BF16 forward, decoded into theta = (Re a, Im a, Re w, Im w)_p.
__global__ void __launch_bounds__(NH) k_mlp_start(int n, const double2* __restrict__ sig,
                                                  const float* __restrict__ w,
                                                  double* __restrict__ theta) {
  extern __shared__ __align__(16) char smraw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smraw);
  load_weights<true>(S, w);
  for (int c0 = blockIdx.x * CPB; c0 < n; c0 += gridDim.x * CPB) {
    const int nc = min(CPB, n - c0);
    load_features<true>(S, sig, c0, nc);
    forward<true>(S);
    const int c = threadIdx.x / NOUT, o = threadIdx.x % NOUT;
    if (c < nc) {
      const double v = double(S.o[c][o]);
      theta[size_t(c0 + c) * NOUT + o] = (o % 4) < 2 ? v * S.s[c] : v;
    }
    __syncthreads();
  }
}

// One training pass over the batch: loss and gradient (accumulated into grad and loss with
// FP32 atomics; both must start at zero).
__global__ void __launch_bounds__(NH) k_mlp_train(int n, OmegaArr om, const double2* __restrict__ sig,
                                                  const float* __restrict__ w,
                                                  float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) char smraw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smraw);
  __shared__ float go[CPB][NOUT];
  __shared__ float gz2[CPB][NH];
  __shared__ float gz1[CPB][NH];
  const int t = threadIdx.x;
  load_weights<false>(S, w);
  const float invB = 1.0f / float(n);
  for (int c0 = blockIdx.x * CPB; c0 < n; c0 += gridDim.x * CPB) {
    const int nc = min(CPB, n - c0);
    load_features<false>(S, sig, c0, nc);
    forward<false>(S);
    // loss and dL/do per curve (FP32 complex arithmetic)
    if (t < CPB) {
      const int c = t;
      float g[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) g[o] = 0.f;
      if (c < nc) {
        const float s = float(S.s[c]);
        float ar[2], ai[2], wr[2], wi[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          ar[p] = s * S.o[c][4 * p];
          ai[p] = s * S.o[c][4 * p + 1];
          wr[p] = S.o[c][4 * p + 2];
          wi[p] = S.o[c][4 * p + 3];
        }
        const float coef = 2.0f * invB / (float(NW) * s * s);
        float L = 0.f;
        for (int j = 0; j < NW; ++j) {
          const double2 yj = sig[size_t(c0 + c) * NW + j];
          const float oj = float(om.v[j]);
          float fr = 0.f, fi = 0.f, pr[2], pi[2];
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            // phi = 1 / (i w_j - w_p)
            const float dr = -wr[p], di = oj - wi[p];
            const float den = dr * dr + di * di;
            pr[p] = dr / den;
            pi[p] = -di / den;
            fr += ar[p] * pr[p] - ai[p] * pi[p];
            fi += ar[p] * pi[p] + ai[p] * pr[p];
          }
          const float rr = fr - float(yj.x), ri = fi - float(yj.y);
          L += rr * rr + ri * ri;
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            // d f / d(Re of output a) = s phi;  d f / d(Re w_p) = a_p phi^2
            const float qr = pr[p] * pr[p] - pi[p] * pi[p], qi = 2.f * pr[p] * pi[p];
            const float dwr = ar[p] * qr - ai[p] * qi, dwi = ar[p] * qi + ai[p] * qr;
            // Re(conj(r) D) and Re(conj(r) i D)
            g[4 * p + 0] += coef * s * (rr * pr[p] + ri * pi[p]);
            g[4 * p + 1] += coef * s * (rr * -pi[p] + ri * pr[p]);
            g[4 * p + 2] += coef * (rr * dwr + ri * dwi);
            g[4 * p + 3] += coef * (rr * -dwi + ri * dwr);
          }
        }
        atomicAdd(loss, L * invB / (float(NW) * s * s));
      }
#pragma unroll
      for (int o = 0; o < NOUT; ++o) go[c][o] = g[o];
    }
    __syncthreads();
    // back-propagation: gz2 = (go W3) * silu'(z2), gz1 = (gz2 W2) * silu'(z1)
    for (int c = 0; c < CPB; ++c) {
      float a = 0.f;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) a = fmaf(go[c][o], S.W3[o * NH + t], a);
      gz2[c][t] = a * dsilu_f(S.z2[c][t]);
    }
    __syncthreads();
    {
      float acc[CPB];
#pragma unroll
      for (int c = 0; c < CPB; ++c) acc[c] = 0.f;
      for (int u = 0; u < NH; ++u) {
        const float wv = S.W2[u * S2 + t];
#pragma unroll
        for (int c = 0; c < CPB; ++c) acc[c] = fmaf(gz2[c][u], wv, acc[c]);
      }
#pragma unroll
      for (int c = 0; c < CPB; ++c) gz1[c][t] = acc[c] * dsilu_f(S.z1[c][t]);
    }
    __syncthreads();
    // parameter gradients of this CTA's curves, added into the batch gradient
    for (int k = 0; k < NIN; ++k) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < CPB; ++c) a = fmaf(gz1[c][t], S.x[c][k], a);
      atomicAdd(grad + OFF_W1 + t * NIN + k, a);
    }
    for (int k = 0; k < NH; ++k) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < CPB; ++c) a = fmaf(gz2[c][t], S.h1[c][k], a);
      atomicAdd(grad + OFF_W2 + t * NH + k, a);
    }
    {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int c = 0; c < CPB; ++c) {
        a1 += gz1[c][t];
        a2 += gz2[c][t];
      }
      atomicAdd(grad + OFF_B1 + t, a1);
      atomicAdd(grad + OFF_B2 + t, a2);
    }
    for (int o = 0; o < NOUT; ++o) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < CPB; ++c) a = fmaf(go[c][o], S.h2[c][t], a);
      atomicAdd(grad + OFF_W3 + o * NH + t, a);
    }
    if (t < NOUT) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < CPB; ++c) a += go[c][t];
      atomicAdd(grad + OFF_B3 + t, a);
    }
    __syncthreads();
  }
}

__global__ void k_adam(int np, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float bc1, float bc2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

constexpr size_t SMEM_FWD = sizeof(MlpSmem);

int grid_for(int n, const DeviceCtx& ctx) {
  const int blocks = (n + CPB - 1) / CPB;
  return blocks < ctx.sm_count * 4 ? blocks : ctx.sm_count * 4;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
  GW_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return GW_OK;
}

}  // namespace

int mlp_forward(int n, const double* sigma, const float* w, float* out, cudaStream_t s) {
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  rc = set_smem(k_mlp_forward, SMEM_FWD);
  if (rc) return rc;
  k_mlp_forward<<<grid_for(n, ctx), NH, SMEM_FWD, s>>>(n, reinterpret_cast<const double2*>(sigma), w, out);
  GW_LAUNCH_CHECK("k_mlp_forward");
  return GW_OK;
}

int mlp_start(int n, const double* sigma, const float* w, double* theta, cudaStream_t s) {
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  rc = set_smem(k_mlp_start, SMEM_FWD);
  if (rc) return rc;
  k_mlp_start<<<grid_for(n, ctx), NH, SMEM_FWD, s>>>(n, reinterpret_cast<const double2*>(sigma), w, theta);
  GW_LAUNCH_CHECK("k_mlp_start");
  return GW_OK;
}

int mlp_train_step(int n, const OmegaArr& om, const double* sigma, float* w, float* grad, float* m,
                   float* v, float lr, int step, float* loss, cudaStream_t s) {
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  rc = set_smem(k_mlp_train, SMEM_FWD);
  if (rc) return rc;
  GW_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * MLP_NPARAM, s));
  GW_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
  k_mlp_train<<<grid_for(n, ctx), NH, SMEM_FWD, s>>>(n, om, reinterpret_cast<const double2*>(sigma),
                                                      w, grad, loss);
  GW_LAUNCH_CHECK("k_mlp_train");
  if (lr > 0.0f) {
    const float bc1 = 1.0f - powf(0.9f, float(step));
    const float bc2 = 1.0f - powf(0.999f, float(step));
    k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(MLP_NPARAM, w, grad, m, v, lr, bc1, bc2);
    GW_LAUNCH_CHECK("k_adam");
  }
  return GW_OK;
}

}  // namespace gw
