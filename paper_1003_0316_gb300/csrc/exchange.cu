// Exchange self-energy (Eq. HFterm_MB in the Coulomb eigenbasis, plus the divergent term of
// Eq. exchange_div in its erf form; Sec. III.C-D), FP64:
//   Sigma_x,s = - sum_q w_q sum_{p: state(p) = s, eps_p < 0} sum_mu v_mu |m_p,mu|^2
//               - f_s (4 pi / V) C,     f_s = 1 if eps_s < 0.
// One warp per pair (lanes over the basis index, coalesced row reads), FP64 atomics into the
// state's entry.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int XMAXQ = 64;

struct XLaunch {
  const void* M[XMAXQ];
  const int* state[XMAXQ];
  const double* eps[XMAXQ];
  const double* v[XMAXQ];
  int64_t npair[XMAXQ];
  int64_t pair0[XMAXQ + 1];
  int nb[XMAXQ];
  double wq[XMAXQ];
  int nq;
};

template <typename C>
__global__ void k_sigma_x(XLaunch L, int nsig, double* __restrict__ out, unsigned* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  const int64_t total = L.pair0[L.nq];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += warps) {
    int q = 0;
    while (q + 1 < L.nq && e >= L.pair0[q + 1]) ++q;
    const int64_t p = e - L.pair0[q];
    const double ep = L.eps[q][p];
    if (!(ep < 0.0)) continue;                 // only occupied partners n'
    const int st = L.state[q][p];
    if (st < 0 || st >= nsig) {
      if (lane == 0) raise_status(status, ST_EINVAL);
      continue;
    }
    const int nb = L.nb[q];
    const C* row = static_cast<const C*>(L.M[q]) + size_t(p) * nb;
    double acc = 0.0;
    for (int mu = lane; mu < nb; mu += 32) {
      const double x = double(row[mu].x), y = double(row[mu].y);
      acc = fma(L.v[q][mu], x * x + y * y, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(out + st, -L.wq[q] * acc);
  }
}

__global__ void k_sigma_x_div(int nsig, const double* __restrict__ eps_state, double term,
                              double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsig && eps_state[s] < 0.0) out[s] -= term;
}

}  // namespace

int sigma_x(int nq, const double* wq, const int64_t* npair, const int* nb, const void* const* M,
            int dtype, const int* const* state, const double* const* eps, const double* const* v,
            int nsig, const double* eps_state, double cbz, double volume, double* out,
            cudaStream_t s, const DeviceCtx& ctx) {
  GW_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * nsig, s));
  for (int q0 = 0; q0 < nq; q0 += XMAXQ) {
    const int n = nq - q0 < XMAXQ ? nq - q0 : XMAXQ;
    XLaunch L{};
    L.nq = n;
    L.pair0[0] = 0;
    for (int q = 0; q < n; ++q) {
      L.M[q] = M[q0 + q];
      L.state[q] = state[q0 + q];
      L.eps[q] = eps[q0 + q];
      L.v[q] = v[q0 + q];
      L.npair[q] = npair[q0 + q];
      L.nb[q] = nb[q0 + q];
      L.wq[q] = wq[q0 + q];
      L.pair0[q + 1] = L.pair0[q] + npair[q0 + q];
    }
    if (L.pair0[n] == 0) continue;
    const int64_t blocks64 = (L.pair0[n] + 7) / 8;
    const unsigned blocks = unsigned(blocks64 < int64_t(ctx.sm_count) * 32 ? blocks64 : int64_t(ctx.sm_count) * 32);
    if (dtype == GW_C128)
      k_sigma_x<double2><<<blocks, 256, 0, s>>>(L, nsig, out, ctx.status);
    else
      k_sigma_x<float2><<<blocks, 256, 0, s>>>(L, nsig, out, ctx.status);
    GW_LAUNCH_CHECK("k_sigma_x");
  }
  const double term = 4.0 * 3.14159265358979323846 / volume * cbz;
  k_sigma_x_div<<<(nsig + 255) / 256, 256, 0, s>>>(nsig, eps_state, term, out);
  GW_LAUNCH_CHECK("k_sigma_x_div");
  return GW_OK;
}

}  // namespace gw
