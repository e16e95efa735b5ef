// Internal declarations shared by the translation units of libgw.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <math.h>

#include "gw.h"

namespace gw {

// ---------------------------------------------------------------- errors ----
// Bits of the device status word (one per device, see gw_check).
enum : unsigned {
  ST_EINVAL = 1u << 0,
  ST_ENONFINITE = 1u << 1,
  ST_ENOTHPD = 1u << 2,
  ST_ETIMEOUT = 1u << 3,
};

int set_error(int code, const char* fmt, ...);  // records a thread-local message
int cuda_error(cudaError_t e, const char* where);

#define GW_CUDA_TRY(call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::gw::cuda_error(e_, #call); \
  } while (0)

#define GW_LAUNCH_CHECK(where)                              \
  do {                                                     \
    cudaError_t e_ = cudaGetLastError();                   \
    if (e_ != cudaSuccess) return ::gw::cuda_error(e_, where); \
  } while (0)

// Per-device context: status word address and SM count.
struct DeviceCtx {
  unsigned* status;   // device address of the status word
  int sm_count;
  int device;
};
int device_ctx(DeviceCtx* out);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device), thread safe
// (a mutex guards the record of what was set; a larger size is set again).
int set_max_dyn_smem(const void* kernel, size_t bytes, int device);

__device__ __forceinline__ void raise_status(unsigned* status, unsigned bit) {
  atomicOr(status, bit);
}

// ------------------------------------------------------------- omega mesh ---
struct OmegaArr {
  double v[GW_MAX_NW];
};

// ---------------------------------------------------------- workspace -------
// Bump allocator over the caller's workspace (256-byte aligned slices).
struct WsCursor {
  char* base;
  size_t size;
  size_t used;
  __host__ void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    if (base == nullptr || off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};
inline size_t ws_round(size_t b) { return (b + 255) & ~size_t(255); }

// ---------------------------------------------------------- launchers -------
// transition energies of one q
int launch_make_delta(int nk, int nocc, int nunocc, const double* eo, int ldo, const double* eu,
                      int ldu, const int* kq, double* delta, cudaStream_t s, const DeviceCtx& ctx);
// a1
int launch_weights(int64_t K, const double* delta, const double* f, double pref, int nw,
                   const OmegaArr& om, double* w, cudaStream_t s, const DeviceCtx& ctx);

// a2
struct PolQ {
  const void* M;
  const double* delta;
  const double* dbar;   // extrapolar correction: Delta_bar per transition (NULL: none)
  const double* f;
  double* P;
  int64_t K;
  int nb;
};
// resolved execution options (defaults filled in)
struct PolOpts {
  bool accumulate = false;
  int group_items_per_sm = 4;
  int b_stages = 4;
  int fp64_waves = 4;
  bool serial_prep = false;        // no overlap of a group's preparation with the HERK before
  void* const* input_events = nullptr;   // per q: cudaEvent_t to wait for before reading its inputs
  void* const* events = nullptr;   // cudaEvent_t pairs around the HERK launches
  int n_events = 0;
  int launches = 0;                // out: HERK launches of the call
};
int resolve_pol_options(const gw_pol_options* o, PolOpts* out);
// records the pair's start (end = false) or end event of HERK launch `idx`, if one was given
int record_herk_event(PolOpts& o, int idx, bool end, cudaStream_t s);
size_t pol_fp64_workspace(int nq, const int64_t* K, const int* nb, int nw, const PolOpts& o);
int pol_fp64(int nq, const PolQ* qs, double pref, int nw, const OmegaArr& om, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx, PolOpts& o);
size_t pol_tc_workspace(int nq, const int64_t* K, const int* nb, int nw, int precision,
                        const PolOpts& o);
// the HERK wait counters of a profiling build (GW_EUNSUPPORTED otherwise)
int herk_wait_profile(unsigned long long* counters, int n, int reset);
int pol_tc(int nq, const PolQ* qs, double pref, int nw, const OmegaArr& om, int precision,
           bool real, void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx,
           PolOpts& o);

// extrapolar correction (completeness term of P, extra pair coefficients of Sigma^c)
struct ComplQ {
  const void* C;        // [nkn][nb][nb] complex128 / complex64 / float32
  const double* dbar;   // [nkn]
  const double* f;      // [nkn] or NULL
  double* P;            // [nw][nb][nb] complex128, accumulated
  int64_t nkn;
  int nb;
};
int completeness_add(int nq, const ComplQ* qs, int dtype, double pref, int nw, const OmegaArr& om,
                     cudaStream_t s, const DeviceCtx& ctx);
size_t sigma_extrapolar_workspace(int nq, int nw, int nsig, int sm_count);
int sigma_extrapolar(int nq, const double* wq, const int* nb, int nsig, const double* const* S,
                     int nw, const OmegaArr& om, const double* const* Wc, const int64_t* npair,
                     const int* const* pair_state, const double* const* c, const double* ebar,
                     int nw_out, const OmegaArr& om_out, double* sigma, double* cbar, void* ws,
                     size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);

// a3
size_t dielectric_workspace(int nq, const int* nb, int nw);
int dielectric_wc(int nq, const int* nb, int nw, const double* const* v, const double* const* P,
                  double* const* Wc, void* ws, size_t ws_bytes, cudaStream_t s,
                  const DeviceCtx& ctx);
// real symmetric systems (inversion symmetry): real factor and inverse, W^c imaginary parts 0
size_t dielectric_real_workspace(int nq, const int* nb, int nw);
int dielectric_wc_real(int nq, const int* nb, int nw, const double* const* v,
                       const double* const* P, double* const* Wc, void* ws, size_t ws_bytes,
                       cudaStream_t s, const DeviceCtx& ctx);

// a5
size_t paircoef_workspace(int nq, const int64_t* npair, const int* nb, int nw, int precision);
int paircoef(int nq, const int64_t* npair, const int* nb, const void* const* Msig, int dtype,
             int nw, const double* const* Wc, double* const* c, int precision, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);

// a6
size_t convolve_workspace(int nq, const int64_t* npair, int nw, int nw_out);
int convolve(int nq, const double* wq, const int64_t* npair, int nw, const OmegaArr& om,
             const double* const* c, const int* const* pair_state, const double* const* eps,
             int nw_out, const OmegaArr& om_out, int nsig, double* sigma, void* ws,
             size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);
// the same, adding into sigma when accumulate is set (workspace: convolve_workspace)
int convolve_acc(int nq, const double* wq, const int64_t* npair, int nw, const OmegaArr& om,
                 const double* const* c, const int* const* pair_state, const double* const* eps,
                 int nw_out, const OmegaArr& om_out, int nsig, double* sigma, bool accumulate,
                 void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);

// quasiparticle energies
int qp_solve(int n, int npole, const double* params, const double* eps, const double* sigx,
             const double* vxc, double* E, double* Z, int* status, cudaStream_t s);

// diagnostic of the bounded waits
int selftest_bounded_wait(double limit_ms, cudaStream_t s, const DeviceCtx& ctx);
int probe_mma_issue(int variant, int rounds, double* cycles_per_mma, cudaStream_t s,
                    const DeviceCtx& ctx);

// memory waves
int plan_waves(int nq, const int64_t* K, const int* nb, int nw, int precision, size_t budget,
               int* wave_of_q, int* nwaves);

// exchange self-energy
int sigma_x(int nq, const double* wq, const int64_t* npair, const int* nb, const void* const* M,
            int dtype, const int* const* state, const double* const* eps, const double* const* v,
            int nsig, const double* eps_state, double cbz, double volume, double* out,
            cudaStream_t s, const DeviceCtx& ctx);

// a4 (q = Gamma)
size_t gamma_workspace(int nb, int nw);
int gamma_screened_w(int nb, int nw, const double* v, const double* Paug, double* Wc,
                     double* head, double* L, double* u_out, void* ws, size_t ws_bytes,
                     cudaStream_t s, const DeviceCtx& ctx);
size_t bz_constant_workspace(const DeviceCtx& ctx);
int bz_constant_sc(double a, int n, double beta, double* out, void* ws, size_t ws_bytes,
                   cudaStream_t s, const DeviceCtx& ctx);
size_t sigma_div_workspace(int nw, int nsig);
int sigma_div(int nw, const OmegaArr& om, const double* head, double cbz, double volume, int nsig,
              const double* eps_state, int nw_out, const OmegaArr& om_out, double* sigma,
              void* ws, size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);

}  // namespace gw

namespace gw {
int synth_projections(uint64_t seed, uint32_t tid, uint32_t q, int64_t row0, int64_t rows, int nb,
                      int dtype, void* out, cudaStream_t s, const DeviceCtx& ctx);
int launch_lm(int ncurve, int nw, const OmegaArr& om, const double* sigma, const double* sign,
              int npole, const double* theta_init, double* params, double* cost, int* iters,
              int* status, int keep_better, cudaStream_t s);
int mlp_forward(int n, const double* sigma, const float* w, float* out, cudaStream_t s);
int mlp_start(int n, const double* sigma, const float* w, double* theta, cudaStream_t s);
int mlp_train_step(int n, const OmegaArr& om, const double* sigma, float* w, float* grad, float* m,
                   float* v, float lr, int step, float* loss, cudaStream_t s);
int dielectric_wc_noalloc(int nb, int nw, const double* v, const double* P, double* Wc,
                          cudaStream_t s, const DeviceCtx& ctx);
size_t quad_tc_workspace(int nq, const int64_t* npair, const int* nb, int nw, int precision);
int quad_tc(int nq, const int64_t* npair, const int* nb, const void* const* Msig, int nw,
            const double* const* Wc, double* const* c, int precision, bool real, void* ws,
            size_t ws_bytes, cudaStream_t s, const DeviceCtx& ctx);
constexpr int MLP_NIN = 48, MLP_NH = 128, MLP_NOUT = 8;
constexpr int MLP_NPARAM = MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NOUT * MLP_NH + MLP_NOUT;
}  // namespace gw
