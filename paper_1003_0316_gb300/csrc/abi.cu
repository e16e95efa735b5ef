// C ABI entry points of libgw: argument validation, the error model, workspace
// sizing and dispatch to the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <map>
#include <utility>
#include <string>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  return set_error(GW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// One status word per device; its address is looked up once per device.
static __device__ unsigned g_status_word;
static std::mutex g_ctx_mu;
static DeviceCtx g_ctx[64];
static bool g_ctx_ok[64];

int device_ctx(DeviceCtx* out) {
  int dev = 0;
  GW_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(GW_EINVAL, "device id %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  if (!g_ctx_ok[dev]) {
    DeviceCtx c{};
    c.device = dev;
    void* p = nullptr;
    GW_CUDA_TRY(cudaGetSymbolAddress(&p, g_status_word));
    c.status = static_cast<unsigned*>(p);
    GW_CUDA_TRY(cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev));
    g_ctx[dev] = c;
    g_ctx_ok[dev] = true;
  }
  *out = g_ctx[dev];
  return GW_OK;
}

static std::mutex g_attr_mu;
static std::map<std::pair<const void*, int>, size_t> g_attr_set;

int set_max_dyn_smem(const void* kernel, size_t bytes, int device) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(kernel, device);
  auto it = g_attr_set.find(key);
  if (it != g_attr_set.end() && it->second >= bytes) return GW_OK;
  GW_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  g_attr_set[key] = bytes;
  return GW_OK;
}

static int fill_omega(int nw, const double* omega, OmegaArr* o, bool require_positive,
                      bool require_ascending) {
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (omega == nullptr) return set_error(GW_EINVAL, "omega_host is NULL");
  memset(o, 0, sizeof(*o));
  for (int j = 0; j < nw; ++j) {
    double w = omega[j];
    if (!std::isfinite(w)) return set_error(GW_EINVAL, "omega[%d] not finite", j);
    if (require_positive ? !(w > 0.0) : !(w >= 0.0))
      return set_error(GW_EINVAL, "omega[%d]=%g must be %s", j, w,
                       require_positive ? "> 0" : ">= 0");
    if (require_ascending && j > 0 && !(w > omega[j - 1]))
      return set_error(GW_EINVAL, "omega must be strictly ascending (index %d)", j);
    o->v[j] = w;
  }
  return GW_OK;
}

static int check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return GW_OK;
  if (ws == nullptr || ws_bytes < need)
    return set_error(GW_EWORKSPACE, "workspace of %zu bytes given, %zu needed", ws_bytes, need);
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return set_error(GW_EWORKSPACE, "workspace not 256-byte aligned");
  return GW_OK;
}

int resolve_pol_options(const gw_pol_options* o, PolOpts* out) {
  *out = PolOpts{};
  if (o == nullptr) return GW_OK;
  if (o->group_items_per_sm < 0 || o->fp64_waves < 0 || o->n_herk_events < 0)
    return set_error(GW_EINVAL, "negative count in gw_pol_options");
  if (o->b_stages != 0 && o->b_stages != 4 && o->b_stages != 6)
    return set_error(GW_EINVAL, "b_stages=%d: 0, 4 or 6", o->b_stages);
  if (o->n_herk_events > 0 && o->herk_events == nullptr)
    return set_error(GW_EINVAL, "n_herk_events > 0 with NULL herk_events");
  out->accumulate = o->accumulate != 0;
  if (o->group_items_per_sm) out->group_items_per_sm = o->group_items_per_sm;
  if (o->b_stages) out->b_stages = o->b_stages;
  if (o->fp64_waves) out->fp64_waves = o->fp64_waves;
  out->serial_prep = o->serial_prep != 0;
  out->input_events = o->input_events;
  out->events = o->herk_events;
  out->n_events = o->n_herk_events;
  return GW_OK;
}

int record_herk_event(PolOpts& o, int idx, bool end, cudaStream_t s) {
  if (o.events == nullptr || idx >= o.n_events) return GW_OK;
  cudaEvent_t ev = static_cast<cudaEvent_t>(o.events[2 * idx + (end ? 1 : 0)]);
  if (ev == nullptr) return GW_OK;
  GW_CUDA_TRY(cudaEventRecord(ev, s));
  return GW_OK;
}

}  // namespace gw

using namespace gw;

extern "C" {

int gw_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* gw_last_error(void) { return g_last_error.c_str(); }

int gw_check(gw_stream_t stream) {
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  GW_CUDA_TRY(cudaStreamSynchronize(stream));
  unsigned word = 0;
  GW_CUDA_TRY(cudaMemcpy(&word, ctx.status, sizeof(word), cudaMemcpyDeviceToHost));
  unsigned zero = 0;
  GW_CUDA_TRY(cudaMemcpy(ctx.status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
  if (word & ST_ETIMEOUT) return set_error(GW_ETIMEOUT, "a bounded device wait expired");
  if (word & ST_ENOTHPD)
    return set_error(GW_ENOTHPD, "dielectric matrix not positive definite (P not NSD)");
  if (word & ST_ENONFINITE) return set_error(GW_ENONFINITE, "non-finite value on the device");
  if (word & ST_EINVAL)
    return set_error(GW_EINVAL, "invalid input data found on the device (Delta <= 0 or e == 0)");
  return GW_OK;
}

int gw_herk_wait_profile(unsigned long long* counters, int n, int reset) {
  return herk_wait_profile(counters, n, reset);
}

int gw_make_delta(int nk, int nocc, int nunocc, const double* eps_occ_dev, int ld_occ,
                  const double* eps_unocc_dev, int ld_unocc, const int* kq_dev,
                  double* delta_dev, gw_stream_t stream) {
  if (nk < 0 || nocc < 0 || nunocc < 0)
    return set_error(GW_EINVAL, "negative size (nk=%d, nocc=%d, nunocc=%d)", nk, nocc, nunocc);
  if (ld_occ < nocc || ld_unocc < nunocc)
    return set_error(GW_EINVAL, "leading dimension below its count (ld_occ=%d, ld_unocc=%d)",
                     ld_occ, ld_unocc);
  if (int64_t(nk) * nocc * nunocc == 0) return GW_OK;
  if (!eps_occ_dev || !eps_unocc_dev || !kq_dev || !delta_dev)
    return set_error(GW_EINVAL, "NULL eps_occ_dev, eps_unocc_dev, kq_dev or delta_dev");
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return launch_make_delta(nk, nocc, nunocc, eps_occ_dev, ld_occ, eps_unocc_dev, ld_unocc, kq_dev,
                           delta_dev, stream, ctx);
}

int gw_transition_weights(int64_t K, const double* delta_dev, const double* f_dev,
                          double prefactor, int nw, const double* omega_host, double* w_dev,
                          gw_stream_t stream) {
  if (K < 0) return set_error(GW_EINVAL, "K=%lld < 0", (long long)K);
  OmegaArr om;
  int rc = fill_omega(nw, omega_host, &om, false, false);
  if (rc) return rc;
  if (K == 0) return GW_OK;
  if (delta_dev == nullptr || w_dev == nullptr)
    return set_error(GW_EINVAL, "NULL delta_dev or w_dev");
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return launch_weights(K, delta_dev, f_dev, prefactor, nw, om, w_dev, stream, ctx);
}

static int validate_pol(int nq, const int64_t* K, const int* nb, int precision) {
  if (nq < 1) return set_error(GW_EINVAL, "nq=%d < 1", nq);
  if (K == nullptr || nb == nullptr) return set_error(GW_EINVAL, "NULL K_host or nb_host");
  for (int q = 0; q < nq; ++q) {
    if (K[q] < 0) return set_error(GW_EINVAL, "K[%d] < 0", q);
    if (nb[q] < 1 || nb[q] > 8192) return set_error(GW_EINVAL, "nb[%d]=%d outside [1, 8192]", q, nb[q]);
  }
  if (precision != GW_FP64 && precision != GW_TF32X3 && precision != GW_BF16X3)
    return set_error(GW_EINVAL, "unknown precision %d", precision);
  return GW_OK;
}

static size_t polarization_workspace_impl(int nq, const int64_t* K_host, const int* nb_host,
                                          int nw, int precision, const PolOpts& o) {
  if (validate_pol(nq, K_host, nb_host, precision) || nw < 1 || nw > GW_MAX_NW) return 0;
  if (precision == GW_FP64) return pol_fp64_workspace(nq, K_host, nb_host, nw, o);
  return pol_tc_workspace(nq, K_host, nb_host, nw, precision, o);
}

size_t gw_polarization_workspace(int nq, const int64_t* K_host, const int* nb_host, int nw,
                                 int precision) {
  return polarization_workspace_impl(nq, K_host, nb_host, nw, precision, PolOpts{});
}

size_t gw_polarization_workspace_ex(int nq, const int64_t* K_host, const int* nb_host, int nw,
                                    int precision, const gw_pol_options* options) {
  PolOpts o;
  if (resolve_pol_options(options, &o)) return 0;
  return polarization_workspace_impl(nq, K_host, nb_host, nw, precision, o);
}

static int polarization_impl(int nq, const int64_t* K_host, const int* nb_host,
                             const void* const* M_dev, int m_dtype, const double* const* delta_dev,
                             const double* const* dbar_dev, const double* const* f_dev,
                             double prefactor, int nw, const double* omega_host,
                             double* const* P_dev, int precision, void* ws_dev, size_t ws_bytes,
                             gw_stream_t stream, const gw_pol_options* options = nullptr) {
  PolOpts po;
  int rc = resolve_pol_options(options, &po);
  if (rc) return rc;
  rc = validate_pol(nq, K_host, nb_host, precision);
  if (rc) return rc;
  OmegaArr om;
  if ((rc = fill_omega(nw, omega_host, &om, false, false))) return rc;
  if (M_dev == nullptr || delta_dev == nullptr || P_dev == nullptr)
    return set_error(GW_EINVAL, "NULL M_dev, delta_dev or P_dev array");
  if (precision == GW_FP64 && m_dtype != GW_C128)
    return set_error(GW_EUNSUPPORTED, "GW_FP64 needs complex128 projections");
  if (precision != GW_FP64 && m_dtype != GW_C64 && m_dtype != GW_R32)
    return set_error(GW_EUNSUPPORTED, "tensor-core precisions need complex64 or real float32 projections");
  if (!std::isfinite(prefactor)) return set_error(GW_EINVAL, "prefactor not finite");
  std::vector<PolQ> qs(nq);
  for (int q = 0; q < nq; ++q) {
    qs[q].M = M_dev[q];
    qs[q].delta = delta_dev[q];
    qs[q].dbar = dbar_dev ? dbar_dev[q] : nullptr;
    qs[q].f = f_dev ? f_dev[q] : nullptr;
    qs[q].P = P_dev[q];
    qs[q].K = K_host[q];
    qs[q].nb = nb_host[q];
    if (qs[q].P == nullptr) return set_error(GW_EINVAL, "P_dev[%d] is NULL", q);
    if (qs[q].K > 0 && (qs[q].M == nullptr || qs[q].delta == nullptr))
      return set_error(GW_EINVAL, "M_dev[%d] or delta_dev[%d] is NULL", q, q);
    if (dbar_dev && qs[q].K > 0 && qs[q].dbar == nullptr)
      return set_error(GW_EINVAL, "delta_bar_dev[%d] is NULL", q);
    if (precision != GW_FP64 && (reinterpret_cast<uintptr_t>(qs[q].M) & 15u))
      return set_error(GW_EINVAL, "M_dev[%d] not 16-byte aligned", q);
  }
  size_t need = polarization_workspace_impl(nq, K_host, nb_host, nw, precision, po);
  if ((rc = check_ws(ws_dev, ws_bytes, need))) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  if (precision == GW_FP64)
    rc = pol_fp64(nq, qs.data(), prefactor, nw, om, ws_dev, ws_bytes, stream, ctx, po);
  else
    rc = pol_tc(nq, qs.data(), prefactor, nw, om, precision, m_dtype == GW_R32, ws_dev, ws_bytes,
                stream, ctx, po);
  if (options != nullptr && options->herk_launches_out != nullptr)
    *options->herk_launches_out = po.launches;
  return rc;
}

int gw_polarization(int nq, const int64_t* K_host, const int* nb_host, const void* const* M_dev,
                    int m_dtype, const double* const* delta_dev, const double* const* f_dev,
                    double prefactor, int nw, const double* omega_host, double* const* P_dev,
                    int precision, void* ws_dev, size_t ws_bytes, gw_stream_t stream) {
  return polarization_impl(nq, K_host, nb_host, M_dev, m_dtype, delta_dev, nullptr, f_dev,
                           prefactor, nw, omega_host, P_dev, precision, ws_dev, ws_bytes, stream);
}

int gw_polarization_ex(int nq, const int64_t* K_host, const int* nb_host, const void* const* M_dev,
                       int m_dtype, const double* const* delta_dev, const double* const* f_dev,
                       double prefactor, int nw, const double* omega_host, double* const* P_dev,
                       int precision, const gw_pol_options* options, void* ws_dev,
                       size_t ws_bytes, gw_stream_t stream) {
  return polarization_impl(nq, K_host, nb_host, M_dev, m_dtype, delta_dev, nullptr, f_dev,
                           prefactor, nw, omega_host, P_dev, precision, ws_dev, ws_bytes, stream,
                           options);
}

int gw_polarization_extrapolar(int nq, const int64_t* K_host, const int* nb_host,
                               const void* const* M_dev, int m_dtype,
                               const double* const* delta_dev, const double* const* delta_bar_dev,
                               const double* const* f_dev, const int64_t* nkn_host,
                               const void* const* C_dev, const double* const* delta_bar_kn_dev,
                               const double* const* f_kn_dev, double prefactor, int nw,
                               const double* omega_host, double* const* P_dev, int precision,
                               void* ws_dev, size_t ws_bytes, gw_stream_t stream) {
  if (delta_bar_dev == nullptr || nkn_host == nullptr || C_dev == nullptr ||
      delta_bar_kn_dev == nullptr)
    return set_error(GW_EINVAL, "NULL delta_bar_dev, nkn_host, C_dev or delta_bar_kn_dev");
  for (int q = 0; q < nq; ++q) {
    if (nkn_host[q] < 0) return set_error(GW_EINVAL, "nkn[%d] < 0", q);
    if (nkn_host[q] > 0 && (C_dev[q] == nullptr || delta_bar_kn_dev[q] == nullptr))
      return set_error(GW_EINVAL, "C_dev[%d] or delta_bar_kn_dev[%d] is NULL", q, q);
  }
  int rc = polarization_impl(nq, K_host, nb_host, M_dev, m_dtype, delta_dev, delta_bar_dev, f_dev,
                             prefactor, nw, omega_host, P_dev, precision, ws_dev, ws_bytes, stream);
  if (rc) return rc;
  OmegaArr om;
  if ((rc = fill_omega(nw, omega_host, &om, false, false))) return rc;
  std::vector<ComplQ> cq(nq);
  for (int q = 0; q < nq; ++q) {
    cq[q].C = C_dev[q];
    cq[q].dbar = delta_bar_kn_dev[q];
    cq[q].f = f_kn_dev ? f_kn_dev[q] : nullptr;
    cq[q].P = P_dev[q];
    cq[q].nkn = nkn_host[q];
    cq[q].nb = nb_host[q];
  }
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return completeness_add(nq, cq.data(), m_dtype, prefactor, nw, om, stream, ctx);
}

size_t gw_screened_w_workspace(int nq, const int* nb_host, int nw) {
  if (nq < 1 || nb_host == nullptr || nw < 1 || nw > GW_MAX_NW) return 0;
  for (int q = 0; q < nq; ++q)
    if (nb_host[q] < 1 || nb_host[q] > 8192) return 0;
  return dielectric_workspace(nq, nb_host, nw);
}

int gw_screened_w(int nq, const int* nb_host, int nw, const double* const* v_dev,
                  const double* const* P_dev, double* const* Wc_dev, void* ws_dev,
                  size_t ws_bytes, gw_stream_t stream) {
  if (nq < 1 || nb_host == nullptr) return set_error(GW_EINVAL, "nq < 1 or NULL nb_host");
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (v_dev == nullptr || P_dev == nullptr || Wc_dev == nullptr)
    return set_error(GW_EINVAL, "NULL v_dev, P_dev or Wc_dev array");
  for (int q = 0; q < nq; ++q) {
    if (nb_host[q] < 1 || nb_host[q] > 8192) return set_error(GW_EINVAL, "nb[%d]=%d", q, nb_host[q]);
    if (!v_dev[q] || !P_dev[q] || !Wc_dev[q]) return set_error(GW_EINVAL, "NULL pointer for q=%d", q);
  }
  size_t need = dielectric_workspace(nq, nb_host, nw);
  int rc = check_ws(ws_dev, ws_bytes, need);
  if (rc) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return dielectric_wc(nq, nb_host, nw, v_dev, P_dev, Wc_dev, ws_dev, ws_bytes, stream, ctx);
}

size_t gw_screened_w_real_workspace(int nq, const int* nb_host, int nw) {
  if (nq < 1 || nb_host == nullptr || nw < 1 || nw > GW_MAX_NW) return 0;
  for (int q = 0; q < nq; ++q)
    if (nb_host[q] < 1 || nb_host[q] > 8192) return 0;
  return dielectric_real_workspace(nq, nb_host, nw);
}

int gw_screened_w_real(int nq, const int* nb_host, int nw, const double* const* v_dev,
                       const double* const* P_dev, double* const* Wc_dev, void* ws_dev,
                       size_t ws_bytes, gw_stream_t stream) {
  if (nq < 1 || nb_host == nullptr) return set_error(GW_EINVAL, "nq < 1 or NULL nb_host");
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (v_dev == nullptr || P_dev == nullptr || Wc_dev == nullptr)
    return set_error(GW_EINVAL, "NULL v_dev, P_dev or Wc_dev array");
  for (int q = 0; q < nq; ++q) {
    if (nb_host[q] < 1 || nb_host[q] > 8192) return set_error(GW_EINVAL, "nb[%d]=%d", q, nb_host[q]);
    if (!v_dev[q] || !P_dev[q] || !Wc_dev[q]) return set_error(GW_EINVAL, "NULL pointer for q=%d", q);
  }
  int rc = check_ws(ws_dev, ws_bytes, dielectric_real_workspace(nq, nb_host, nw));
  if (rc) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return dielectric_wc_real(nq, nb_host, nw, v_dev, P_dev, Wc_dev, ws_dev, ws_bytes, stream, ctx);
}

int gw_screened_w_noalloc(int nb, int nw, const double* v_dev, const double* P_dev,
                          double* Wc_dev, gw_stream_t stream) {
  if (nb < 1 || nb > 8192) return set_error(GW_EINVAL, "nb=%d outside [1, 8192]", nb);
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (!v_dev || !P_dev || !Wc_dev) return set_error(GW_EINVAL, "NULL v_dev, P_dev or Wc_dev");
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return dielectric_wc_noalloc(nb, nw, v_dev, P_dev, Wc_dev, stream, ctx);
}

static int validate_pairs(int nq, const int64_t* npair, const int* nb, int precision, int m_dtype) {
  if (nq < 1 || npair == nullptr || nb == nullptr)
    return set_error(GW_EINVAL, "nq < 1 or NULL npair_host/nb_host");
  for (int q = 0; q < nq; ++q) {
    if (npair[q] < 0) return set_error(GW_EINVAL, "npair[%d] < 0", q);
    if (nb[q] < 1 || nb[q] > 8192) return set_error(GW_EINVAL, "nb[%d]=%d", q, nb[q]);
  }
  if (precision != GW_FP64 && precision != GW_TF32X3 && precision != GW_BF16X3)
    return set_error(GW_EINVAL, "unknown precision %d", precision);
  if (precision == GW_FP64 && m_dtype != GW_C128)
    return set_error(GW_EUNSUPPORTED, "GW_FP64 needs complex128 projections");
  if (precision != GW_FP64 && m_dtype != GW_C64 && m_dtype != GW_R32)
    return set_error(GW_EUNSUPPORTED, "tensor-core precisions need complex64 or real float32 projections");
  return GW_OK;
}

int gw_sigma_pair_coeffs(int nq, const int64_t* npair_host, const int* nb_host,
                         const void* const* Msig_dev, int m_dtype, int nw,
                         const double* const* Wc_dev, double* const* c_dev, int precision,
                         void* ws_dev, size_t ws_bytes, gw_stream_t stream) {
  int rc = validate_pairs(nq, npair_host, nb_host, precision, m_dtype);
  if (rc) return rc;
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (!Msig_dev || !Wc_dev || !c_dev) return set_error(GW_EINVAL, "NULL pointer array");
  for (int q = 0; q < nq; ++q) {
    if (npair_host[q] > 0 && (!Msig_dev[q] || !Wc_dev[q] || !c_dev[q]))
      return set_error(GW_EINVAL, "NULL pointer for q=%d", q);
    if (precision != GW_FP64 && (reinterpret_cast<uintptr_t>(Msig_dev[q]) & 15u))
      return set_error(GW_EINVAL, "Msig_dev[%d] not 16-byte aligned", q);
  }
  size_t need = paircoef_workspace(nq, npair_host, nb_host, nw, precision);
  if ((rc = check_ws(ws_dev, ws_bytes, need))) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return paircoef(nq, npair_host, nb_host, Msig_dev, m_dtype, nw, Wc_dev, c_dev, precision,
                  ws_dev, ws_bytes, stream, ctx);
}

size_t gw_sigma_convolve_workspace(int nq, const int64_t* npair_host) {
  if (nq < 1 || !npair_host) return 0;
  for (int q = 0; q < nq; ++q)
    if (npair_host[q] < 0) return 0;
  return convolve_workspace(nq, npair_host, 0, 0);
}

int gw_sigma_convolve(int nq, const double* wq_host, const int64_t* npair_host, int nw,
                      const double* omega_host, const double* const* c_dev,
                      const int* const* pair_state_dev, const double* const* eps_dev,
                      int nw_out, const double* omega_out_host, int nsig, double* sigma_dev,
                      void* ws_dev, size_t ws_bytes, gw_stream_t stream) {
  if (nq < 1 || !wq_host || !npair_host) return set_error(GW_EINVAL, "nq < 1 or NULL host array");
  if (nw < 4) return set_error(GW_EINVAL, "the convolution needs nw >= 4 nodes (nw=%d)", nw);
  OmegaArr om, om_out;
  int rc = fill_omega(nw, omega_host, &om, true, true);
  if (rc) return rc;
  if (nw_out < 1 || nw_out > GW_MAX_NW || !omega_out_host)
    return set_error(GW_EINVAL, "nw_out=%d outside [1, %d] or NULL omega_out", nw_out, GW_MAX_NW);
  memset(&om_out, 0, sizeof(om_out));
  for (int i = 0; i < nw_out; ++i) {
    if (!std::isfinite(omega_out_host[i])) return set_error(GW_EINVAL, "omega_out[%d] not finite", i);
    om_out.v[i] = omega_out_host[i];
  }
  if (nsig < 1 || !sigma_dev) return set_error(GW_EINVAL, "nsig < 1 or NULL sigma_dev");
  if (!c_dev || !pair_state_dev || !eps_dev) return set_error(GW_EINVAL, "NULL pointer array");
  for (int q = 0; q < nq; ++q) {
    if (npair_host[q] < 0) return set_error(GW_EINVAL, "npair[%d] < 0", q);
    if (!std::isfinite(wq_host[q])) return set_error(GW_EINVAL, "wq[%d] not finite", q);
    if (npair_host[q] > 0 && (!c_dev[q] || !pair_state_dev[q] || !eps_dev[q]))
      return set_error(GW_EINVAL, "NULL pointer for q=%d", q);
  }
  if ((rc = check_ws(ws_dev, ws_bytes, gw_sigma_convolve_workspace(nq, npair_host)))) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return convolve(nq, wq_host, npair_host, nw, om, c_dev, pair_state_dev, eps_dev, nw_out, om_out,
                  nsig, sigma_dev, ws_dev, ws_bytes, stream, ctx);
}

size_t gw_sigma_extrapolar_workspace(int nq, int nw, int nsig) {
  if (nq < 1 || nw < 1 || nw > GW_MAX_NW || nsig < 1) return 0;
  return sigma_extrapolar_workspace(nq, nw, nsig, 0);
}

int gw_sigma_extrapolar(int nq, const double* wq_host, const int* nb_host, int nsig,
                        const double* const* S_dev, int nw, const double* omega_host,
                        const double* const* Wc_dev, const int64_t* npair_host,
                        const int* const* pair_state_dev, const double* const* c_dev,
                        const double* ebar_host, int nw_out, const double* omega_out_host,
                        double* sigma_dev, double* cbar_dev, void* ws_dev, size_t ws_bytes,
                        gw_stream_t stream) {
  if (nq < 1 || !wq_host || !nb_host || !npair_host || !ebar_host)
    return set_error(GW_EINVAL, "nq < 1 or NULL host array");
  if (nw < 4) return set_error(GW_EINVAL, "the convolution needs nw >= 4 nodes (nw=%d)", nw);
  OmegaArr om, om_out;
  int rc = fill_omega(nw, omega_host, &om, true, true);
  if (rc) return rc;
  if (nw_out < 1 || nw_out > GW_MAX_NW || !omega_out_host)
    return set_error(GW_EINVAL, "nw_out=%d outside [1, %d] or NULL omega_out", nw_out, GW_MAX_NW);
  memset(&om_out, 0, sizeof(om_out));
  for (int i = 0; i < nw_out; ++i) {
    if (!std::isfinite(omega_out_host[i])) return set_error(GW_EINVAL, "omega_out[%d] not finite", i);
    om_out.v[i] = omega_out_host[i];
  }
  if (nsig < 1 || !sigma_dev) return set_error(GW_EINVAL, "nsig < 1 or NULL sigma_dev");
  if (!S_dev || !Wc_dev || !pair_state_dev || !c_dev) return set_error(GW_EINVAL, "NULL pointer array");
  for (int q = 0; q < nq; ++q) {
    if (nb_host[q] < 1 || nb_host[q] > 8192) return set_error(GW_EINVAL, "nb[%d]=%d", q, nb_host[q]);
    if (npair_host[q] < 0) return set_error(GW_EINVAL, "npair[%d] < 0", q);
    if (!std::isfinite(wq_host[q])) return set_error(GW_EINVAL, "wq[%d] not finite", q);
    if (!(ebar_host[q] > 0.0) || !std::isfinite(ebar_host[q]))
      return set_error(GW_EINVAL, "ebar[%d] must be a finite positive energy", q);
    if (!S_dev[q] || !Wc_dev[q]) return set_error(GW_EINVAL, "NULL S_dev or Wc_dev for q=%d", q);
    if (npair_host[q] > 0 && (!c_dev[q] || !pair_state_dev[q]))
      return set_error(GW_EINVAL, "NULL pair pointer for q=%d", q);
  }
  if ((rc = check_ws(ws_dev, ws_bytes, gw_sigma_extrapolar_workspace(nq, nw, nsig)))) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return sigma_extrapolar(nq, wq_host, nb_host, nsig, S_dev, nw, om, Wc_dev, npair_host,
                          pair_state_dev, c_dev, ebar_host, nw_out, om_out, sigma_dev, cbar_dev,
                          ws_dev, ws_bytes, stream, ctx);
}

size_t gw_sigma_workspace(int nq, const int64_t* npair_host, const int* nb_host, int nw,
                          int precision) {
  if (nq < 1 || !npair_host || !nb_host || nw < 1 || nw > GW_MAX_NW) return 0;
  size_t b = 0;
  for (int q = 0; q < nq; ++q) {
    if (npair_host[q] < 0) return 0;
    b += ws_round(sizeof(double) * size_t(nw) * size_t(npair_host[q]));
  }
  // the pair-coefficient scratch and the convolution's share the space after the coefficients
  return b + std::max(paircoef_workspace(nq, npair_host, nb_host, nw, precision),
                      convolve_workspace(nq, npair_host, nw, 0));
}

int gw_sigma_c(int nq, const double* wq_host, const int64_t* npair_host, const int* nb_host,
               const void* const* Msig_dev, int m_dtype, const int* const* pair_state_dev,
               const double* const* eps_dev, int nw, const double* omega_host,
               const double* const* Wc_dev, int nw_out, const double* omega_out_host, int nsig,
               double* sigma_dev, int precision, void* ws_dev, size_t ws_bytes,
               gw_stream_t stream) {
  int rc = validate_pairs(nq, npair_host, nb_host, precision, m_dtype);
  if (rc) return rc;
  size_t need = gw_sigma_workspace(nq, npair_host, nb_host, nw, precision);
  if ((rc = check_ws(ws_dev, ws_bytes, need))) return rc;
  if (nw < 4 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [4, %d]", nw, GW_MAX_NW);
  WsCursor cur{static_cast<char*>(ws_dev), ws_bytes, 0};
  std::vector<double*> cbuf(nq);
  for (int q = 0; q < nq; ++q)
    cbuf[q] = static_cast<double*>(cur.take(sizeof(double) * size_t(nw) * size_t(npair_host[q])));
  size_t off = (cur.used + 255) & ~size_t(255);
  rc = gw_sigma_pair_coeffs(nq, npair_host, nb_host, Msig_dev, m_dtype, nw, Wc_dev, cbuf.data(),
                            precision, static_cast<char*>(ws_dev) + off, ws_bytes - off, stream);
  if (rc) return rc;
  std::vector<const double*> cc(cbuf.begin(), cbuf.end());
  return gw_sigma_convolve(nq, wq_host, npair_host, nw, omega_host, cc.data(), pair_state_dev,
                           eps_dev, nw_out, omega_out_host, nsig, sigma_dev,
                           static_cast<char*>(ws_dev) + off, ws_bytes - off, stream);
}

}  // extern "C"

extern "C" {

int gw_continue(int ncurve, int nw, const double* omega_host, const double* sigma_dev,
                const double* sign_dev, int npole, int method, const float* mlp_dev,
                double* params_dev, double* cost_dev, int* iters_dev, int* status_dev,
                gw_stream_t stream) {
  if (ncurve < 0) return set_error(GW_EINVAL, "ncurve < 0");
  OmegaArr om;
  int rc = fill_omega(nw, omega_host, &om, true, false);
  if (rc) return rc;
  if (npole < 1 || npole > 5) return set_error(GW_EINVAL, "npole=%d outside [1, 5]", npole);
  if (2 * nw < 4 * npole) return set_error(GW_EINVAL, "fewer data (2 nw) than parameters (4 npole)");
  if (ncurve == 0) return GW_OK;
  if (!sigma_dev || !params_dev || !cost_dev || !iters_dev || !status_dev)
    return set_error(GW_EINVAL, "NULL sigma/params/cost/iters/status pointer");
  if (method == GW_FIT_PLAIN)
    return launch_lm(ncurve, nw, om, sigma_dev, sign_dev, npole, nullptr, params_dev, cost_dev,
                     iters_dev, status_dev, 0, stream);
  if (method != GW_FIT_MLP && method != GW_FIT_MLP_ONLY)
    return set_error(GW_EINVAL, "unknown fit method %d", method);
  if (npole != 2 || nw != 24 || !mlp_dev)
    return set_error(GW_EINVAL, "the learned start needs npole = 2, nw = 24 and weights");
  // the network's proposal is written into params_dev and read back as the start
  rc = mlp_start(ncurve, sigma_dev, mlp_dev, params_dev, stream);
  if (rc) return rc;
  rc = launch_lm(ncurve, nw, om, sigma_dev, sign_dev, npole, params_dev, params_dev, cost_dev,
                 iters_dev, status_dev, 0, stream);
  if (rc || method == GW_FIT_MLP_ONLY) return rc;
  return launch_lm(ncurve, nw, om, sigma_dev, sign_dev, npole, nullptr, params_dev, cost_dev,
                   iters_dev, status_dev, 1, stream);
}

int gw_mlp_param_count(void) { return MLP_NPARAM; }

int gw_mlp_forward(int n, const double* sigma_dev, const float* mlp_dev, float* out_dev,
                   gw_stream_t stream) {
  if (n < 0 || (n > 0 && (!sigma_dev || !mlp_dev || !out_dev)))
    return set_error(GW_EINVAL, "bad MLP forward arguments");
  if (n == 0) return GW_OK;
  return mlp_forward(n, sigma_dev, mlp_dev, out_dev, stream);
}

int gw_mlp_train_step(int n, const double* omega_host, const double* sigma_dev, float* mlp_dev,
                      float* grad_dev, float* m_dev, float* v_dev, float lr, int step,
                      float* loss_dev, gw_stream_t stream) {
  OmegaArr om;
  int rc = fill_omega(24, omega_host, &om, true, false);
  if (rc) return rc;
  if (n < 1 || !sigma_dev || !mlp_dev || !grad_dev || !loss_dev)
    return set_error(GW_EINVAL, "bad MLP training arguments");
  if (lr > 0.0f && (!m_dev || !v_dev || step < 1))
    return set_error(GW_EINVAL, "Adam step needs moments and step >= 1");
  return mlp_train_step(n, om, sigma_dev, mlp_dev, grad_dev, m_dev, v_dev, lr, step, loss_dev, stream);
}

int gw_synth_projections(uint64_t seed, uint32_t tid, uint32_t q, int64_t row0, int64_t rows,
                         int nb, int m_dtype, void* out_dev, gw_stream_t stream) {
  if (row0 < 0 || rows < 0 || nb < 1) return set_error(GW_EINVAL, "bad synth sizes");
  if (m_dtype != GW_C128 && m_dtype != GW_C64) return set_error(GW_EINVAL, "bad dtype");
  if (rows > 0 && !out_dev) return set_error(GW_EINVAL, "NULL out_dev");
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return synth_projections(seed, tid, q, row0, rows, nb, m_dtype, out_dev, stream, ctx);
}

}  // extern "C"

extern "C" {

size_t gw_gamma_workspace(int nb, int nw) {
  if (nb < 1 || nw < 1) return 0;
  return gamma_workspace(nb, nw);
}

int gw_gamma_screened_w(int nb, int nw, const double* v_dev, const double* Paug_dev,
                        double* Wc_dev, double* head_dev, double* L_dev, double* u_dev,
                        void* ws_dev, size_t ws_bytes, gw_stream_t stream) {
  if (nb < 1 || nb > 8192) return set_error(GW_EINVAL, "nb=%d outside [1, 8192]", nb);
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (!v_dev || !Paug_dev || !Wc_dev || !head_dev)
    return set_error(GW_EINVAL, "NULL v_dev, Paug_dev, Wc_dev or head_dev");
  int rc = check_ws(ws_dev, ws_bytes, gamma_workspace(nb, nw));
  if (rc) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return gamma_screened_w(nb, nw, v_dev, Paug_dev, Wc_dev, head_dev, L_dev, u_dev, ws_dev,
                          ws_bytes, stream, ctx);
}

size_t gw_bz_constant_workspace(void) {
  DeviceCtx ctx;
  if (device_ctx(&ctx)) return 0;
  return bz_constant_workspace(ctx);
}

int gw_bz_constant_sc(double a, int n, double beta, double* out_host, void* ws_dev,
                      size_t ws_bytes, gw_stream_t stream) {
  if (!(a > 0.0) || n < 1 || !(beta > 0.0 && beta < 1.0) || !out_host)
    return set_error(GW_EINVAL, "need a > 0, n >= 1, 0 < beta < 1 and an output");
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return bz_constant_sc(a, n, beta, out_host, ws_dev, ws_bytes, stream, ctx);
}

size_t gw_sigma_div_workspace(int nw, int nsig) {
  if (nw < 1 || nsig < 1) return 0;
  return sigma_div_workspace(nw, nsig);
}

int gw_sigma_div(int nw, const double* omega_host, const double* head_dev, double cbz,
                 double volume, int nsig, const double* eps_state_dev, int nw_out,
                 const double* omega_out_host, double* sigma_dev, void* ws_dev, size_t ws_bytes,
                 gw_stream_t stream) {
  if (nw < 4) return set_error(GW_EINVAL, "the convolution needs nw >= 4 nodes (nw=%d)", nw);
  OmegaArr om, om_out;
  int rc = fill_omega(nw, omega_host, &om, true, true);
  if (rc) return rc;
  if (nw_out < 1 || nw_out > GW_MAX_NW || !omega_out_host)
    return set_error(GW_EINVAL, "nw_out=%d outside [1, %d] or NULL omega_out", nw_out, GW_MAX_NW);
  memset(&om_out, 0, sizeof(om_out));
  for (int i = 0; i < nw_out; ++i) {
    if (!std::isfinite(omega_out_host[i])) return set_error(GW_EINVAL, "omega_out[%d] not finite", i);
    om_out.v[i] = omega_out_host[i];
  }
  if (nsig < 1 || !sigma_dev || !head_dev || !eps_state_dev)
    return set_error(GW_EINVAL, "nsig < 1 or NULL sigma_dev, head_dev or eps_state_dev");
  if (!std::isfinite(cbz) || !(volume > 0.0)) return set_error(GW_EINVAL, "bad BZ constant or volume");
  if ((rc = check_ws(ws_dev, ws_bytes, sigma_div_workspace(nw, nsig)))) return rc;
  DeviceCtx ctx;
  if ((rc = device_ctx(&ctx))) return rc;
  return sigma_div(nw, om, head_dev, cbz, volume, nsig, eps_state_dev, nw_out, om_out, sigma_dev,
                   ws_dev, ws_bytes, stream, ctx);
}

}  // extern "C"

extern "C" {

int gw_sigma_x(int nq, const double* wq_host, const int64_t* npair_host, const int* nb_host,
               const void* const* Msig_dev, int m_dtype, const int* const* pair_state_dev,
               const double* const* eps_dev, const double* const* v_dev, int nsig,
               const double* eps_state_dev, double cbz, double volume, double* sigma_x_dev,
               gw_stream_t stream) {
  if (nq < 1 || !wq_host || !npair_host || !nb_host) return set_error(GW_EINVAL, "nq < 1 or NULL host array");
  if (m_dtype != GW_C128 && m_dtype != GW_C64) return set_error(GW_EINVAL, "m_dtype=%d", m_dtype);
  if (nsig < 1 || !sigma_x_dev || !eps_state_dev) return set_error(GW_EINVAL, "nsig < 1 or NULL output");
  if (!std::isfinite(cbz) || !(volume > 0.0)) return set_error(GW_EINVAL, "bad BZ constant or volume");
  if (!Msig_dev || !pair_state_dev || !eps_dev || !v_dev) return set_error(GW_EINVAL, "NULL pointer array");
  for (int q = 0; q < nq; ++q) {
    if (npair_host[q] < 0 || nb_host[q] < 1) return set_error(GW_EINVAL, "bad sizes for q=%d", q);
    if (!std::isfinite(wq_host[q])) return set_error(GW_EINVAL, "wq[%d] not finite", q);
    if (npair_host[q] > 0 && (!Msig_dev[q] || !pair_state_dev[q] || !eps_dev[q] || !v_dev[q]))
      return set_error(GW_EINVAL, "NULL pointer for q=%d", q);
  }
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return sigma_x(nq, wq_host, npair_host, nb_host, Msig_dev, m_dtype, pair_state_dev, eps_dev, v_dev,
                 nsig, eps_state_dev, cbz, volume, sigma_x_dev, stream, ctx);
}

}  // extern "C"

extern "C" {

int gw_plan_waves(int nq, const int64_t* K_host, const int* nb_host, int nw, int precision,
                  size_t budget_bytes, int* wave_of_q, int* nwaves_out) {
  int rc = validate_pol(nq, K_host, nb_host, precision);
  if (rc) return rc;
  if (nw < 1 || nw > GW_MAX_NW) return set_error(GW_EINVAL, "nw=%d outside [1, %d]", nw, GW_MAX_NW);
  if (!wave_of_q || !nwaves_out) return set_error(GW_EINVAL, "NULL output");
  return plan_waves(nq, K_host, nb_host, nw, precision, budget_bytes, wave_of_q, nwaves_out);
}

}  // extern "C"

extern "C" {

int gw_selftest_bounded_wait(double limit_ms, gw_stream_t stream) {
  if (!(limit_ms > 0.0 && limit_ms <= 1000.0))
    return set_error(GW_EINVAL, "limit_ms=%g outside (0, 1000]", limit_ms);
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return selftest_bounded_wait(limit_ms, stream, ctx);
}

int gw_probe_mma_issue(int variant, int rounds, double* cycles_per_mma_host, gw_stream_t stream) {
  if (variant < 0 || variant > 5) return set_error(GW_EINVAL, "variant=%d not in 0..5", variant);
  if (rounds < 2 || rounds > 100000) return set_error(GW_EINVAL, "rounds=%d not in 2..100000", rounds);
  if (!cycles_per_mma_host) return set_error(GW_EINVAL, "NULL cycles_per_mma_host");
  DeviceCtx ctx;
  int rc = device_ctx(&ctx);
  if (rc) return rc;
  return probe_mma_issue(variant, rounds, cycles_per_mma_host, stream, ctx);
}

}  // extern "C"

extern "C" {

int gw_qp_solve(int n, int npole, const double* params_dev, const double* eps_dev,
                const double* sigx_dev, const double* vxc_dev, double* E_dev, double* Z_dev,
                int* status_dev, gw_stream_t stream) {
  if (n < 0) return set_error(GW_EINVAL, "n < 0");
  if (npole < 1 || npole > 5) return set_error(GW_EINVAL, "npole=%d outside [1, 5]", npole);
  if (n == 0) return GW_OK;
  if (!params_dev || !eps_dev || !sigx_dev || !vxc_dev || !E_dev)
    return set_error(GW_EINVAL, "NULL params, eps, sigx, vxc or E pointer");
  return qp_solve(n, npole, params_dev, eps_dev, sigx_dev, vxc_dev, E_dev, Z_dev, status_dev,
                  stream);
}

}  // extern "C"
