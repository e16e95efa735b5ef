/*
 * gw.h -- C ABI of the GB300 (sm_103a) GW hot path: imaginary-frequency
 * polarization, screened interaction, correlation self-energy and its analytic
 * continuation, after Friedrich, Bluegel and Schindlmayr, "Efficient
 * implementation of the GW approximation within the all-electron FLAPW method"
 * (Sec. III.C and III.E).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are device pointers, *_host host pointers. Arrays of
 *     per-q device pointers (e.g. `const void* const* M_dev`) are HOST arrays whose
 *     entries are device pointers. The caller owns every buffer; the library keeps
 *     no pointer after a call returns and never frees caller memory.
 *   - Complex data is interleaved (re, im): complex128 = two doubles, complex64 = two
 *     floats. Matrices are row-major and dense (leading dimension = row length).
 *   - Every compute call only enqueues work ordered on `stream` (no host
 *     synchronisation; gw_polarization* fork to two streams of the library and join them
 *     back to `stream` before returning).
 *     Argument errors are returned at once (GW_EINVAL, message in gw_last_error()).
 *     Errors found on the device (a non-positive-definite dielectric matrix, a
 *     non-finite value, an expired bounded wait) are recorded in a library-owned
 *     device status word and returned by gw_check(), which synchronises the
 *     stream and clears the word. Outputs are unspecified after an error.
 *   - Scratch memory comes from the caller: query the size with the matching
 *     *_workspace() function, pass a device buffer of at least that many bytes
 *     (256-byte aligned); a smaller buffer gives GW_EWORKSPACE.
 *   - Symbols are the paper's: q transfer momentum (the paper's k in Eq. polar_MB),
 *     k summed Bloch vector, t = (k, n occ, n' unocc) a transition with
 *     Delta_t = e_n'(k+q) - e_n(k) > 0, N_b the size of the Coulomb eigenbasis,
 *     omega_j > 0 the imaginary-frequency mesh.
 */
#ifndef GW_H
#define GW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gw_stream_t; /* a cudaStream_t; NULL = legacy default stream */

enum gw_status {
  GW_OK = 0,
  GW_EINVAL = 1,        /* bad argument (sizes, pointers, Delta <= 0, e_n' == 0, ...) */
  GW_EWORKSPACE = 2,    /* workspace missing or too small */
  GW_ECUDA = 3,         /* a CUDA runtime/driver call failed */
  GW_ENONFINITE = 4,    /* a non-finite value was produced or read */
  GW_ENOTHPD = 5,       /* 1 - v^1/2 P v^1/2 not positive definite (P not NSD) */
  GW_ETIMEOUT = 6,      /* a bounded device-side wait expired */
  GW_ENOCONV = 7,       /* a fit did not converge (per-curve status holds details) */
  GW_EUNSUPPORTED = 8   /* combination not built (e.g. precision for this dtype) */
};

/* GW_R32: real float32 projections (inversion-symmetric systems, Sec. II: real basis and
 * wave functions), for the tensor-core precisions of gw_polarization; P is then real
 * symmetric, computed as one real SYRK of half the size and stored with zero imaginary parts. */
enum gw_dtype { GW_C128 = 0, GW_C64 = 1, GW_R32 = 2 };

/* Arithmetic of the P and Sigma contractions. GW_FP64: double precision on the
 * FP64 pipe (M must be GW_C128). GW_TF32X3 ("FP32-split"): tensor-core products of
 * a two-term TF32 split of each FP32 operand (hi*hi + hi*lo + lo*hi), FP32
 * accumulation drained into FP64 partial sums (M must be GW_C64). GW_BF16X3: the
 * same with a two-term BF16 split. */
enum gw_precision { GW_FP64 = 0, GW_TF32X3 = 1, GW_BF16X3 = 2 };

enum gw_fit_method { GW_FIT_PLAIN = 0, GW_FIT_MLP = 1, GW_FIT_MLP_ONLY = 2 };

/* Library version: major * 10000 + minor * 100 + patch. */
int gw_version(void);

/* Message of the last error returned on the calling host thread ("" if none). */
const char* gw_last_error(void);

/* Synchronise `stream`, then return and clear the device status word of the
 * current device (GW_OK if no device-side error was recorded). */
int gw_check(gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * Transition energies of one transfer momentum q (the energy differences in the bracket of
 * Eq. polar_MB, Sec. III.C): for t = (k N_occ + n) N_unocc + n',
 *   Delta_t = e_unocc[kq[k]][n'] - e_occ[k][n],
 * k = 0 .. N_k-1 the mesh points, n < N_occ, n' < N_unocc, kq[k] the mesh index of k + q.
 *   eps_occ_dev   [N_k][ld_occ] double (energies from the Fermi level, Sec. II), ld_occ >= N_occ;
 *   eps_unocc_dev [N_k][ld_unocc] double, ld_unocc >= N_unocc;
 *   kq_dev        [N_k] int, each in [0, N_k);
 *   delta_dev     [N_k N_occ N_unocc] double output (the layout of the projections' rows).
 * Errors: GW_EINVAL for negative sizes, a leading dimension below its count or NULL pointers
 * (nothing is launched); a kq entry outside [0, N_k) is reported by gw_check as GW_EINVAL and
 * its transitions are set to 0 (which gw_polarization then rejects as Delta <= 0). */
int gw_make_delta(int nk, int nocc, int nunocc, const double* eps_occ_dev, int ld_occ,
                  const double* eps_unocc_dev, int ld_unocc, const int* kq_dev,
                  double* delta_dev, gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a1. Transition weights (bracket of Eq. polar_MB at w = i omega, Sec. III.C):
 *   w[j][t] = prefactor * f_t * ( 1/(i omega_j - Delta_t) - 1/(i omega_j + Delta_t) )
 *           = -prefactor * f_t * 2 Delta_t / (Delta_t^2 + omega_j^2).
 * prefactor = 2/N_k (spin sum over the BZ density). f_dev may be NULL (f_t = 1).
 *   delta_dev [K] double, f_dev [K] double or NULL, omega_host [nw] double,
 *   w_dev [nw][K] double (output).
 * Errors: GW_EINVAL if K < 0, nw < 1 or nw > GW_MAX_NW, a NULL required pointer,
 * or omega_j < 0. Delta_t <= 0 is reported by gw_check as GW_EINVAL. */
#define GW_MAX_NW 64
int gw_transition_weights(int64_t K, const double* delta_dev, const double* f_dev,
                          double prefactor, int nw, const double* omega_host,
                          double* w_dev, gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a2. Polarization in the Coulomb eigenbasis (Eq. polar_MB at w = i omega):
 *   P_IJ(q, i omega_j) = sum_t w_tj M_{t,I} conj(M_{t,J}),
 * a weighted Hermitian rank-K_q update per frequency; negative semidefinite.
 * Batched over nq transfer momenta with their own K_q and N_b(q):
 *   K_host[nq], nb_host[nq]                   sizes (K_q >= 0, 1 <= N_b <= 8192),
 *   M_dev[q]      [K_q][N_b] complex (m_dtype) projections M_{t,I},
 *   delta_dev[q]  [K_q] double                 Delta_t > 0,
 *   f_dev         NULL, or host array of nq device pointers ([K_q] double, entries
 *                 may be NULL),
 *   omega_host    [nw] double, 1 <= nw <= GW_MAX_NW,
 *   P_dev[q]      [nw][N_b][N_b] complex128 output, both triangles written.
 * precision: GW_FP64 needs GW_C128; GW_TF32X3 and GW_BF16X3 need GW_C64.
 * Workspace: gw_polarization_workspace() bytes. */
size_t gw_polarization_workspace(int nq, const int64_t* K_host, const int* nb_host,
                                 int nw, int precision);
int gw_polarization(int nq, const int64_t* K_host, const int* nb_host,
                    const void* const* M_dev, int m_dtype,
                    const double* const* delta_dev, const double* const* f_dev,
                    double prefactor, int nw, const double* omega_host,
                    double* const* P_dev, int precision,
                    void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* Execution options of gw_polarization_ex (no counterpart in the paper: they control how the
 * GPU computes Eq. polar_MB, not what is computed; every choice gives the same P up to the
 * rounding of its precision). NULL, or a zero-initialised struct, gives the behaviour of
 * gw_polarization.
 *   accumulate          nonzero: P_dev[q] += this call's sum over its transitions (P is
 *                       additive over transitions, so disjoint slices of a K too large for
 *                       one call are processed one after another into one P); 0: overwrite.
 *   group_items_per_sm  split-precision paths: q points are prepared and launched in groups,
 *                       a group closing at this many work items (128 x 128 tile x frequency)
 *                       per SM; 0 means 4. Larger groups share one launch, smaller ones need
 *                       less workspace.
 *   b_stages            split-precision paths: shared-memory stages of the B operand, 4 or 6
 *                       (two rounds more in flight, less L1 for the A loads); 0 means 4.
 *   fp64_waves          GW_FP64: the K splits fill at least this many waves of CTAs; 0 means 4.
 *   herk_events         NULL, or n_herk_events pairs of cudaEvent_t (created by the caller,
 *                       layout [start, end] per pair): the call records the pair around each
 *                       of its first n_herk_events HERK launches, on the stream the HERK runs
 *                       on (the dominant kernel alone, without the per-q preparation);
 *   n_herk_events       the number of pairs in herk_events;
 *   herk_launches_out   NULL, or (host) the number of HERK launches of the call;
 *   serial_prep         split-precision paths with more than one group: nonzero runs each
 *                       group's preparation (weights, operand copies) on `stream` before its
 *                       HERK launch; 0 (default) prepares group g + 1 on a low-priority stream
 *                       of the library while the HERK of group g runs on a high-priority one
 *                       (the HERK's last, partial wave leaves SMs idle), with two workspace
 *                       slots. Both streams are forked from `stream` at entry and joined to it
 *                       before the call returns: the call is ordered on `stream` either way,
 *                       and a capture of `stream` into a CUDA graph takes both in;
 *   input_events        NULL, or per q (host array) a cudaEvent_t or NULL: the call reads the
 *                       projections and energies of q only after that event (e.g. recorded
 *                       after their host-to-device copy on another stream), so the copies of
 *                       later q overlap the work on earlier ones within one call.
 * gw_polarization_workspace_ex gives the workspace for the same options (group_items_per_sm
 * and fp64_waves change it). Errors: GW_EINVAL for b_stages other than 0, 4 or 6, negative
 * counts. */
typedef struct gw_pol_options {
  int accumulate;
  int group_items_per_sm;
  int b_stages;
  int fp64_waves;
  void* const* herk_events;
  int n_herk_events;
  int* herk_launches_out;
  int serial_prep;
  void* const* input_events;
} gw_pol_options;
size_t gw_polarization_workspace_ex(int nq, const int64_t* K_host, const int* nb_host, int nw,
                                    int precision, const gw_pol_options* options);
int gw_polarization_ex(int nq, const int64_t* K_host, const int* nb_host,
                       const void* const* M_dev, int m_dtype,
                       const double* const* delta_dev, const double* const* f_dev,
                       double prefactor, int nw, const double* omega_host,
                       double* const* P_dev, int precision, const gw_pol_options* options,
                       void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* Wait profile of the split-precision HERK (no counterpart in the paper: an instrument of the
 * kernel design). Only a library built with GW_HERK_WAIT_PROFILE defined (the package's build
 * script with --prof, as libgw_prof.so) counts; every other build returns GW_EUNSUPPORTED. The
 * counters are SM cycles (clock64) of the one issuing thread of each role (lane 0 of each
 * A-transform and epilogue warp), summed over the CTAs of every HERK launch since the last
 * reset, on the current device, in this order:
 *    0 A transform: total   1 waits for the round's weights   2 waits for a free A slot
 *    3 A transform: rounds (count)
 *    4 MMA issue: total     5 waits for the B stage   6 waits for the A slot
 *    7 waits for the drained accumulator   8 MMA issue: rounds (count)
 *    9 epilogue: total     10 waits for a finished accumulator   11 drains (TMEM loads + sums)
 *   12 FP64 folds          13 epilogue: periods (count)
 *   14 B producer: total   15 its waits for a free stage
 *   16 weight producer: total   17 its waits for a free slot
 * gw_herk_wait_profile synchronises the device, copies the first min(n, 18) counters to the host
 * array `counters` (n may be 0) and, if reset != 0, zeroes them. The counting build is slower
 * (clock reads in every loop); its times are not the library's. Errors: GW_EUNSUPPORTED,
 * GW_EINVAL (n < 0, or counters NULL with n > 0), GW_ECUDA. */
#define GW_HERK_WAIT_COUNTERS 18
int gw_herk_wait_profile(unsigned long long* counters, int n, int reset);

/* ---------------------------------------------------------------------------
 * Extrapolar correction of the polarization (Sec. V, the paragraph on the convergence with
 * the number of bands; the scheme of Bruneval and Gonze). The unoccupied sum of Eq. polar_MB
 * is cut at a band N'; every band n' > N' is put at one energy e_bar (the paper takes 16 Ry
 * above the highest kept band), and the completeness of the one-particle states turns the
 * sum over those bands into a full-band integral minus the kept bands:
 *   P^EX_IJ = sum_t [w_tj(Delta_t) - w_tj(Delta_bar_t)] M_{t,I} conj(M_{t,J})
 *           + sum_kn w_j(Delta_bar_kn) C^kn_IJ,
 * w the a1 weight (prefactor and symmetry weight included), kn an occupied state (k, n),
 * Delta_bar_kn = e_bar - e_n(k), Delta_bar_t = Delta_bar of the occupied state of t, and
 * C^kn_IJ = <phi_nk| M_I conj(M_J) |phi_nk>, the full-band sum of M_{kn n',I} conj(M_{kn n',J}).
 * Arguments as gw_polarization, plus per q:
 *   delta_bar_dev[q] [K_q] double > 0 (Delta_bar_t of each kept transition),
 *   nkn_host[q] number of occupied states, C_dev[q] [nkn][N_b][N_b] Hermitian, of the
 *   projections' element type (complex128 for GW_FP64, complex64, or float32 for GW_R32),
 *   delta_bar_kn_dev[q] [nkn] double > 0, f_kn_dev (may be NULL, or f_kn_dev[q]) [nkn] double.
 * P_dev[q] is overwritten with P^EX. The completeness term reads the upper triangle of each
 * C^kn and adds it and its Hermitian mirror; complex128 input is summed in FP64, complex64
 * and float32 input in FP32 per chunk of 32 states with an error-free two-float running sum.
 * Workspace: gw_polarization_workspace(). Delta_bar <= 0 is reported by gw_check as GW_EINVAL. */
int gw_polarization_extrapolar(int nq, const int64_t* K_host, const int* nb_host,
                               const void* const* M_dev, int m_dtype,
                               const double* const* delta_dev, const double* const* delta_bar_dev,
                               const double* const* f_dev, const int64_t* nkn_host,
                               const void* const* C_dev, const double* const* delta_bar_kn_dev,
                               const double* const* f_kn_dev, double prefactor, int nw,
                               const double* omega_host, double* const* P_dev, int precision,
                               void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* Memory waves for many q points (no counterpart in the paper: a scheduling aid for inputs
 * larger than device memory). Assigns each q to a wave so that, per wave, the projections
 * (complex128 for GW_FP64, complex64 otherwise), the gw_polarization workspace of the wave and
 * the P outputs fit in budget_bytes; first-fit decreasing by footprint. Host only.
 *   wave_of_q [nq] output (0-based), *nwaves_out the number of waves. GW_EINVAL if one q
 *   alone exceeds the budget. */
int gw_plan_waves(int nq, const int64_t* K_host, const int* nb_host, int nw, int precision,
                  size_t budget_bytes, int* wave_of_q, int* nwaves_out);

/* ---------------------------------------------------------------------------
 * a3. Dielectric matrix and correlation part of the screened interaction in the
 * Coulomb eigenbasis (Eqs. dielec_MB, screen_MB and W^c = W - v, Sec. III.C):
 *   eps = 1 - v^1/2 P v^1/2,   W^c = v^1/2 (eps^{-1} - 1) v^1/2,
 * computed in FP64 from the Cholesky factor of eps (HPD on the imaginary axis).
 *   v_dev[q]  [N_b] double > 0 Coulomb eigenvalues,
 *   P_dev[q]  [nw][N_b][N_b] complex128 (Hermitian NSD),
 *   Wc_dev[q] [nw][N_b][N_b] complex128 output (may alias P_dev[q]).
 * The factorisation runs over many CTAs (per 32-wide panel: the diagonal block, the panel
 * below it, the trailing update), the inverse factor by block columns, W^c by block rows.
 * A failed factorisation (eps not positive definite, or non-finite entries) is reported by
 * gw_check as GW_ENOTHPD (GW_ENONFINITE); the later phases still run on the half-finished
 * factor, so Wc_dev (and P_dev where it aliases Wc_dev) is undefined after such an error.
 * Workspace: gw_screened_w_workspace() bytes, per (q, frequency) system
 * 16 (2 N_b^2 + 1024 ceil(N_b / 32)) bytes rounded up to 256. */
size_t gw_screened_w_workspace(int nq, const int* nb_host, int nw);
int gw_screened_w(int nq, const int* nb_host, int nw, const double* const* v_dev,
                  const double* const* P_dev, double* const* Wc_dev,
                  void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* The same for real symmetric P (inversion-symmetric systems, e.g. the GW_R32 polarization;
 * Sec. II: with inversion symmetry the basis and the wave functions can be chosen real): the
 * Cholesky factor and the inverse are real (a quarter of the FP64 work), the imaginary parts of
 * P_dev are not read (taken as zero), W^c is written with zero imaginary parts. Same layouts
 * and errors as gw_screened_w. Workspace: gw_screened_w_real_workspace() bytes, per system
 * 8 (2 N_b^2 + 1024 ceil(N_b / 32)) bytes rounded up to 256. */
size_t gw_screened_w_real_workspace(int nq, const int* nb_host, int nw);
int gw_screened_w_real(int nq, const int* nb_host, int nw, const double* const* v_dev,
                       const double* const* P_dev, double* const* Wc_dev,
                       void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* Variant of gw_screened_w that allocates nothing, for callers that cannot allocate
 * device memory when they call the library: for example a host application that has
 * already handed all device memory to its own pool, or a latency-critical loop in which a
 * cudaMalloc (which may synchronise the device and can fail under memory pressure) is
 * not acceptable. The paper has no counterpart to this entry point.
 *
 * One q at a time: v_dev [nb] double, P_dev [nw][nb][nb] complex128 (Hermitian NSD),
 * Wc_dev [nw][nb][nb] complex128 output (may alias P_dev). The scratch lives in a
 * library-owned static device array of GW_NOALLOC_SCRATCH_BYTES on every device that
 * loads the library (held until the process exits). Each (q, frequency) system needs
 * 16 * nb * (nb + 32) bytes; the nw systems are processed in batches that fit, one after
 * another on `stream`. nb whose single system does not fit (nb > 1008) gives GW_EINVAL;
 * nothing is allocated or freed.
 *
 * The first call on a device looks up the device address of the array (with that device
 * current); make that first call before any stream capture. All calls share the array and
 * it keeps the last call's contents (nothing in it needs to start at zero); calls that
 * overlap on the GPU (other streams, other host threads) race on it and must be ordered by
 * the caller. Errors are reported as for gw_screened_w. */
#define GW_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int gw_screened_w_noalloc(int nb, int nw, const double* v_dev, const double* P_dev,
                          double* Wc_dev, gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a5. Pair coefficients of the self-energy (band-space factor of Eq. SEc_AC):
 *   c[j][p] = Re( sum_{mu,nu} conj(m_{p,mu}) W^c_{mu nu}(q, i omega_j) m_{p,nu} ),
 * p = (state n, band n'), m_{p,mu} = <E_mu phi_n | phi_n'>. Real and <= 0.
 *   npair_host[nq], nb_host[nq]; Msig_dev[q] [npair_q][N_b] complex (m_dtype);
 *   Wc_dev[q] [nw][N_b][N_b] complex128; c_dev[q] [nw][npair_q] double output.
 * precision as for gw_polarization. Workspace: gw_sigma_workspace(). */
int gw_sigma_pair_coeffs(int nq, const int64_t* npair_host, const int* nb_host,
                         const void* const* Msig_dev, int m_dtype, int nw,
                         const double* const* Wc_dev, double* const* c_dev,
                         int precision, void* ws_dev, size_t ws_bytes,
                         gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a6. Frequency convolution (Eq. SEc_AC and the paragraph after it):
 *   Sigma^c_s(i w_i) = -1/(2 pi) sum_q w_q sum_{p: state(p) = s}
 *                      int dw' c_p(w') / (i w_i + i w' - e_p)
 * with c_p(w') a cubic spline in lambda = w'/(1+w') through the node values
 * c[j][p] (not-a-knot at the first node, first piece extrapolated to 0, slope at the
 * last node clamped to the tail's), the tail c_N w_N^2 / w'^2 beyond the last node,
 * and each spline segment and the tail integrated analytically.
 *   wq_host[nq] BZ weights; c_dev[q] [nw][npair_q] double;
 *   pair_state_dev[q] [npair_q] int in [0, nsig); eps_dev[q] [npair_q] double != 0;
 *   omega_host [nw] (ascending, > 0); omega_out_host [nw_out] (any real values);
 *   sigma_dev [nsig][nw_out] complex128 output (overwritten).
 * The closed-form integrals depend only on (e_p, omega_i) and the spline is linear in the node
 * values, so pairs with the same energy (bit-identical e_p) share the weights T_ij(e_p): they
 * are computed once per distinct energy of a q point (found by a hash of the energies in the
 * workspace) and applied to every such pair.
 * Workspace: gw_sigma_convolve_workspace() bytes.
 * e_p == 0 is reported by gw_check as GW_EINVAL. */
size_t gw_sigma_convolve_workspace(int nq, const int64_t* npair_host);
int gw_sigma_convolve(int nq, const double* wq_host, const int64_t* npair_host,
                      int nw, const double* omega_host, const double* const* c_dev,
                      const int* const* pair_state_dev, const double* const* eps_dev,
                      int nw_out, const double* omega_out_host, int nsig,
                      double* sigma_dev, void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* Extrapolar correction of Sigma^c (Sec. V, band convergence, with the full W^c rather than a
 * plasmon-pole model): the partner bands n' > N' of every state s sit at e_bar_q, so they act
 * as one extra pair per (q, s) with energy e_bar_q and coefficient
 *   cbar_{q,j,s} = sum_IJ W^c_IJ(q, i omega_j) S^{q,s}_IJ - sum_{p: state(p) = s} c_{q,j,p},
 * S^{q,s}_IJ = <phi_s| conj(M_I) M_J |phi_s> (the full-band sum of conj(m_I) m_J over the
 * partners of s at k0 + q), which is convolved over frequency by the a6 rule and ADDED to
 * sigma_dev. Per q: S_dev[q] [nsig][N_b][N_b] complex128 (Hermitian), Wc_dev[q]
 * [nw][N_b][N_b] complex128, c_dev[q] [nw][npair_q] the kept pairs' coefficients
 * (gw_sigma_pair_coeffs), pair_state_dev[q] [npair_q], ebar_host[q] > 0.
 * sigma_dev [nsig][nw_out] complex128 (accumulated); cbar_dev [nq][nw][nsig] double output or
 * NULL. FP64. Workspace: gw_sigma_extrapolar_workspace(). */
size_t gw_sigma_extrapolar_workspace(int nq, int nw, int nsig);
int gw_sigma_extrapolar(int nq, const double* wq_host, const int* nb_host, int nsig,
                        const double* const* S_dev, int nw, const double* omega_host,
                        const double* const* Wc_dev, const int64_t* npair_host,
                        const int* const* pair_state_dev, const double* const* c_dev,
                        const double* ebar_host, int nw_out, const double* omega_out_host,
                        double* sigma_dev, double* cbar_dev, void* ws_dev, size_t ws_bytes,
                        gw_stream_t stream);

/* a5 + a6 in one call (the Sigma^c step of the hot path). */
size_t gw_sigma_workspace(int nq, const int64_t* npair_host, const int* nb_host, int nw,
                          int precision);
int gw_sigma_c(int nq, const double* wq_host, const int64_t* npair_host,
               const int* nb_host, const void* const* Msig_dev, int m_dtype,
               const int* const* pair_state_dev, const double* const* eps_dev,
               int nw, const double* omega_host, const double* const* Wc_dev,
               int nw_out, const double* omega_out_host, int nsig, double* sigma_dev,
               int precision, void* ws_dev, size_t ws_bytes, gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a4. q = Gamma head and wings (Sec. III.D, Eqs. polar_Gamma and screen_Gamma and the
 * expressions after them; Eq. correlation_div). FP64.
 *   Paug_dev [nw][nb+3][nb+3] complex128: the polarization (gw_polarization, FP64 or
 *     split precision) of the augmented projections [p | M], where the first three columns
 *     p_t hold the linear-in-k coefficients of the projection onto the divergent Coulomb
 *     eigenfunction (k.p input), so that H = Paug[:3,:3], s_nu = Paug[:3, 3+nu],
 *     P~ = Paug[3:,3:];
 *   v_dev [nb] the Coulomb eigenvalues of the body.
 * Writes, per frequency: Wc_dev [nw][nb][nb] the body W~^c plus the l = 0 average of the
 * rank-one term of Eq. screen_Gamma; head_dev [nw] K^c_00 = sqrt(4 pi) <4 pi / e^T L e> -
 * (4 pi)^(3/2) (sphere average); L_dev [nw][3][3] complex128 and u_dev [nw][nb][3]
 * complex128 (u_nu = sum_mu s_mu W~_mu,nu), both optional (NULL).
 * The head and wings follow the exact block inverse of the full problem:
 *   W_11 = 4 pi / (k^2 e^T L e), W_1nu = 4 pi e^T u_nu / (k e^T L e),
 *   L = 1 - 4 pi H - 4 pi sum_nu u_nu s_nu^H.
 * A direction with e^T L e <= 0 is reported by gw_check as GW_EINVAL. */
size_t gw_gamma_workspace(int nb, int nw);
int gw_gamma_screened_w(int nb, int nw, const double* v_dev, const double* Paug_dev,
                        double* Wc_dev, double* head_dev, double* L_dev, double* u_dev,
                        void* ws_dev, size_t ws_bytes, gw_stream_t stream);
/* BZ constant (V / 8 pi^3) int_BZ d^3k / k^2 - sum_{k != 0} 1/k^2 of a simple-cubic lattice
 * (lattice constant a, n x n x n k mesh, V = (n a)^3) in the erf form of Sec. III.D with
 * exp(-beta q0^2) = beta. The lattice sum runs on the device; the result is returned to
 * out_host, so this call synchronizes the stream. */
size_t gw_bz_constant_workspace(void);
int gw_bz_constant_sc(double a, int n, double beta, double* out_host, void* ws_dev,
                      size_t ws_bytes, gw_stream_t stream);
/* Eq. correlation_div: adds -C / (4 pi^(3/2) V) int dw' K^c_00(w') / (i w + i w' - e_s) to
 * sigma_dev [nsig][nw_out] (complex128) for each state s (energy eps_state_dev[s] != 0),
 * the frequency integral by the a6 spline-in-lambda and tail rule on the nodes omega_host. */
size_t gw_sigma_div_workspace(int nw, int nsig);
int gw_sigma_div(int nw, const double* omega_host, const double* head_dev, double cbz,
                 double volume, int nsig, const double* eps_state_dev, int nw_out,
                 const double* omega_out_host, double* sigma_dev, void* ws_dev, size_t ws_bytes,
                 gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * Exchange self-energy (Eq. HFterm_MB in the Coulomb eigenbasis, Sec. III.C, plus the
 * divergent term of Eq. exchange_div in its erf form, Sec. III.D). FP64:
 *   Sigma_x[s] = - sum_q w_q sum_{p: state(p) = s, eps_p < 0} sum_mu v_mu |Msig_p,mu|^2
 *                - f_s (4 pi / volume) cbz,   f_s = 1 if eps_state[s] < 0, else 0.
 *   Msig_dev[q] [npair_q][nb_q] complex (m_dtype), pair_state_dev[q] [npair_q] in [0, nsig),
 *   eps_dev[q] [npair_q] energies of the partner bands n' (occupied when negative),
 *   v_dev[q] [nb_q] Coulomb eigenvalues, eps_state_dev [nsig], cbz the BZ constant
 *   (gw_bz_constant_sc), volume the crystal volume; sigma_x_dev [nsig] double output
 *   (overwritten). A pair state outside [0, nsig) is reported by gw_check as GW_EINVAL. */
int gw_sigma_x(int nq, const double* wq_host, const int64_t* npair_host, const int* nb_host,
               const void* const* Msig_dev, int m_dtype, const int* const* pair_state_dev,
               const double* const* eps_dev, const double* const* v_dev, int nsig,
               const double* eps_state_dev, double cbz, double volume, double* sigma_x_dev,
               gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * a7. Analytic continuation (Eq. modelf): fit f(z) = sum_p a_p / (z - w_p) to each
 * curve Sigma(i omega_j) by FP64 Levenberg-Marquardt (Marquardt's diagonal
 * scaling; cost 1/2 sum_j |f(i omega_j) - Sigma_j|^2).
 *   sigma_dev [ncurve][nw] complex128; sign_dev [ncurve] double (sign of the state
 *   energy, picks the default start w_p = s (0.5, 2, 5, 10, 20)_p - 0.1 i s) or NULL
 *   (+1); npole in [1, 5].
 *   method GW_FIT_PLAIN: default start, residues by linear least squares.
 *   method GW_FIT_MLP: start proposed by the network (npole = 2, nw = 24,
 *     mlp_dev = packed FP32 weights, see gw_mlp_param_count); the fit from the
 *     default start is also run and the lower-cost result is kept (iters and status
 *     are those of the kept fit).
 *   method GW_FIT_MLP_ONLY: the fit from the network's start alone (for measuring
 *     what the learned start gains over the default one).
 *   params_dev [ncurve][npole][4] double output (Re a, Im a, Re w, Im w);
 *   cost_dev [ncurve], iters_dev [ncurve], status_dev [ncurve] outputs
 *   (status 0 converged, 1 iteration limit, 2 damping overflow). */
int gw_continue(int ncurve, int nw, const double* omega_host, const double* sigma_dev,
                const double* sign_dev, int npole, int method, const float* mlp_dev,
                double* params_dev, double* cost_dev, int* iters_dev, int* status_dev,
                gw_stream_t stream);

/* Quasiparticle energies (Eq. quasipart_corr with the continued Sigma^c of Eq. modelf), FP64:
 * E = eps + Sigma_x + Re f(E) - v_xc by Newton's method from E = eps (|dE| <= 1e-14 max(1,|E|),
 * at most 100 steps), f(E) = sum_p a_p / (E - w_p) (the real part is the same for the conjugated
 * form that Eq. modelf prescribes for Re w < 0).
 *   params_dev [n][npole][4] (Re a, Im a, Re w, Im w) as written by gw_continue; eps_dev,
 *   sigx_dev, vxc_dev [n]; outputs E_dev [n], Z_dev [n] = 1 / (1 - Re f'(E)) (or NULL),
 *   status_dev [n] (0 converged, 1 step limit; or NULL). */
int gw_qp_solve(int n, int npole, const double* params_dev, const double* eps_dev,
                const double* sigx_dev, const double* vxc_dev, double* E_dev, double* Z_dev,
                int* status_dev, gw_stream_t stream);

/* Learned initialiser: MLP 48 -> 128 -> 128 -> 8 (SiLU), input the curve on 24 nodes
 * scaled by s = max |Sigma_j|, output (Re a/s, Im a/s, Re w, Im w) for 2 poles.
 * Packed FP32 parameter layout: W1[128][48], b1[128], W2[128][128], b2[128],
 * W3[8][128], b3[8]. */
int gw_mlp_param_count(void);
/* Inference forward pass: input, weights, biases and hidden activations rounded to BF16
 * (round to nearest even), FP32 accumulation and SiLU; sigma_dev [n][24] complex128,
 * out_dev [n][8] float. */
int gw_mlp_forward(int n, const double* sigma_dev, const float* mlp_dev, float* out_dev,
                   gw_stream_t stream);
/* One FP32 training step on a batch: loss = mean_b (1/24) sum_j |f(i w_j) - y_j|^2/s^2.
 * Writes the batch loss to loss_dev[0] and the gradient into grad_dev (packed
 * layout); then, if lr > 0, applies one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 * step number `step` >= 1) to mlp_dev with moments m_dev, v_dev (packed layout). */
int gw_mlp_train_step(int n, const double* omega_host, const double* sigma_dev,
                      float* mlp_dev, float* grad_dev, float* m_dev, float* v_dev,
                      float lr, int step, float* loss_dev, gw_stream_t stream);

/* Diagnostic (no counterpart in the paper): one device thread waits, with a wall-time limit
 * of limit_ms (0 < limit_ms <= 1000), on an mbarrier that nothing arrives on, the same bounded
 * wait that the pipelined kernels use; on expiry it records a timeout in the status word and
 * returns. The next gw_check then returns GW_ETIMEOUT (and clears the word); the context stays
 * usable. For testing the timeout path without hanging the GPU. */
int gw_selftest_bounded_wait(double limit_ms, gw_stream_t stream);

/* Diagnostic (no counterpart in the paper): the issue rate of the split-precision HERK's
 * tcgen05.mma sequence (rounds of 12 MMAs of 128 x 128 x 16 BF16, A from TMEM, B from a
 * 64-byte-swizzled shared-memory ring, 3 commits per round) in one CTA per SM, on random
 * operands, alone or beside warps of independent FMA chains (warp w runs on SM sub-partition
 * w mod 4). variant: 0 issuer alone; 1 a branch on a shared-memory value before each round;
 * 2 three FMA warps on the issuer's sub-partition; 3 three FMA warps on the other three;
 * 4 as 2 with MMAs of 128 x 256 x 16; 5 two issuers on two sub-partitions, concurrent, three
 * FMA warps beside each. rounds: 2 .. 100000. Writes (host) the average SM cycles per
 * 128 x 128 x 16 MMA (64 = the tensor pipe's rate) and synchronises the stream. Allocates
 * and frees 16 bytes of device memory. Errors: GW_EINVAL, GW_ECUDA; a bounded wait that
 * expired is reported by gw_check as GW_ETIMEOUT. */
int gw_probe_mma_issue(int variant, int rounds, double* cycles_per_mma_host, gw_stream_t stream);

/* ---------------------------------------------------------------------------
 * Synthetic-input generator (not part of the method): fills projections with
 * complex normals (Philox4x32-10 keyed by seed, counter (element index, q, tid),
 * Box-Muller) scaled by 1/(1 + I/16), exactly as the host-side input module does,
 * so large inputs can be created on the device. out_dev [rows][nb] of m_dtype,
 * element (r, I) uses index (row0 + r) * nb + I. */
int gw_synth_projections(uint64_t seed, uint32_t tid, uint32_t q, int64_t row0,
                         int64_t rows, int nb, int m_dtype, void* out_dev,
                         gw_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GW_H */
