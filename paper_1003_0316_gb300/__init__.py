"""Python binding of libgw (the GB300 GW hot path).

Argument marshalling only: every step runs in the CUDA kernels of libgw.so, which
is built in-tree by ``paper_1003_0316_gb300._build``. Tensors are torch CUDA
tensors (complex128 / complex64 / float64 / int32) on the current device; the
calls enqueue on torch's current stream. There is no CPU fallback: importing this
package without the compiled library raises ImportError.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# GW_LIBRARY=prof selects the profiling build (HERK wait counters, built with --prof)
_VARIANT = os.environ.get("GW_LIBRARY", "")
if _VARIANT not in ("", "prof"):
    raise ImportError(f"GW_LIBRARY={_VARIANT!r}: only 'prof' (or unset) is known")
_LIB_PATH = os.path.join(_PKG, "libgw_prof.so" if _VARIANT == "prof" else "libgw.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built; run `python paper_1003_0316_gb300/_build.py"
                      f"{' --prof' if _VARIANT else ''}`")
_lib = ctypes.CDLL(_LIB_PATH)

GW_OK, GW_EINVAL, GW_EWORKSPACE, GW_ECUDA, GW_ENONFINITE, GW_ENOTHPD, GW_ETIMEOUT, \
    GW_ENOCONV, GW_EUNSUPPORTED = range(9)
GW_C128, GW_C64, GW_R32 = 0, 1, 2
GW_FP64, GW_TF32X3, GW_BF16X3 = 0, 1, 2
GW_FIT_PLAIN, GW_FIT_MLP, GW_FIT_MLP_ONLY = 0, 1, 2
FIT_METHODS = {"plain": GW_FIT_PLAIN, "mlp": GW_FIT_MLP, "mlp_only": GW_FIT_MLP_ONLY}
PRECISIONS = {"fp64": GW_FP64, "tf32x3": GW_TF32X3, "bf16x3": GW_BF16X3}
MAX_NW = 64
SIGMA_MIXED = True   # the pair coefficients have tensor-core (split precision) paths

_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_f64 = ctypes.c_double
_f32 = ctypes.c_float
_sz = ctypes.c_size_t
_P = ctypes.POINTER


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("gw_version", _i32)
_sig("gw_last_error", ctypes.c_char_p)
_sig("gw_check", _i32, _vp)
_sig("gw_make_delta", _i32, _i32, _i32, _i32, _vp, _i32, _vp, _i32, _vp, _vp, _vp)
_sig("gw_transition_weights", _i32, _i64, _vp, _vp, _f64, _i32, _P(_f64), _vp, _vp)
_sig("gw_polarization_workspace", _sz, _i32, _P(_i64), _P(_i32), _i32, _i32)
_sig("gw_polarization", _i32, _i32, _P(_i64), _P(_i32), _P(_vp), _i32, _P(_vp), _P(_vp), _f64,
     _i32, _P(_f64), _P(_vp), _i32, _vp, _sz, _vp)
class PolOptions(ctypes.Structure):
    """gw_pol_options (include/gw.h)."""
    _fields_ = [("accumulate", _i32), ("group_items_per_sm", _i32), ("b_stages", _i32),
                ("fp64_waves", _i32), ("herk_events", _P(_vp)), ("n_herk_events", _i32),
                ("herk_launches_out", _P(_i32)), ("serial_prep", _i32),
                ("input_events", _P(_vp))]


_sig("gw_polarization_workspace_ex", _sz, _i32, _P(_i64), _P(_i32), _i32, _i32, _P(PolOptions))
_sig("gw_polarization_ex", _i32, _i32, _P(_i64), _P(_i32), _P(_vp), _i32, _P(_vp), _P(_vp), _f64,
     _i32, _P(_f64), _P(_vp), _i32, _P(PolOptions), _vp, _sz, _vp)
_sig("gw_polarization_extrapolar", _i32, _i32, _P(_i64), _P(_i32), _P(_vp), _i32, _P(_vp), _P(_vp),
     _P(_vp), _P(_i64), _P(_vp), _P(_vp), _P(_vp), _f64, _i32, _P(_f64), _P(_vp), _i32, _vp, _sz,
     _vp)
_sig("gw_sigma_extrapolar_workspace", _sz, _i32, _i32, _i32)
_sig("gw_sigma_extrapolar", _i32, _i32, _P(_f64), _P(_i32), _i32, _P(_vp), _i32, _P(_f64),
     _P(_vp), _P(_i64), _P(_vp), _P(_vp), _P(_f64), _i32, _P(_f64), _vp, _vp, _vp, _sz, _vp)
_sig("gw_screened_w_workspace", _sz, _i32, _P(_i32), _i32)
_sig("gw_screened_w", _i32, _i32, _P(_i32), _i32, _P(_vp), _P(_vp), _P(_vp), _vp, _sz, _vp)
_sig("gw_screened_w_noalloc", _i32, _i32, _i32, _vp, _vp, _vp, _vp)
_sig("gw_screened_w_real_workspace", _sz, _i32, _P(_i32), _i32)
_sig("gw_screened_w_real", _i32, _i32, _P(_i32), _i32, _P(_vp), _P(_vp), _P(_vp), _vp, _sz, _vp)
_sig("gw_sigma_pair_coeffs", _i32, _i32, _P(_i64), _P(_i32), _P(_vp), _i32, _i32, _P(_vp),
     _P(_vp), _i32, _vp, _sz, _vp)
_sig("gw_sigma_convolve_workspace", _sz, _i32, _P(_i64))
_sig("gw_sigma_convolve", _i32, _i32, _P(_f64), _P(_i64), _i32, _P(_f64), _P(_vp), _P(_vp),
     _P(_vp), _i32, _P(_f64), _i32, _vp, _vp, _sz, _vp)
_sig("gw_sigma_workspace", _sz, _i32, _P(_i64), _P(_i32), _i32, _i32)
_sig("gw_sigma_c", _i32, _i32, _P(_f64), _P(_i64), _P(_i32), _P(_vp), _i32, _P(_vp), _P(_vp),
     _i32, _P(_f64), _P(_vp), _i32, _P(_f64), _i32, _vp, _i32, _vp, _sz, _vp)
_sig("gw_continue", _i32, _i32, _i32, _P(_f64), _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp,
     _vp)
_sig("gw_mlp_param_count", _i32)
_sig("gw_mlp_forward", _i32, _i32, _vp, _vp, _vp, _vp)
_sig("gw_mlp_train_step", _i32, _i32, _P(_f64), _vp, _vp, _vp, _vp, _vp, _f32, _i32, _vp, _vp)
_sig("gw_gamma_workspace", _sz, _i32, _i32)
_sig("gw_gamma_screened_w", _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp)
_sig("gw_bz_constant_workspace", _sz)
_sig("gw_bz_constant_sc", _i32, _f64, _i32, _f64, _P(_f64), _vp, _sz, _vp)
_sig("gw_sigma_div_workspace", _sz, _i32, _i32)
_sig("gw_sigma_div", _i32, _i32, _P(_f64), _vp, _f64, _f64, _i32, _vp, _i32, _P(_f64), _vp, _vp,
     _sz, _vp)
_sig("gw_sigma_x", _i32, _i32, _P(_f64), _P(_i64), _P(_i32), _P(_vp), _i32, _P(_vp), _P(_vp), _P(_vp),
     _i32, _vp, _f64, _f64, _vp, _vp)
_sig("gw_plan_waves", _i32, _i32, _P(_i64), _P(_i32), _i32, _i32, _sz, _P(_i32), _P(_i32))
_sig("gw_selftest_bounded_wait", _i32, _f64, _vp)
_sig("gw_qp_solve", _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("gw_synth_projections", _i32, _u64, _u32, _u32, _i64, _i64, _i32, _i32, _vp, _vp)
_sig("gw_herk_wait_profile", _i32, _P(ctypes.c_ulonglong), _i32, _i32)
_sig("gw_probe_mma_issue", _i32, _i32, _i32, _P(_f64), _vp)


class GWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libgw error {code}: {msg}")
        self.code = code


def _raise(rc):
    if rc != GW_OK:
        raise GWError(rc, _lib.gw_last_error().decode())


def lib_path():
    return _LIB_PATH


def version():
    return _lib.gw_version()


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


def _arr(ctype, vals):
    vals = list(vals)
    return (ctype * len(vals))(*vals)


def _ptrs(ts):
    return (_vp * len(ts))(*[(t.data_ptr() if t is not None else None) for t in ts])


def _om(omega):
    om = [float(x) for x in (omega.tolist() if hasattr(omega, "tolist") else omega)]
    return _arr(_f64, om), len(om)


def _ws(nbytes, device):
    if nbytes == 0:
        return None, _vp(None), 0
    buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
    return buf, _vp(buf.data_ptr()), int(nbytes)


def selftest_bounded_wait(limit_ms=5.0):
    """Launch a wait that nothing ends; the next check() raises GW_ETIMEOUT."""
    _raise(_lib.gw_selftest_bounded_wait(float(limit_ms), _stream()))


def check(stream=None):
    """Synchronise the stream and raise if a device-side error was recorded."""
    _raise(_lib.gw_check(stream if stream is not None else _stream()))


def _dtype_code(t):
    if t.dtype == torch.complex128:
        return GW_C128
    if t.dtype == torch.complex64:
        return GW_C64
    if t.dtype == torch.float32:
        return GW_R32
    raise TypeError(f"projections must be complex128, complex64 or float32, got {t.dtype}")


MMA_ISSUE_VARIANTS = ("issuer alone", "branch on a shared value before each round",
                      "3 FMA warps on the issuer's sub-partition",
                      "3 FMA warps on the other sub-partitions",
                      "3 FMA warps on the issuer's sub-partition, 128 x 256 x 16 MMAs",
                      "2 concurrent issuers, 3 FMA warps beside each")


def probe_mma_issue(variant, rounds=500):
    """SM cycles per 128 x 128 x 16 MMA of the HERK's MMA sequence under load (include/gw.h,
    gw_probe_mma_issue); variant indexes MMA_ISSUE_VARIANTS."""
    out = _f64(0.0)
    _raise(_lib.gw_probe_mma_issue(int(variant), int(rounds), ctypes.byref(out), _stream()))
    return out.value


HERK_WAIT_COUNTERS = ("a_total", "a_wait_weights", "a_wait_slot", "a_rounds",
                      "mma_total", "mma_wait_b", "mma_wait_a", "mma_wait_acc", "mma_rounds",
                      "epi_total", "epi_wait_acc", "epi_drain", "epi_fold", "epi_periods",
                      "bprod_total", "bprod_wait", "wprod_total", "wprod_wait")


def herk_wait_profile(reset=True):
    """The split-precision HERK's wait counters (include/gw.h, gw_herk_wait_profile) as a dict
    of cycle sums and counts, plus the fraction of each role's time spent in each wait; only
    the profiling build (GW_LIBRARY=prof) counts, any other raises GWError(GW_EUNSUPPORTED)."""
    n = len(HERK_WAIT_COUNTERS)
    c = (ctypes.c_ulonglong * n)()
    _raise(_lib.gw_herk_wait_profile(c, n, 1 if reset else 0))
    d = dict(zip(HERK_WAIT_COUNTERS, (int(v) for v in c)))
    frac = lambda a, b: d[a] / d[b] if d[b] else None
    d["fractions"] = {
        "a_wait_weights": frac("a_wait_weights", "a_total"),
        "a_wait_slot": frac("a_wait_slot", "a_total"),
        "mma_wait_b": frac("mma_wait_b", "mma_total"),
        "mma_wait_a": frac("mma_wait_a", "mma_total"),
        "mma_wait_acc": frac("mma_wait_acc", "mma_total"),
        "epi_wait_acc": frac("epi_wait_acc", "epi_total"),
        "epi_drain": frac("epi_drain", "epi_total"),
        "epi_fold": frac("epi_fold", "epi_total"),
        "bprod_wait": frac("bprod_wait", "bprod_total"),
        "wprod_wait": frac("wprod_wait", "wprod_total")}
    d["cycles_per_drain"] = frac("epi_drain", "epi_periods")
    # two MMA issuers each take every other round: a CTA's time per round is half of this ratio
    d["cycles_per_round"] = (d["mma_total"] / (2 * d["mma_rounds"])) if d["mma_rounds"] else None
    return d


# ------------------------------------------------------- transition energies ---
def make_delta(eps_occ, eps_unocc, kq, nunocc=None, out=None):
    """Delta[t] = eps_unocc[kq[k]][n'] - eps_occ[k][n], t = (k N_occ + n) N_unocc + n'
    (float64 [N_k N_occ N_unocc]); eps_occ [N_k][N_occ], eps_unocc [N_k][>= N_unocc] float64,
    kq [N_k] int32 (mesh index of k + q), all on the device; N_unocc defaults to the width of
    eps_unocc."""
    nk, nocc = eps_occ.shape
    nu = eps_unocc.shape[1] if nunocc is None else int(nunocc)
    if out is None:
        out = torch.empty(nk * nocc * nu, dtype=torch.float64, device=eps_occ.device)
    _raise(_lib.gw_make_delta(nk, nocc, nu, eps_occ.data_ptr(), eps_occ.stride(0),
                              eps_unocc.data_ptr(), eps_unocc.stride(0), kq.data_ptr(),
                              out.data_ptr(), _stream()))
    return out


# ---------------------------------------------------------------- a1 --------
def transition_weights(delta, omega, prefactor, f=None):
    """w[j, t] = -prefactor f_t 2 Delta_t / (Delta_t^2 + omega_j^2) (float64 [nw][K])."""
    om, nw = _om(omega)
    K = delta.numel()
    w = torch.empty((nw, K), dtype=torch.float64, device=delta.device)
    _raise(_lib.gw_transition_weights(K, delta.data_ptr(), f.data_ptr() if f is not None else None,
                                      float(prefactor), nw, om, w.data_ptr(), _stream()))
    return w


# ---------------------------------------------------------------- a2 --------
def polarization_workspace(Ks, nbs, nw, precision):
    return _lib.gw_polarization_workspace(len(Ks), _arr(_i64, Ks), _arr(_i32, nbs), nw,
                                          PRECISIONS.get(precision, precision))


def _pol_options(options):
    """A PolOptions from a dict (keys as in gw_pol_options; "herk_events": a list of
    (start, end) torch.cuda.Event pairs). Returns (struct or None, keep-alive objects)."""
    if not options:
        return None, ()
    o = PolOptions()
    o.accumulate = int(bool(options.get("accumulate", False)))
    o.group_items_per_sm = int(options.get("group_items_per_sm", 0))
    o.b_stages = int(options.get("b_stages", 0))
    o.fp64_waves = int(options.get("fp64_waves", 0))
    o.serial_prep = int(bool(options.get("serial_prep", False)))
    keep = []
    ins = options.get("input_events")
    if ins:
        arr = (_vp * len(ins))(*[(e.cuda_event if e is not None else None) for e in ins])
        keep.append(arr)
        o.input_events = ctypes.cast(arr, _P(_vp))
    evs = options.get("herk_events")
    if evs:
        handles = []
        for a, b in evs:
            for e in (a, b):
                if not e.cuda_event:             # torch creates the event on its first record
                    e.record()
                handles.append(e.cuda_event)
        arr = (_vp * len(handles))(*handles)
        keep.append(arr)
        o.herk_events = ctypes.cast(arr, _P(_vp))
        o.n_herk_events = len(evs)
    cnt = _i32(0)
    keep.append(cnt)
    o.herk_launches_out = ctypes.pointer(cnt)
    return o, keep


def polarization_workspace_ex(Ks, nbs, nw, precision, options=None):
    o, _keep = _pol_options(options)
    return _lib.gw_polarization_workspace_ex(len(Ks), _arr(_i64, Ks), _arr(_i32, nbs), nw,
                                             PRECISIONS.get(precision, precision),
                                             ctypes.byref(o) if o is not None else None)


def polarization(Ms, deltas, omega, prefactor, precision="fp64", fs=None, out=None, ws=None,
                 options=None):
    """P[q] = sum_t w_tj M_tI conj(M_tJ) for each q (complex128 [nw][N_b][N_b]).
    options: None or a dict of gw_pol_options fields (accumulate, group_items_per_sm,
    b_stages, fp64_waves, serial_prep, input_events = [torch.cuda.Event per q, recorded],
    herk_events = [(start, end), ...] torch.cuda.Event pairs); after the
    call options["herk_launches"] holds the number of HERK launches."""
    prec = PRECISIONS.get(precision, precision)
    om, nw = _om(omega)
    nq = len(Ms)
    Ks = [m.shape[0] for m in Ms]
    nbs = [m.shape[1] for m in Ms]
    dev = Ms[0].device
    if out is None:
        out = [torch.empty((nw, nb, nb), dtype=torch.complex128, device=dev) for nb in nbs]
    o, keep = _pol_options(options)
    need = polarization_workspace_ex(Ks, nbs, nw, prec, options)
    if ws is None:
        wsb, wsp, wsn = _ws(need, dev)
    else:
        wsb, wsp, wsn = ws, _vp(ws.data_ptr()), ws.numel()
    fptr = _ptrs(fs) if fs is not None else None
    if o is None:
        _raise(_lib.gw_polarization(nq, _arr(_i64, Ks), _arr(_i32, nbs), _ptrs(Ms),
                                    _dtype_code(Ms[0]), _ptrs(deltas), fptr, float(prefactor), nw,
                                    om, _ptrs(out), prec, wsp, wsn, _stream()))
    else:
        _raise(_lib.gw_polarization_ex(nq, _arr(_i64, Ks), _arr(_i32, nbs), _ptrs(Ms),
                                       _dtype_code(Ms[0]), _ptrs(deltas), fptr, float(prefactor),
                                       nw, om, _ptrs(out), prec, ctypes.byref(o), wsp, wsn,
                                       _stream()))
        options["herk_launches"] = keep[-1].value
    return out


def polarization_streamed(host_Ms, host_deltas, omega, prefactor, precision="bf16x3",
                          dev_Ms=None, dev_deltas=None, out=None, ws=None, copy_stream=None):
    """P[q] for projections that live in (pinned) host memory: the host-to-device copies run on a
    copy stream, one q after the other, each followed by an event; one polarization call over all
    q waits for each q's event before reading that q's inputs (gw_pol_options.input_events), so
    the transfer of later q overlaps the tensor-core work on earlier ones. dev_Ms / dev_deltas:
    device buffers (allocated if None); ws: a workspace of polarization_workspace over all q.
    Returns the list of P (complex128 [nw][N_b][N_b])."""
    om, nw = _om(omega)
    nq = len(host_Ms)
    cur = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    cs = copy_stream if copy_stream is not None else torch.cuda.Stream(device=dev)
    if dev_Ms is None:
        dev_Ms = [torch.empty(m.shape, dtype=m.dtype, device=dev) for m in host_Ms]
    if dev_deltas is None:
        dev_deltas = [torch.empty(d.shape, dtype=d.dtype, device=dev) for d in host_deltas]
    if out is None:
        out = [torch.empty((nw, m.shape[1], m.shape[1]), dtype=torch.complex128, device=dev)
               for m in host_Ms]
    cs.wait_stream(cur)               # earlier work on the current stream is done with the buffers
    ready = []
    with torch.cuda.stream(cs):
        for q in range(nq):
            dev_Ms[q].copy_(host_Ms[q], non_blocking=True)
            dev_deltas[q].copy_(host_deltas[q], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
            ready.append(ev)
    polarization(dev_Ms, dev_deltas, omega, prefactor, precision, out=out, ws=ws,
                 options={"input_events": ready})
    for t in list(dev_Ms) + list(dev_deltas):
        t.record_stream(cs)
    return out


def polarization_extrapolar(Ms, deltas, dbars, Cs, dbar_kns, omega, prefactor, precision="fp64",
                            fs=None, f_kns=None, out=None, ws=None):
    """P^EX[q]: the kept transitions at their own energies and every band beyond the cutoff
    at e_bar (extrapolar correction, Sec. V). dbars[q] [K_q] Delta_bar of each transition's
    occupied state, Cs[q] [nkn][N_b][N_b] the completeness integrals (same element type as
    Ms), dbar_kns[q] [nkn]."""
    prec = PRECISIONS.get(precision, precision)
    om, nw = _om(omega)
    nq = len(Ms)
    Ks = [m.shape[0] for m in Ms]
    nbs = [m.shape[1] for m in Ms]
    nkns = [c.shape[0] for c in Cs]
    dev = Ms[0].device
    if out is None:
        out = [torch.empty((nw, nb, nb), dtype=torch.complex128, device=dev) for nb in nbs]
    need = polarization_workspace(Ks, nbs, nw, prec)
    if ws is None:
        wsb, wsp, wsn = _ws(need, dev)
    else:
        wsb, wsp, wsn = ws, _vp(ws.data_ptr()), ws.numel()
    fptr = _ptrs(fs) if fs is not None else None
    fkptr = _ptrs(f_kns) if f_kns is not None else None
    _raise(_lib.gw_polarization_extrapolar(
        nq, _arr(_i64, Ks), _arr(_i32, nbs), _ptrs(Ms), _dtype_code(Ms[0]), _ptrs(deltas),
        _ptrs(dbars), fptr, _arr(_i64, nkns), _ptrs(Cs), _ptrs(dbar_kns), fkptr,
        float(prefactor), nw, om, _ptrs(out), prec, wsp, wsn, _stream()))
    return out


def plan_waves(Ks, nbs, nw, precision, budget_bytes):
    """Group q points into memory waves (first-fit decreasing); returns a list of waves, each
    a list of q indices in increasing order."""
    nq = len(Ks)
    wave = (_i32 * nq)()
    nwaves = _i32(0)
    _raise(_lib.gw_plan_waves(nq, _arr(_i64, Ks), _arr(_i32, nbs), nw,
                              PRECISIONS.get(precision, precision), int(budget_bytes), wave,
                              ctypes.byref(nwaves)))
    return [[q for q in range(nq) if wave[q] == w] for w in range(nwaves.value)]


# ---------------------------------------------------------------- a3 --------
def screened_w_workspace(nbs, nw):
    return _lib.gw_screened_w_workspace(len(nbs), _arr(_i32, nbs), nw)


def screened_w(Ps, vs, out=None, ws=None, real=False):
    """W^c[q] = v^1/2 (eps^-1 - 1) v^1/2, eps = 1 - v^1/2 P v^1/2 (complex128). real=True: P is
    real symmetric (inversion symmetry), solved with real arithmetic."""
    nq = len(Ps)
    nw = Ps[0].shape[0]
    nbs = [p.shape[1] for p in Ps]
    dev = Ps[0].device
    if out is None:
        out = [torch.empty_like(p) for p in Ps]
    wsq = _lib.gw_screened_w_real_workspace if real else _lib.gw_screened_w_workspace
    need = wsq(nq, _arr(_i32, nbs), nw)
    if ws is None:
        wsb, wsp, wsn = _ws(need, dev)
    else:
        wsb, wsp, wsn = ws, _vp(ws.data_ptr()), ws.numel()
    fn = _lib.gw_screened_w_real if real else _lib.gw_screened_w
    _raise(fn(nq, _arr(_i32, nbs), nw, _ptrs(vs), _ptrs(Ps), _ptrs(out), wsp, wsn, _stream()))
    return out


NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


def screened_w_noalloc(P, v, out=None):
    """W^c for one q without any device allocation by the library (static scratch; see
    gw_screened_w_noalloc in include/gw.h). Allocates `out` here only if not given."""
    nw, nb = P.shape[0], P.shape[1]
    if out is None:
        out = torch.empty_like(P)
    _raise(_lib.gw_screened_w_noalloc(nb, nw, v.data_ptr(), P.data_ptr(), out.data_ptr(),
                                      _stream()))
    return out


# ---------------------------------------------------------------- a5/a6 -----
def sigma_workspace(npairs, nbs, nw, precision):
    return _lib.gw_sigma_workspace(len(npairs), _arr(_i64, npairs), _arr(_i32, nbs), nw,
                                   PRECISIONS.get(precision, precision))


def sigma_pair_coeffs(Msigs, Wcs, precision="fp64", out=None):
    prec = PRECISIONS.get(precision, precision)
    nq = len(Msigs)
    nw = Wcs[0].shape[0]
    npairs = [m.shape[0] for m in Msigs]
    nbs = [m.shape[1] for m in Msigs]
    dev = Msigs[0].device
    if out is None:
        out = [torch.empty((nw, n), dtype=torch.float64, device=dev) for n in npairs]
    need = sigma_workspace(npairs, nbs, nw, prec)
    wsb, wsp, wsn = _ws(need, dev)
    _raise(_lib.gw_sigma_pair_coeffs(nq, _arr(_i64, npairs), _arr(_i32, nbs), _ptrs(Msigs),
                                     _dtype_code(Msigs[0]), nw, _ptrs(Wcs), _ptrs(out), prec, wsp,
                                     wsn, _stream()))
    return out


def sigma_convolve(wq, cs, pair_states, epss, omega, omega_out, nsig, out=None):
    om, nw = _om(omega)
    omo, nwo = _om(omega_out)
    nq = len(cs)
    npairs = [c.shape[1] for c in cs]
    dev = cs[0].device
    if out is None:
        out = torch.empty((nsig, nwo), dtype=torch.complex128, device=dev)
    wsb, wsp, wsn = _ws(_lib.gw_sigma_convolve_workspace(nq, _arr(_i64, npairs)), dev)
    _raise(_lib.gw_sigma_convolve(nq, _arr(_f64, wq), _arr(_i64, npairs), nw, om, _ptrs(cs),
                                  _ptrs(pair_states), _ptrs(epss), nwo, omo, nsig, out.data_ptr(),
                                  wsp, wsn, _stream()))
    return out


def sigma_c(wq, Msigs, pair_states, epss, Wcs, omega, omega_out, nsig, precision="fp64",
            out=None, ws=None):
    prec = PRECISIONS.get(precision, precision)
    om, nw = _om(omega)
    omo, nwo = _om(omega_out)
    nq = len(Msigs)
    npairs = [m.shape[0] for m in Msigs]
    nbs = [m.shape[1] for m in Msigs]
    dev = Msigs[0].device
    if out is None:
        out = torch.empty((nsig, nwo), dtype=torch.complex128, device=dev)
    need = sigma_workspace(npairs, nbs, nw, prec)
    if ws is None:
        wsb, wsp, wsn = _ws(need, dev)
    else:
        wsb, wsp, wsn = ws, _vp(ws.data_ptr()), ws.numel()
    _raise(_lib.gw_sigma_c(nq, _arr(_f64, wq), _arr(_i64, npairs), _arr(_i32, nbs), _ptrs(Msigs),
                           _dtype_code(Msigs[0]), _ptrs(pair_states), _ptrs(epss), nw, om,
                           _ptrs(Wcs), nwo, omo, nsig, out.data_ptr(), prec, wsp, wsn, _stream()))
    return out


def sigma_extrapolar(wq, Ss, Wcs, pair_states, cs, ebars, omega, omega_out, sigma, cbar=None):
    """Adds the extrapolar correction of Sigma^c (Sec. V) to sigma [nsig][nw_out]: per (q, s)
    one extra pair at e_bar_q with coefficient sum_IJ W^c_IJ S^s_IJ minus the kept pairs'
    coefficients cs[q] [nw][npair_q]. Ss[q] [nsig][N_b][N_b] complex128. Returns (sigma,
    cbar [nq][nw][nsig])."""
    om, nw = _om(omega)
    omo, nwo = _om(omega_out)
    nq = len(Ss)
    nsig = Ss[0].shape[0]
    nbs = [x.shape[1] for x in Ss]
    npairs = [c.shape[1] for c in cs]
    dev = Ss[0].device
    if cbar is None:
        cbar = torch.empty((nq, nw, nsig), dtype=torch.float64, device=dev)
    wsb, wsp, wsn = _ws(_lib.gw_sigma_extrapolar_workspace(nq, nw, nsig), dev)
    _raise(_lib.gw_sigma_extrapolar(nq, _arr(_f64, wq), _arr(_i32, nbs), nsig, _ptrs(Ss), nw, om,
                                    _ptrs(Wcs), _arr(_i64, npairs), _ptrs(pair_states), _ptrs(cs),
                                    _arr(_f64, ebars), nwo, omo, sigma.data_ptr(), cbar.data_ptr(),
                                    wsp, wsn, _stream()))
    return sigma, cbar


# ---------------------------------------------------------- exchange --------
def sigma_x(wq, Msigs, pair_states, epss, vs, nsig, eps_state, cbz, volume, out=None):
    """Exchange self-energy per state (FP64): the regular sum over occupied partners plus
    the divergent term of occupied states."""
    nq = len(Msigs)
    dev = Msigs[0].device
    if out is None:
        out = torch.empty(nsig, dtype=torch.float64, device=dev)
    _raise(_lib.gw_sigma_x(nq, _arr(_f64, wq), _arr(_i64, [m.shape[0] for m in Msigs]),
                           _arr(_i32, [m.shape[1] for m in Msigs]), _ptrs(Msigs),
                           _dtype_code(Msigs[0]), _ptrs(pair_states), _ptrs(epss), _ptrs(vs), nsig,
                           eps_state.data_ptr(), float(cbz), float(volume), out.data_ptr(),
                           _stream()))
    return out


# ---------------------------------------------------------------- a4 --------
def gamma_screened_w(Paug, v, out=None, want_L=True, want_u=True):
    """q = Gamma: from the polarization of the augmented projections [p | M] (three k.p
    columns first), the body W~^c with the l = 0 average of the rank-one term, the head
    coefficient K^c_00 per frequency, and (optionally) L [nw][3][3] and u [nw][nb][3].
    Returns (Wc, head, L, u)."""
    nw, na, _ = Paug.shape
    nb = na - 3
    dev = Paug.device
    if out is None:
        out = torch.empty((nw, nb, nb), dtype=torch.complex128, device=dev)
    head = torch.empty(nw, dtype=torch.float64, device=dev)
    L = torch.empty((nw, 3, 3), dtype=torch.complex128, device=dev) if want_L else None
    u = torch.empty((nw, nb, 3), dtype=torch.complex128, device=dev) if want_u else None
    _buf, wsp, wsn = _ws(_lib.gw_gamma_workspace(nb, nw), dev)
    _raise(_lib.gw_gamma_screened_w(nb, nw, v.data_ptr(), Paug.data_ptr(), out.data_ptr(),
                                    head.data_ptr(), L.data_ptr() if L is not None else None,
                                    u.data_ptr() if u is not None else None, wsp, wsn,
                                    _stream()))
    return out, head, L, u


def bz_constant_sc(a, n, beta=0.005, device="cuda"):
    """BZ constant of a simple-cubic lattice in the erf form (synchronizes the stream)."""
    out = ctypes.c_double(0.0)
    _buf, wsp, wsn = _ws(_lib.gw_bz_constant_workspace(), torch.device(device))
    _raise(_lib.gw_bz_constant_sc(float(a), int(n), float(beta), ctypes.byref(out), wsp, wsn,
                                  _stream()))
    return out.value


def sigma_div(omega, head, cbz, volume, eps_state, omega_out, sigma):
    """Adds the divergent head term of Sigma^c (Eq. correlation_div) to sigma [nsig][nw_out]."""
    om, nw = _om(omega)
    omo, nwo = _om(omega_out)
    nsig = eps_state.shape[0]
    _buf, wsp, wsn = _ws(_lib.gw_sigma_div_workspace(nw, nsig), sigma.device)
    _raise(_lib.gw_sigma_div(nw, om, head.data_ptr(), float(cbz), float(volume), nsig,
                             eps_state.data_ptr(), nwo, omo, sigma.data_ptr(), wsp, wsn,
                             _stream()))
    return sigma


# ---------------------------------------------------------------- a7 --------
def continue_fit(sigma, omega, npole=2, sign=None, method="plain", mlp=None):
    """Multipole fit per curve; returns (params [n][npole][4], cost, iters, status).
    method: "plain" (default start), "mlp" (learned start, default start as fallback, the
    lower cost kept) or "mlp_only" (learned start alone); the learned start needs mlp
    (packed FP32 weights), npole = 2 and 24 frequencies."""
    om, nw = _om(omega)
    n = sigma.shape[0]
    dev = sigma.device
    params = torch.empty((n, npole, 4), dtype=torch.float64, device=dev)
    cost = torch.empty(n, dtype=torch.float64, device=dev)
    iters = torch.empty(n, dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    m = FIT_METHODS[method]
    _raise(_lib.gw_continue(n, nw, om, sigma.data_ptr(), sign.data_ptr() if sign is not None else None,
                            npole, m, mlp.data_ptr() if mlp is not None else None,
                            params.data_ptr(), cost.data_ptr(), iters.data_ptr(), status.data_ptr(),
                            _stream()))
    return params, cost, iters, status


def qp_solve(params, eps, sigx, vxc):
    """Quasiparticle energies by Newton's method on the continued self-energy; returns
    (E, Z, status) per state."""
    n, npole = params.shape[0], params.shape[1]
    dev = params.device
    E = torch.empty(n, dtype=torch.float64, device=dev)
    Z = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    _raise(_lib.gw_qp_solve(n, npole, params.data_ptr(), eps.data_ptr(), sigx.data_ptr(),
                            vxc.data_ptr(), E.data_ptr(), Z.data_ptr(), st.data_ptr(), _stream()))
    return E, Z, st


def mlp_param_count():
    return _lib.gw_mlp_param_count()


def mlp_forward(sigma, mlp, out=None):
    n = sigma.shape[0]
    if out is None:
        out = torch.empty((n, 8), dtype=torch.float32, device=sigma.device)
    _raise(_lib.gw_mlp_forward(n, sigma.data_ptr(), mlp.data_ptr(), out.data_ptr(), _stream()))
    return out


def mlp_init(seed, device="cuda"):
    """Packed FP32 parameters: Glorot-uniform weights, zero biases (host draw, seeded)."""
    g = torch.Generator().manual_seed(int(seed))
    parts = []
    for n_in, n_out in ((48, 128), (128, 128), (128, 8)):
        lim = (6.0 / (n_in + n_out)) ** 0.5
        parts.append((torch.rand((n_out, n_in), generator=g, dtype=torch.float64) * 2 - 1) * lim)
        parts.append(torch.zeros(n_out, dtype=torch.float64))
    w = torch.cat([t.reshape(-1) for t in parts]).to(torch.float32)
    assert w.numel() == mlp_param_count()
    return w.to(device)


def train_mlp(curves, omega, mlp, steps, batch=512, lr=1e-3, seed=0, log_every=0):
    """Adam training of the learned start on curves [n][24] (complex128, on the device):
    each step draws a batch (seeded permutation per epoch) and calls mlp_train_step, which
    runs forward, loss, back-propagation and the Adam update on the device. Returns the
    per-step batch losses (read back at the end)."""
    n = curves.shape[0]
    dev = curves.device
    npar = mlp_param_count()
    grad = torch.empty(npar, dtype=torch.float32, device=dev)
    m = torch.zeros(npar, dtype=torch.float32, device=dev)
    v = torch.zeros(npar, dtype=torch.float32, device=dev)
    losses = torch.empty(steps, dtype=torch.float32, device=dev)
    g = torch.Generator().manual_seed(int(seed))
    perm = torch.randperm(n, generator=g).to(dev)
    pos = 0
    for t in range(1, steps + 1):
        if pos + batch > n:
            perm = torch.randperm(n, generator=g).to(dev)
            pos = 0
        xb = curves.index_select(0, perm[pos:pos + batch]).contiguous()
        pos += batch
        mlp_train_step(xb, omega, mlp, grad, m, v, lr, t, losses[t - 1:t])
    return losses.cpu()


def mlp_train_step(sigma, omega, mlp, grad, m, v, lr, step, loss):
    om, nw = _om(omega)
    _raise(_lib.gw_mlp_train_step(sigma.shape[0], om, sigma.data_ptr(), mlp.data_ptr(),
                                  grad.data_ptr(), m.data_ptr() if m is not None else None,
                                  v.data_ptr() if v is not None else None, float(lr), int(step),
                                  loss.data_ptr(), _stream()))


# ------------------------------------------------------------ inputs --------
def synth_projections(seed, tid, q, row0, rows, nb, dtype=torch.complex64, device="cuda", out=None):
    """Device-side twin of the host input generator (Philox4x32-10 + Box-Muller)."""
    if out is None:
        out = torch.empty((rows, nb), dtype=dtype, device=device)
    code = GW_C128 if dtype == torch.complex128 else GW_C64
    _raise(_lib.gw_synth_projections(int(seed), int(tid), int(q), int(row0), int(rows), int(nb),
                                     code, out.data_ptr(), _stream()))
    return out
