"""Autotuner of the split-precision polarization (no counterpart in the paper: it chooses how
the GPU evaluates Eq. polar_MB, never what is computed).

For a problem shape (N_MPB, K transitions, n_omega frequencies) it times the candidate
execution options of gw_polarization_ex -- the split precision (BF16x3 / TF32x3), the
shared-memory B stages of the tensor-core kernel (4 / 6) and the q grouping (work items per
SM at which a group of q points closes) -- on a representative problem of that shape
generated on the device. A precision is accepted only if its polarization on that problem
stays within the error bound (relative Frobenius over a sampled block of basis indices)
against the library's FP64 GPU path on the same complex64 data; the fastest accepted
candidate is kept and cached per shape bucket in a JSON file, so later runs (and later
processes) reuse it without timing anything.

Shape buckets: N_MPB rounded up to a multiple of 128 (the tile edge of the kernel), K rounded
to a power of two, n_omega as is, and the device name.
"""
import json
import math
import os
import time

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1003_0316_gb300",
                             "autotune.json")
PRECISIONS = ("bf16x3", "tf32x3")
B_STAGES = (4, 6)
GROUP_ITEMS = (2, 4, 8)
REP_K = 262144          # transitions of the representative problem (at most the real K)
REP_Q = 4               # q points of the representative problem (the grouping matters)
SAMPLE_COLS = 24        # basis indices of the sampled error block


def bucket(nb, K, nw, device_name=""):
    """Cache key of a shape: N_MPB up to a multiple of 128, K to a power of two."""
    nbb = 128 * max(1, math.ceil(nb / 128))
    kb = 1 << max(0, int(round(math.log2(max(1, K)))))
    return f"{device_name}|nb{nbb}|K{kb}|nw{nw}"


def load_cache(path):
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(precisions=PRECISIONS):
    return [{"precision": p, "b_stages": b, "group_items_per_sm": g}
            for p in precisions for b in B_STAGES for g in GROUP_ITEMS]


def select(results, bound):
    """The fastest candidate whose precision met the bound. results: list of dicts with
    "precision", "b_stages", "group_items_per_sm", "ms" and "err" (the error of its precision).
    Returns the chosen entry, or None if no precision met the bound."""
    ok = [r for r in results if r["err"] is not None and r["err"] <= bound and r["ms"] > 0]
    if not ok:
        return None
    return min(ok, key=lambda r: (r["ms"], r["precision"] != "tf32x3", r["b_stages"],
                                  r["group_items_per_sm"]))


def tune(nb, K, nw, precisions=PRECISIONS, bound=1e-6, cache_path=None, measure=None,
         device_name=None, force=False):
    """Options for gw_polarization_ex at this shape: a dict with "precision", "b_stages",
    "group_items_per_sm" (plus the measured "ms" and "err"), from the cache if present.
    measure(candidate, nb, K, nw) -> (ms, err) may be given (tests); by default the
    representative problem is timed on the current CUDA device."""
    if device_name is None:
        device_name = _device_name()
    cache_path = cache_path or DEFAULT_CACHE
    key = bucket(nb, K, nw, device_name) + "|" + ",".join(precisions) + f"|{bound:g}"
    cache = load_cache(cache_path)
    if not force and key in cache:
        return dict(cache[key], cached=True)
    measure = measure or _measure_on_device
    errs = {}
    results = []
    for c in candidates(precisions):
        ms, err = measure(c, nb, K, nw)
        errs.setdefault(c["precision"], err)
        results.append(dict(c, ms=ms, err=errs[c["precision"]]))
    best = select(results, bound)
    if best is None:
        raise RuntimeError(f"no split precision meets the bound {bound:g} at N_b={nb}, K={K}")
    entry = {"precision": best["precision"], "b_stages": best["b_stages"],
             "group_items_per_sm": best["group_items_per_sm"], "ms": best["ms"],
             "err": best["err"], "bound": bound, "when": time.strftime("%Y-%m-%dT%H:%M:%S"),
             "tried": [{k: r[k] for k in ("precision", "b_stages", "group_items_per_sm", "ms", "err")}
                       for r in results]}
    cache[key] = entry
    save_cache(cache_path, cache)
    return dict(entry, cached=False)


def options_of(entry, **extra):
    """The gw_polarization_ex options dict of a tuned entry."""
    d = {"b_stages": entry["b_stages"], "group_items_per_sm": entry["group_items_per_sm"]}
    d.update(extra)
    return d


def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


_rep_state = {}


def _measure_on_device(c, nb, K, nw):
    """Time candidate c on REP_Q q points of N_b = nb with K_rep / REP_Q transitions each
    (projections and energies generated on the device), and the error of its precision on a
    sampled block against the FP64 path (computed once per shape)."""
    import torch
    import paper_1003_0316_gb300 as gw
    dev = torch.device("cuda", torch.cuda.current_device())
    k_rep = max(REP_Q, min(K, REP_K))
    kq = k_rep // REP_Q
    skey = (nb, kq, nw)
    st = _rep_state.get(skey)
    if st is None:
        _rep_state.clear()
        g = torch.Generator(device="cpu").manual_seed(nb * 7919 + kq)
        # complex normal projections (the library's counter-based generator, tensor id 3)
        Ms = [gw.synth_projections(0x5eed + q, 3, q, 0, kq, nb, dtype=torch.complex64)
              for q in range(REP_Q)]
        ds = [(0.05 + 2.4 * torch.rand(kq, generator=g, dtype=torch.float64)).to(dev)
              for _ in range(REP_Q)]
        # nw imaginary frequencies spread over [0, 50] Ha like the method's mesh
        om = [math.tan((j + 0.5) / nw * math.atan(50.0)) for j in range(nw)]
        cols = torch.linspace(0, nb - 1, min(SAMPLE_COLS, nb)).round().long().unique().to(dev)
        Mc = Ms[0][:, cols].to(torch.complex128).contiguous()
        ref = gw.polarization([Mc], [ds[0]], om, 1.0, "fp64")[0]
        st = {"Ms": Ms, "ds": ds, "om": om, "cols": cols, "ref": ref, "err": {}}
        _rep_state[skey] = st
    opts = {"b_stages": c["b_stages"], "group_items_per_sm": c["group_items_per_sm"]}
    Ks = [m.shape[0] for m in st["Ms"]]
    ws = torch.empty(max(1, gw.polarization_workspace_ex(Ks, [nb] * REP_Q, nw, c["precision"], opts)),
                     dtype=torch.uint8, device=dev)
    out = [torch.empty((nw, nb, nb), dtype=torch.complex128, device=dev) for _ in range(REP_Q)]
    gw.polarization(st["Ms"], st["ds"], st["om"], 1.0, c["precision"], out=out, ws=ws, options=opts)
    gw.check()
    if c["precision"] not in st["err"]:
        cols = st["cols"]
        got = out[0][:, cols][:, :, cols]
        st["err"][c["precision"]] = float(torch.linalg.vector_norm(got - st["ref"]) /
                                          torch.linalg.vector_norm(st["ref"]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        gw.polarization(st["Ms"], st["ds"], st["om"], 1.0, c["precision"], out=out, ws=ws,
                        options=opts)
    e1.record()
    torch.cuda.synchronize()
    gw.check()
    return e0.elapsed_time(e1) / 2, st["err"][c["precision"]]
