"""Correlation self-energy curves produced by the library's own pipeline: training and
evaluation data for the learned start of the analytic continuation (Eq. modelf).

One run is one seed of the 4x4x4-mesh workload (8 transfer momenta q of weight 1/8, N_MPB =
600, 16 occupied / 400 unoccupied bands, 16 imaginary frequencies): the polarization (split
precision, Eq. polar_MB), the FP64 screened interaction (Eqs. dielec_MB, screen_MB), and for
each of the 8 k0 points of the mesh with n_i in {0, 1} the Sigma^c of all 416 bands at k0
(Eq. SEc_AC; pair coefficients in TF32x3, the convolution in FP64) on the 24-node output mesh:
3,328 curves per run. Every step runs in the library's kernels. Each run is written as one
shard (curves [n][24] complex128 and the signs of the states' energies, which select the
default start of the fit) and recorded in a manifest; a run already in the manifest is
skipped, so an interrupted generation resumes where it stopped.
"""
import hashlib
import json
import os

import numpy as np

NODES = 24


def _workload(seed):
    import synth_inputs as S
    wl = S.medium_mixed()
    wl.seed = int(seed)
    wl.states = tuple(range(wl.nocc + wl.nunocc_max))          # every band at k0
    return wl


def run_curves(seed, precision="bf16x3", sigma_precision="tf32x3"):
    """Curves of one run: (curves [8 * 416][24] complex128, signs [8 * 416])."""
    import torch
    import synth_inputs as S
    import paper_1003_0316_gb300 as gw
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = _workload(seed)
    om, om_out = wl.omega(), S.omega_mesh(NODES)
    P = [torch.empty((wl.nw, nb, nb), dtype=torch.complex128, device=dev) for nb in wl.nb]
    ws = torch.empty(gw.polarization_workspace([wl.K(0)], [wl.nb[0]], wl.nw, precision),
                     dtype=torch.uint8, device=dev)
    for i in range(wl.nq):                       # one q at a time: one q's projections resident
        M = gw.synth_projections(wl.seed, S.TID_M, wl.qs[i], 0, wl.K(i), wl.nb[i],
                                 dtype=torch.complex64)
        d = gw.make_delta(torch.as_tensor(wl.eps_occ(), device=dev),
                          torch.as_tensor(wl.eps_unocc(), device=dev),
                          torch.as_tensor(wl.kplus(np.arange(wl.nk), wl.qs[i]).astype(np.int32),
                                          device=dev), nunocc=wl.nunocc[i])
        gw.polarization([M], [d], om, wl.prefactor, precision, out=[P[i]], ws=ws)
        del M
    del ws
    W = gw.screened_w(P, [torch.as_tensor(wl.v(i), device=dev) for i in range(wl.nq)], out=P)
    curves, signs = [], []
    nsig = len(wl.states)
    for k0 in wl.qs:                              # the 8 k0 points
        wl.k0 = int(k0)
        ps, eps = zip(*[wl.sigma_pairs(i) for i in range(wl.nq)])
        Ms = [gw.synth_projections(wl.seed, S.TID_MSIG, wl.msig_counter(i), 0, len(ps[i]),
                                   wl.nb[i], dtype=torch.complex64).mul_(wl.msig_scale)
              for i in range(wl.nq)]
        sig = gw.sigma_c(list(wl.wq), Ms, [torch.as_tensor(p, dtype=torch.int32, device=dev)
                                           for p in ps],
                         [torch.as_tensor(e, device=dev) for e in eps], W, om, om_out, nsig,
                         precision=sigma_precision)
        gw.check()
        curves.append(sig.cpu().numpy())
        signs.append(np.sign(wl.state_energies()))
        del Ms
    return np.concatenate(curves), np.concatenate(signs)


def _manifest_path(out_dir):
    return os.path.join(out_dir, "manifest.json")


def read_manifest(out_dir):
    try:
        with open(_manifest_path(out_dir)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"shards": []}


def generate(out_dir, seeds, **kw):
    """Runs the seeds not yet in the manifest, one shard each; returns the manifest."""
    os.makedirs(out_dir, exist_ok=True)
    man = read_manifest(out_dir)
    done = {s["seed"] for s in man["shards"]}
    for seed in seeds:
        if int(seed) in done:
            continue
        y, sg = run_curves(int(seed), **kw)
        name = f"curves_{int(seed):x}.npz"
        path = os.path.join(out_dir, name)
        np.savez(path + ".tmp.npz", curves=y, signs=sg)
        os.replace(path + ".tmp.npz", path)
        digest = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
        man["shards"].append({"seed": int(seed), "file": name, "curves": int(len(y)),
                              "nodes": NODES, "sha256_16": digest})
        tmp = _manifest_path(out_dir) + ".tmp"
        with open(tmp, "w") as f:
            json.dump(man, f, indent=1)
        os.replace(tmp, _manifest_path(out_dir))    # the shard is complete before it is listed
    return man


def load(out_dir, seeds=None):
    """(curves, signs) of the listed shards (of the given seeds, in manifest order)."""
    man = read_manifest(out_dir)
    ys, ss = [], []
    for s in man["shards"]:
        if seeds is not None and s["seed"] not in set(int(x) for x in seeds):
            continue
        with np.load(os.path.join(out_dir, s["file"])) as z:
            ys.append(z["curves"])
            ss.append(z["signs"])
    if not ys:
        return np.zeros((0, NODES), dtype=np.complex128), np.zeros(0)
    return np.concatenate(ys), np.concatenate(ss)
