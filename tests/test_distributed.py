"""The multi-GPU path's host logic on CPU ranks (gloo, world size 2): each rank takes its
block of q points, computes its partial Sigma^c (the oracle stands in for the GPU
path), and the one exchange (a sum over ranks) reproduces the single-process result."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_distributed():
    # by path: the package's __init__ loads the CUDA library, which these CPU tests avoid
    spec = importlib.util.spec_from_file_location(
        "gw_distributed", os.path.join(ROOT, "paper_1003_0316_gb300", "distributed.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sigma_of(wl):
    from oracle import polarization as OP, screening as OS, selfenergy as OE
    om = wl.omega()
    cs, ps, es = [], [], []
    for i in range(wl.nq):
        P = OP.polarization(wl.m_full(i), wl.delta(i), om, wl.prefactor)
        W = OS.screened_wc_all(P, wl.v(i))
        cs.append(OE.pair_coefficients(wl.msig_rows(i), W))
        p, e = wl.sigma_pairs(i)
        ps.append(p)
        es.append(e)
    return OE.sigma_c(om, om, list(wl.wq), cs, ps, es, len(wl.sigma_states()))


def _workload():
    import synth_inputs as S
    return S.tiny(nb=10, nocc=2, nunocc=4, mesh=(2, 2, 1), nw=6, seed=77, qs=(0, 1, 2, 3))


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    D = _load_distributed()
    wl = _workload()
    lo, hi = D.shard(wl.nq, rank, world)
    part = torch.as_tensor(_sigma_of(wl.subset(range(lo, hi))))
    D.allreduce_sum_(part)
    np.save(os.path.join(out_dir, f"sigma_{rank}.npy"), part.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_covers_every_unit_once():
    D = _load_distributed()
    for n in (1, 7, 8, 64):
        for world in (1, 2, 3, 8):
            blocks = [D.shard(n, r, world) for r in range(world)]
            covered = [i for lo, hi in blocks for i in range(lo, hi)]
            assert covered == list(range(n))


def test_two_rank_sigma_matches_single_process(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    full = _sigma_of(_workload())
    for r in range(world):
        got = np.load(tmp_path / f"sigma_{r}.npy")
        assert np.allclose(got, full, rtol=1e-12, atol=1e-13 * np.abs(full).max())


def test_bench_launches_its_own_ranks():
    """`bench.py --gpus 2` without a torchrun environment starts two ranks itself (gloo for the
    reference arm, on the CPU) and rank 0 alone prints one line with n_gpus = 2."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    env["OMP_NUM_THREADS"] = "1"
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0", "--oracle-kpoints", "1"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["config"]["workload"].startswith("nk64_16q")
