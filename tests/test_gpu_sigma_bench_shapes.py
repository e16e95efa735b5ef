"""Sigma^c of the split-precision path at the mesh workload's sizes against the FP64 oracle.

One transfer momentum of the 4x4x4-mesh workload (the benchmark's shapes): N_b = 600,
K = 409,600 transitions, 16 frequencies, 16 states x 416 partner bands = 6,656 pairs. The
GPU runs the path the benchmark times: split-precision polarization, FP64 dielectric solve,
split-precision pair coefficients, FP64 convolution. The oracle runs the all-FP64 chain
(Eq. polar_MB -> Eqs. dielec_MB, screen_MB -> Eq. SEc_AC) on the same complex64-rounded
projections, drawn on the host by spawned worker processes.

Bounds of the mixed path: P relative Frobenius <= 1e-6 over the whole [16][600][600] block;
Sigma^c max |dSigma| <= 1e-5 of max |Sigma|, and <= 1e-5 Ha absolute where the pair
coefficients run in TF32x3 (the precision the benchmark uses for them). The Sigma projections
carry the workload's factor 2^-5 (a power of two: no relative rounding changes), which puts
max |Sigma^c| at about 11 Ha. BF16x3 pair coefficients (2^-17 per split operand, summed over
only 2 N_b = 1200 terms) give about 2e-5 Ha there, 2e-6 relative: the absolute bound is not
claimed for them.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import synth_inputs as S
from oracle import chain as OCH

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


@pytest.fixture(scope="module")
def pool():
    n = max(1, min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                   else (os.cpu_count() or 1)))
    with mp.get_context("spawn").Pool(n) as p:
        yield p


@pytest.fixture(scope="module")
def case(pool):
    """Host inputs of q index 1 and the oracle's chain on them (computed once)."""
    wl = S.medium_mixed()
    iq = 1
    M = S.m_rows_parallel(wl, iq, pool, dtype=np.complex64)
    d = wl.delta(iq)
    om = wl.omega()
    v = wl.v(iq)
    ps, eps = wl.sigma_pairs(iq)
    Ms = wl.msig_rows(iq).astype(np.complex64)
    nsig = len(wl.sigma_states())
    wq = wl.wq[iq]
    P, Wc, c, sig = OCH.sigma_one_q(M.astype(np.complex128), d, om, wl.prefactor, v,
                                    Ms.astype(np.complex128), ps, eps, wq, om, nsig, pool=pool)
    return dict(wl=wl, iq=iq, M=M, d=d, om=om, v=v, ps=ps, eps=eps, Ms=Ms, nsig=nsig, wq=wq,
                P=P, Wc=Wc, c=c, sig=sig)


@pytest.mark.parametrize("prec,sprec", [("bf16x3", "tf32x3"), ("bf16x3", "bf16x3"),
                                        ("tf32x3", "tf32x3")])
def test_sigma_mixed_at_bench_shapes(gw, case, prec, sprec):
    """prec: the polarization's split precision; sprec: the pair coefficients' (the benchmark
    runs BF16x3 and TF32x3)."""
    dev = torch.device("cuda:0")
    T = lambda a, dt=None: torch.as_tensor(np.asarray(a), device=dev, dtype=dt)
    om = case["om"]
    P = gw.polarization([T(case["M"])], [T(case["d"])], om, case["wl"].prefactor, prec)
    gw.check()
    eP = float(torch.linalg.vector_norm(P[0] - T(case["P"])) / np.linalg.norm(case["P"]))
    W = gw.screened_w(P, [T(case["v"])])
    c = gw.sigma_pair_coeffs([T(case["Ms"])], W, precision=sprec)[0]
    sig = gw.sigma_convolve([case["wq"]], [c], [T(case["ps"], torch.int32)], [T(case["eps"])],
                            om, om, case["nsig"])
    gw.check()
    sig = sig.cpu().numpy()
    so = case["sig"]
    abs_err = float(np.abs(sig - so).max())
    rel_err = abs_err / float(np.abs(so).max())
    cref = case["c"]
    c_err = float(np.abs(c.cpu().numpy() - cref).max() / np.abs(cref).max())
    print(f"\nP {prec}, pair coefficients {sprec}: P rel Frobenius {eP:.2e}; pair coefficients max err / max|c| {c_err:.2e}; "
          f"Sigma^c max |dSigma| {abs_err:.2e} Ha (max |Sigma| {np.abs(so).max():.3f} Ha, "
          f"relative {rel_err:.2e})")
    assert eP <= 1e-6, eP
    assert rel_err <= 1e-5, rel_err
    if sprec == "tf32x3":
        assert abs_err <= 1e-5, abs_err
