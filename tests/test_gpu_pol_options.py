"""Execution options of the polarization (gw_polarization_ex): K slices accumulated into one P
(P is additive over transitions), the HERK launch events, and the tuning knobs, which change
how the GPU computes Eq. polar_MB but not the result."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import polarization as OP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    import paper_1003_0316_gb300 as g
    return g


def T(a, dt=None):
    return torch.as_tensor(np.asarray(a), device="cuda:0", dtype=dt)


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
def test_k_slices_accumulate_into_one_p(gw, prec):
    wl = S.tiny(nb=150, nocc=4, nunocc=60, mesh=(2, 2, 2), nw=5, seed=71)
    om = wl.omega()
    M = wl.m_full(0)
    d = wl.delta(0)
    dt = np.complex128 if prec == "fp64" else np.complex64
    Md = M.astype(dt)
    full = gw.polarization([T(Md)], [T(d)], om, wl.prefactor, prec)[0]
    P = torch.zeros_like(full)
    cuts = [0, 333, 1000, 1001, len(d)]                 # uneven slices, one of a single row
    for a, b in zip(cuts[:-1], cuts[1:]):
        gw.polarization([T(Md[a:b])], [T(d[a:b])], om, wl.prefactor, prec, out=[P],
                        options={"accumulate": True})
    gw.check()
    ref = OP.polarization(Md.astype(np.complex128), d, om, wl.prefactor)
    bound = 1e-12 if prec == "fp64" else 2e-5
    assert rel_fro(P.cpu().numpy(), ref) <= bound
    assert rel_fro(P.cpu().numpy(), full.cpu().numpy()) <= (1e-13 if prec == "fp64" else 2e-5)
    Pn = P.cpu().numpy()
    assert np.array_equal(Pn, np.conj(np.transpose(Pn, (0, 2, 1))))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("nb", [100, 200, 333])
def test_three_product_layout_against_oracle(gw, prec, nb):
    """N_b = 100, 200, 333 take the three-product layout (C = Mr^T D Mi in every tile, S =
    (Mr + Mi)^T D (Mr + Mi) in the upper tiles, combined after the launch), 333 with ragged
    blocks; one call over all three q and, for N_b = 200, K slices accumulated into one P."""
    wl = S.tiny(nb=nb, nocc=4, nunocc=50, mesh=(2, 2, 1), nw=6, seed=300 + nb)
    om = wl.omega()
    M = wl.m_full(0).astype(np.complex64)
    d = wl.delta(0)
    P = gw.polarization([T(M)], [T(d)], om, wl.prefactor, prec)[0]
    gw.check()
    ref = OP.polarization(M.astype(np.complex128), d, om, wl.prefactor)
    Pn = P.cpu().numpy()
    assert rel_fro(Pn, ref) <= 1e-5
    assert np.array_equal(Pn, np.conj(np.transpose(Pn, (0, 2, 1))))
    # the diagonal is real
    assert np.all(np.diagonal(Pn, axis1=1, axis2=2).imag == 0.0)
    if nb == 200:
        Pa = torch.zeros_like(P)
        cuts = [0, 201, 555, len(d)]
        for a, b in zip(cuts[:-1], cuts[1:]):
            gw.polarization([T(M[a:b])], [T(d[a:b])], om, wl.prefactor, prec, out=[Pa],
                            options={"accumulate": True})
        gw.check()
        Pan = Pa.cpu().numpy()
        assert rel_fro(Pan, ref) <= 1e-5
        assert np.array_equal(Pan, np.conj(np.transpose(Pan, (0, 2, 1))))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tuning_knobs_do_not_change_the_result(gw, prec):
    """b_stages, the q grouping and the overlapped preparation (one group prepared while the
    HERK of the one before runs, or serial_prep) change neither the per-tile order of the sums
    nor the roundings: the results are bit-identical; the HERK events bracket every HERK
    launch."""
    wls = [S.tiny(nb=nb, nocc=3, nunocc=nu, mesh=(2, 2, 1), nw=4, seed=90 + nb)
           for nb, nu in ((96, 30), (40, 7), (130, 55))]
    om = wls[0].omega()
    Ms = [T(w.m_full(0).astype(np.complex64)) for w in wls]
    ds = [T(w.delta(0)) for w in wls]
    ref = gw.polarization(Ms, ds, om, 0.5, prec)
    for opts in ({"b_stages": 6}, {"group_items_per_sm": 1},
                 {"group_items_per_sm": 1, "serial_prep": True},
                 {"group_items_per_sm": 64, "b_stages": 6}):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(4)]
        o = dict(opts, herk_events=evs)
        got = gw.polarization(Ms, ds, om, 0.5, prec, options=o)
        torch.cuda.synchronize()
        gw.check()
        for a, b in zip(got, ref):
            assert torch.equal(a, b), opts
        n = o["herk_launches"]
        assert 1 <= n <= 3
        for a, b in evs[:n]:
            assert a.elapsed_time(b) > 0.0


def test_fp64_waves_option(gw):
    wl = S.tiny(nb=70, nocc=3, nunocc=41, mesh=(2, 2, 2), nw=3, seed=5)
    om = wl.omega()
    M, d = wl.m_full(0), wl.delta(0)
    ref = OP.polarization(M, d, om, wl.prefactor)
    for waves in (1, 4, 16):
        P = gw.polarization([T(M)], [T(d)], om, wl.prefactor, "fp64",
                            options={"fp64_waves": waves})[0]
        gw.check()
        assert rel_fro(P.cpu().numpy(), ref) <= 1e-12
