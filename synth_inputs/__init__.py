"""Seeded synthetic inputs shaped like the paper's systems.

The paper's ground states (FLAPW wave functions and Kohn-Sham energies of real
crystals) are not available, so every input here is drawn from a counter-based
generator and stands in for them:

* Gamma-centred k mesh k = sum_i n_i b_i / N_i (Sec. III.D), k+q indexed on the mesh;
* occupied energies U[-0.5, 0] Ha and unoccupied energies U[0.05, 2] Ha, drawn per
  mesh point and band (energies measured from the Fermi level, Sec. II);
* projections M_{t,I} = (N(0,1) + i N(0,1)) / (1 + I/16), I = 0 .. N_b-1 (Eq. proj_MB
  shape: decaying weight for higher Coulomb eigenfunctions); the self-energy projections
  follow the same law times a workload factor (2^-5 for the mesh workloads, so that
  |Sigma^c| is of physical size);
* Coulomb eigenvalues v_I = 4 pi / (0.1 + I^(2/3)) (Eq. dielec_MB input);
* imaginary-frequency mesh omega_j = tan(theta_j), theta_j the Gauss-Legendre nodes on
  [0, arctan 50] (dense near 0, Sec. III.C);
* model self-energy curves for the analytic continuation (Sec. III.C): sums of simple
  poles shaped like the single-transition closed form of Sigma^c (positive residue, pole
  at eps' + sgn(eps') Omega just off the real axis), many poles per curve.

This module performs none of the method's arithmetic (no weights, no products, no
solves); it only lays out indices and draws numbers. Both the CPU oracle and the
CUDA path's tests read their inputs from here. Every draw is addressed by a counter
(element index, q index, tensor id) and the workload seed, so any subset of a
large tensor can be regenerated without generating the rest.
"""
from dataclasses import dataclass, field
import numpy as np

from .philox import philox4x32_10, uniform53, normal_pair, split_index

# tensor ids: the fourth Philox counter word
TID_EPS_OCC = 1
TID_EPS_UNOCC = 2
TID_M = 3
TID_MSIG = 4
TID_SIZES = 5
TID_KP = 6
TID_MISC = 7
TID_CURVES = 8

SEED_BASE = 0x10030316


def key_of(seed):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def omega_mesh(nw, omega_max=50.0):
    """Tan-mapped Gauss-Legendre nodes on [0, omega_max] (ascending, all > 0)."""
    x, _ = np.polynomial.legendre.leggauss(nw)
    theta = 0.5 * (x + 1.0) * np.arctan(omega_max)
    return np.tan(theta)


def coulomb_eigenvalues(nb):
    i = np.arange(nb, dtype=np.float64)
    return 4.0 * np.pi / (0.1 + i ** (2.0 / 3.0))


def uniforms(seed, tid, idx, q=0):
    """One U[0,1) per element index (from words 0,1 of a Philox block)."""
    k0, k1 = key_of(seed)
    lo, hi = split_index(idx)
    x0, x1, _, _ = philox4x32_10(lo, hi, q, tid, k0, k1)
    return uniform53(x0, x1)


def complex_normals(seed, tid, idx, q):
    """One complex N(0,1)+iN(0,1) per element index (one Philox block each)."""
    k0, k1 = key_of(seed)
    lo, hi = split_index(idx)
    x = philox4x32_10(lo, hi, q, tid, k0, k1)
    re, im = normal_pair(*x)
    return re + 1j * im


@dataclass
class Workload:
    """One synthetic GW problem: k mesh, q list, band counts, basis sizes, mesh."""
    name: str
    seed: int
    mesh: tuple            # (N1, N2, N3)
    qs: tuple              # mesh indices of the transfer momenta
    wq: tuple              # BZ weights of the q points (sum 1)
    nb: tuple              # N_MPB per q
    nocc: int
    nunocc: tuple          # unoccupied bands per q
    nw: int
    states: tuple = None   # band indices at k0 = Gamma that get Sigma (None: all)
    nw_out: int = None     # output mesh size of Sigma (None: nw)
    msig_scale: float = 1.0  # extra factor of the Sigma projections (a power of two)
    k0: int = 0            # mesh index of the Sigma states' k point
    extra: dict = field(default_factory=dict)

    @property
    def nk(self):
        return int(np.prod(self.mesh))

    def subset(self, idx):
        """The same problem restricted to the q points idx (BZ weights kept: a shard of a
        sum over q)."""
        idx = list(idx)
        from dataclasses import replace
        return replace(self, name=f"{self.name}_q{idx[0]}-{idx[-1]}" if idx else self.name + "_empty",
                       qs=tuple(self.qs[i] for i in idx), wq=tuple(self.wq[i] for i in idx),
                       nb=tuple(self.nb[i] for i in idx), nunocc=tuple(self.nunocc[i] for i in idx),
                       extra=dict(self.extra))

    @property
    def nq(self):
        return len(self.qs)

    @property
    def prefactor(self):
        # spin sum (factor 2) over the BZ density 1/N_k (Eq. polar_MB, Sec. II)
        return 2.0 / self.nk

    @property
    def nunocc_max(self):
        return max(self.nunocc)

    @property
    def nband(self):
        return self.nocc + self.nunocc_max

    def K(self, iq):
        return self.nk * self.nocc * self.nunocc[iq]

    def omega(self):
        return omega_mesh(self.nw)

    def omega_out(self):
        return omega_mesh(self.nw_out or self.nw)

    def v(self, iq):
        return coulomb_eigenvalues(self.nb[iq])

    # ---- k mesh -------------------------------------------------------------
    def kplus(self, k, q):
        n1, n2, n3 = self.mesh
        k = np.asarray(k)
        a, b, c = k // (n2 * n3), (k // n3) % n2, k % n3
        qa, qb, qc = q // (n2 * n3), (q // n3) % n2, q % n3
        return (((a + qa) % n1) * n2 + (b + qb) % n2) * n3 + (c + qc) % n3

    def kminus(self, k, q):
        n1, n2, n3 = self.mesh
        k = np.asarray(k)
        a, b, c = k // (n2 * n3), (k // n3) % n2, k % n3
        qa, qb, qc = q // (n2 * n3), (q // n3) % n2, q % n3
        return (((a - qa) % n1) * n2 + (b - qb) % n2) * n3 + (c - qc) % n3

    # ---- band energies ------------------------------------------------------
    def eps_occ(self):
        """[N_k][N_occ] occupied energies, U[-0.5, 0] Ha."""
        idx = np.arange(self.nk * self.nocc, dtype=np.uint64)
        return (-0.5 * uniforms(self.seed, TID_EPS_OCC, idx)).reshape(self.nk, self.nocc)

    def eps_unocc(self):
        """[N_k][max N_unocc] unoccupied energies, U[0.05, 2] Ha."""
        n = self.nunocc_max
        idx = np.arange(self.nk * n, dtype=np.uint64)
        return (0.05 + 1.95 * uniforms(self.seed, TID_EPS_UNOCC, idx)).reshape(self.nk, n)

    def eps_bands(self, k):
        """All band energies at mesh point k: occupied first, then unoccupied."""
        return np.concatenate([self.eps_occ()[k], self.eps_unocc()[k]])

    # ---- transitions t = (k, n occ, n' unocc) for transfer q ----------------
    def delta(self, iq):
        """Delta_t = eps_{n'}(k+q) - eps_n(k), t = (k * N_occ + n) * N_unocc + n'."""
        q = self.qs[iq]
        nu = self.nunocc[iq]
        eo = self.eps_occ()
        eu = self.eps_unocc()[:, :nu]
        kq = self.kplus(np.arange(self.nk), q)
        d = eu[kq][:, None, :] - eo[:, :, None]
        return d.reshape(-1).astype(np.float64)

    def m_rows(self, iq, rows=None, cols=None):
        """Projections M_{t,I} (complex128) for the given rows t and columns I."""
        nb = self.nb[iq]
        K = self.K(iq)
        rows = np.arange(K, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
        cols = np.arange(nb, dtype=np.uint64) if cols is None else np.asarray(cols, dtype=np.uint64)
        idx = rows[:, None] * np.uint64(nb) + cols[None, :]
        z = complex_normals(self.seed, TID_M, idx, self.qs[iq])
        return z / (1.0 + cols.astype(np.float64)[None, :] / 16.0)

    def m_full(self, iq):
        return self.m_rows(iq)

    # ---- self-energy pairs p = (state s at k0, band n' at k0+q) --------------
    def sigma_states(self):
        if self.states is not None:
            return np.asarray(self.states, dtype=np.int64)
        return np.arange(self.nocc + self.nunocc_max, dtype=np.int64)

    def n_pair_bands(self, iq):
        return self.nocc + self.nunocc[iq]

    def sigma_pairs(self, iq):
        """pair_state[p], eps_np[p] for p = s * (N_occ + N_unocc) + n'."""
        q = self.qs[iq]
        ns = len(self.sigma_states())
        nbnd = self.n_pair_bands(iq)
        kq = int(self.kplus(self.k0, q))
        e = np.concatenate([self.eps_occ()[kq], self.eps_unocc()[kq][: self.nunocc[iq]]])
        pair_state = np.repeat(np.arange(ns, dtype=np.int32), nbnd)
        eps_np = np.tile(e, ns)
        return pair_state, eps_np

    def msig_rows(self, iq, rows=None, cols=None):
        nb = self.nb[iq]
        npair = len(self.sigma_states()) * self.n_pair_bands(iq)
        rows = np.arange(npair, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
        cols = np.arange(nb, dtype=np.uint64) if cols is None else np.asarray(cols, dtype=np.uint64)
        idx = rows[:, None] * np.uint64(nb) + cols[None, :]
        z = complex_normals(self.seed, TID_MSIG, idx, self.msig_counter(iq))
        return z * (self.msig_scale / (1.0 + cols.astype(np.float64)[None, :] / 16.0))

    def msig_counter(self, iq):
        """Third Philox counter word of the Sigma projections: q's mesh index, plus N_k k0 for
        states at k0 != Gamma (k0 = 0 keeps the draws of a Gamma-only workload)."""
        return int(self.qs[iq]) + self.nk * int(self.k0)

    def state_energies(self):
        return self.eps_bands(self.k0)[self.sigma_states()]


def _m_block(args):
    wl, iq, r0, r1, cols, dtype = args
    return wl.m_rows(iq, rows=np.arange(r0, r1, dtype=np.uint64), cols=cols).astype(dtype)


def m_rows_parallel(wl, iq, pool, dtype=np.complex128, block=16384, cols=None, rows=None):
    """Projections M_{t,I} of q index iq (the draws of Workload.m_rows) for the rows
    range(*rows) (default: all K) and the given columns (default: all), row blocks drawn by the
    worker processes of `pool` (a multiprocessing pool made with the "spawn" start method, so
    that it is safe next to a CUDA context). Returns [rows][cols] in `dtype`."""
    r_lo, r_hi = rows if rows is not None else (0, wl.K(iq))
    if cols is not None:
        block = max(block, 16384 * 256 // max(1, len(cols)))   # about 4M draws per job
    jobs = [(wl, iq, r0, min(r_hi, r0 + block), cols, dtype) for r0 in range(r_lo, r_hi, block)]
    parts = pool.map(_m_block, jobs)
    ncol = wl.nb[iq] if cols is None else len(cols)
    return np.concatenate(parts) if parts else np.zeros((0, ncol), dtype=dtype)


# Sigma projections of the mesh workloads carry a factor 2^-5, so that the correlation
# self-energy of the synthetic states is of the size of a physical one (max |Sigma^c| about
# 11 Ha on the 4x4x4-mesh workload instead of about 10^4 Ha); a power of two changes no
# relative rounding anywhere on the path.
MSIG_SCALE_PHYSICAL = 2.0 ** -5


def _mesh_index(mesh, a, b, c):
    return (a * mesh[1] + b) * mesh[2] + c


def small_fp64():
    """N_k = 8 (2x2x2), q = Gamma, N_MPB = 64, 4 occ / 28 unocc, 8 frequencies, all 32 states."""
    return Workload(name="fp64_nk8_nb64_nocc4_nunocc28_nw8", seed=SEED_BASE + 0,
                    mesh=(2, 2, 2), qs=(0,), wq=(1.0,), nb=(64,), nocc=4, nunocc=(28,),
                    nw=8, states=None)


def _top_states(wl, n_occ_states, n_unocc_states):
    e = wl.eps_bands(wl.k0)
    occ = np.argsort(e[: wl.nocc])[::-1][:n_occ_states]
    unocc = wl.nocc + np.argsort(e[wl.nocc:])[:n_unocc_states]
    return tuple(int(x) for x in np.concatenate([np.sort(occ), np.sort(unocc)]))


def medium_mixed():
    """N_k = 64 (4x4x4), 8 q (n_i in {0,1}, weight 8/64 each), N_MPB = 600,
    16 occ / 400 unocc (K = 409,600 per q), 16 frequencies, 16 Sigma states."""
    mesh = (4, 4, 4)
    qs = tuple(_mesh_index(mesh, a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1))
    wl = Workload(name="nk64_8q_nb600_nocc16_nunocc400_nw16", seed=SEED_BASE + 1,
                  mesh=mesh, qs=qs, wq=tuple([8.0 / 64.0] * 8), nb=tuple([600] * 8),
                  nocc=16, nunocc=tuple([400] * 8), nw=16, msig_scale=MSIG_SCALE_PHYSICAL)
    wl.states = _top_states(wl, 8, 8)
    return wl


def medium_mixed_sharded(world):
    """The 4x4x4-mesh workload of medium_mixed with 8 q per rank for world ranks (weak
    scaling): the 8 points with n_i in {0,1} first, then further mesh points in index
    order; every q has weight 1 / (8 world)."""
    base = medium_mixed()
    if world == 1:
        return base
    mesh = base.mesh
    nq = 8 * int(world)
    if nq > int(np.prod(mesh)):
        raise ValueError("at most 8 ranks: the 4x4x4 mesh has 64 q points")
    rest = [q for q in range(int(np.prod(mesh))) if q not in base.qs]
    qs = tuple(base.qs) + tuple(rest[:nq - 8])
    wl = Workload(name=f"nk64_{nq}q_nb600_nocc16_nunocc400_nw16", seed=base.seed, mesh=mesh,
                  qs=qs, wq=tuple([1.0 / nq] * nq), nb=tuple([600] * nq), nocc=16,
                  nunocc=tuple([400] * nq), nw=16, msig_scale=MSIG_SCALE_PHYSICAL)
    wl.states = base.states
    return wl


def supercell():
    """Single q = Gamma, N_k = 8, N_MPB = 4096, 256 occ / 3000 unocc, 20 frequencies."""
    wl = Workload(name="nk8_1q_nb4096_nocc256_nunocc3000_nw20", seed=SEED_BASE + 2,
                  mesh=(2, 2, 2), qs=(0,), wq=(1.0,), nb=(4096,), nocc=256,
                  nunocc=(3000,), nw=20, msig_scale=MSIG_SCALE_PHYSICAL)
    wl.states = _top_states(wl, 8, 8)
    return wl


def batched_uneven():
    """64 q (full 4x4x4 mesh, weight 1/64), N_MPB ~ U[300,1500], N_unocc ~ U[200,800],
    32 occ, 16 frequencies."""
    seed = SEED_BASE + 3
    mesh = (4, 4, 4)
    nq = 64
    u = uniforms(seed, TID_SIZES, np.arange(2 * nq, dtype=np.uint64))
    nb = tuple(int(300 + np.floor(x * 1201)) for x in u[:nq])
    nu = tuple(int(200 + np.floor(x * 601)) for x in u[nq:])
    wl = Workload(name="nk64_64q_nbU300-1500_nocc32_nunoccU200-800_nw16", seed=seed,
                  mesh=mesh, qs=tuple(range(nq)), wq=tuple([1.0 / nq] * nq), nb=nb,
                  nocc=32, nunocc=nu, nw=16, msig_scale=MSIG_SCALE_PHYSICAL)
    wl.states = _top_states(wl, 8, 8)
    return wl


def tiny(nb=8, nocc=2, nunocc=3, mesh=(1, 1, 2), nw=6, seed=12345, qs=(0,), nw_out=None):
    """Small case for brute-force and invariant checks."""
    nk = int(np.prod(mesh))
    return Workload(name=f"tiny_nb{nb}", seed=seed, mesh=mesh, qs=tuple(qs),
                    wq=tuple([1.0 / len(qs)] * len(qs)), nb=tuple([nb] * len(qs)),
                    nocc=nocc, nunocc=tuple([nunocc] * len(qs)), nw=nw, nw_out=nw_out)


def sigma_curves_mesh():
    """24-node output mesh used for the analytic-continuation curves."""
    return omega_mesh(24)


CURVE_MAXPOLE = 24


def model_sigma_curves(seed, n, omega, first=0):
    """n model curves y_c(i omega_j) = sum_k r_k / (i omega_j - e_k) and state signs.

    Per curve c (counter index first + c): 4 to 24 poles; each pole k draws a band energy
    eps_k (occupied U[-0.5, 0] or unoccupied U[0.05, 2] Ha, even odds), a plasmon-like
    energy Omega_k ~ U[0.3, 1.5] Ha and a residue r_k ~ U[0.005, 0.1] Ha; the pole sits at
    e_k = eps_k + sgn(eps_k) Omega_k - 0.01 i sgn(eps_k) (the side of the real axis that a
    time-ordered self-energy has). The state sign is +1 or -1 with even odds.
    Returns (curves [n][len(omega)] complex128, sign [n])."""
    omega = np.asarray(omega, dtype=np.float64)
    c = np.arange(first, first + n, dtype=np.int64)
    per = 2 + 5 * CURVE_MAXPOLE
    base = c * per
    u = lambda k: uniforms(seed, TID_CURVES, base + k)
    npole = 4 + np.minimum((u(0) * 21).astype(np.int64), 20)
    sign = np.where(u(1) < 0.5, -1.0, 1.0)
    z = 1j * omega[None, :]
    y = np.zeros((n, len(omega)), dtype=np.complex128)
    for k in range(CURVE_MAXPOLE):
        o = 2 + 5 * k
        occ = u(o) < 0.5
        eps = np.where(occ, -0.5 * u(o + 1), 0.05 + 1.95 * u(o + 1))
        Om = 0.3 + 1.2 * u(o + 2)
        r = 0.005 + 0.095 * u(o + 3)
        sg = np.where(occ, -1.0, 1.0)
        e = eps + sg * Om - 0.01j * sg
        active = (k < npole).astype(np.float64)
        y += (active * r)[:, None] / (z - e[:, None])
    return y, sign
