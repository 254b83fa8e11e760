"""Seeded synthetic inputs for chi0(q, omega): band energies, eigenvectors, E_F, q and omega lists.

This module is the ONE piece shared by the CUDA path (through its binding), the
CPU oracle and the benchmark.  It holds none of the susceptibility arithmetic:
it only builds tight-binding (TB) Hamiltonians, diagonalises them with LAPACK,
picks E_F as a quantile of the grid eigenvalues and lays out q points.

The paper's inputs are FP-LAPW (WIEN2k) band structures of Cr and FeSe
(Sec. II, III); those cannot be produced here, so seeded TB models with the
same structure (9 d-like bands for Cr, 2 Fe x 5 d bands on a tetragonal cell
for FeSe, 40/80-band random models for the band-truncation and large runs)
stand in for them.

Conventions shared with the library and the oracle (both implement them
independently):

* k grid: ``n = (n0, n1, n2)`` cubes.  Periodic grids (TB models) have
  ``n0*n1*n2`` corners, fractional coordinate ``(i0/n0, i1/n1, i2/n2)``; open
  grids (free electron) have ``(n0+1)(n1+1)(n2+1)`` corners spanning the cube
  edge to edge.  Corner index ``c = (i0*N1 + i1)*N2 + i2`` with ``N`` the
  corner counts per axis (``i0`` slowest).
* energies ``E[c, band]`` (float64, ascending per corner), eigenvectors
  ``C[c, orbital, band]`` (complex128 or complex64).
* ``E_F`` is an input to the method; it is never solved for by the library.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 1407344400


# ----------------------------------------------------------------------------------------
# grid helpers
# ----------------------------------------------------------------------------------------
def corner_dims(n: Sequence[int], periodic: bool) -> Tuple[int, int, int]:
    return tuple(int(x) if periodic else int(x) + 1 for x in n)


def corner_index(n: Sequence[int], periodic: bool) -> np.ndarray:
    """Integer grid indices [Nc, 3] of the corners, slowest axis first."""
    N = corner_dims(n, periodic)
    g = np.stack(np.meshgrid(*[np.arange(N[d]) for d in range(3)], indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def corner_frac(n: Sequence[int], periodic: bool) -> np.ndarray:
    """Fractional coordinates [Nc, 3] of the grid corners, slowest axis first."""
    N = corner_dims(n, periodic)
    axes = [np.arange(N[d], dtype=np.float64) / n[d] for d in range(3)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


# ----------------------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------------------
@dataclass
class QPoint:
    """One q point.  Either an on-grid shift (k+q corner = corner + shift, periodic
    grids only) or explicit energies/eigenvectors at every k+q corner."""
    shift: Tuple[int, int, int] = (0, 0, 0)
    Eq: Optional[np.ndarray] = None          # [Nc, nb] float64
    Cq: Optional[np.ndarray] = None          # [Nc, norb, nb] complex
    window: Optional[Tuple[int, int]] = None  # per-q band window [lo, hi); None -> workload window
    gamma: bool = False                       # q is Gamma (or a reciprocal lattice vector)
    frac: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # q in fractional units (informational)


@dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    periodic: bool
    nb: int
    norb: int
    E: np.ndarray                     # [Nc, nb] float64
    C: Optional[np.ndarray]           # [Nc, norb, nb] complex or None (CMA only)
    ef: float
    window: Tuple[int, int]
    cma: bool
    qs: List[QPoint]
    omega: Optional[np.ndarray] = None  # dynamic frequencies, None = static
    meta: dict = field(default_factory=dict)

    @property
    def ncorner(self) -> int:
        N = corner_dims(self.n, self.periodic)
        return N[0] * N[1] * N[2]

    @property
    def ntet(self) -> int:
        return 6 * self.n[0] * self.n[1] * self.n[2]

    def nominal_evals(self, nq: Optional[int] = None, nw: Optional[int] = None) -> int:
        """(tetrahedron x band pair in window x q x omega) tuples; static counts one omega."""
        qs = self.qs if nq is None else self.qs[:nq]
        w = 1 if self.omega is None else len(self.omega)
        if nw is not None:
            w = nw
        tot = 0
        for q in qs:
            lo, hi = q.window if q.window is not None else self.window
            tot += (hi - lo) ** 2
        return self.ntet * tot * w


def builtin_tetra(n: Sequence[int], ids: np.ndarray):
    """Corner indices [len(ids), 4] (int32) and fractional volumes of tetrahedra ``ids`` of the
    periodic mesh n split 6 per cube: tetrahedron 6*cube + p = {000, e_a, e_a + e_b, 111} for
    the p-th axis order (a, b, .) of the permutations of (0, 1, 2) in lexicographic order,
    cube = (i0*n1 + i1)*n2 + i2.  Used to hand a sample of the builtin mesh to both sides as an
    explicit tetrahedron list."""
    import itertools
    n = [int(x) for x in n]
    ids = np.asarray(ids, dtype=np.int64)
    cube, p = ids // 6, ids % 6
    i2 = cube % n[2]
    r = cube // n[2]
    i1 = r % n[1]
    i0 = r // n[1]
    perms = np.array(list(itertools.permutations(range(3))))
    a, b = perms[p, 0], perms[p, 1]
    base = np.stack([i0, i1, i2], axis=1)
    o1 = np.zeros_like(base)
    o1[np.arange(len(ids)), a] = 1
    o2 = o1.copy()
    o2[np.arange(len(ids)), b] = 1
    corners = []
    for off in (np.zeros_like(base), o1, o2, np.ones_like(base)):
        x = (base + off) % np.asarray(n)
        corners.append((x[:, 0] * n[1] + x[:, 1]) * n[2] + x[:, 2])
    vol = np.full(len(ids), 1.0 / (6.0 * n[0] * n[1] * n[2]))
    return np.stack(corners, axis=1).astype(np.int32), vol


# ----------------------------------------------------------------------------------------
# linear algebra for the generators (LAPACK through numpy)
# ----------------------------------------------------------------------------------------
def _eigh_chunk(H: np.ndarray):
    w, v = np.linalg.eigh(H)
    return w, v


def eigh_batched(H: np.ndarray, nproc: int = 1, cdtype=np.complex128, pool=None):
    """Eigen-decomposition of a stack of Hermitian matrices [B, n, n].

    Returns (w [B, n] ascending, v [B, n, n] with v[b, :, j] the j-th eigenvector).
    ``pool``: a process pool to reuse (else one is started for this call when nproc > 1)."""
    B = H.shape[0]
    if nproc <= 1 or B < 4096:
        w, v = _eigh_chunk(H)
        return w, v.astype(cdtype, copy=False)
    import concurrent.futures as cf
    chunks = np.array_split(np.arange(B), nproc * 4)
    w = np.empty(H.shape[:2], dtype=np.float64)
    v = np.empty(H.shape, dtype=cdtype)
    ex = pool if pool is not None else _spawn_pool(nproc)
    try:
        futs = {ex.submit(_eigh_chunk, H[c]): c for c in chunks if len(c)}
        for f in cf.as_completed(futs):
            c = futs[f]
            wc, vc = f.result()
            w[c] = wc
            v[c] = vc
    finally:
        if pool is None:
            ex.shutdown()
    return w, v


def _eig_span(model, kfrac, idx, n, cdtype):
    """Eigen-data of one span of k points (fractional k, or grid indices idx of mesh n)."""
    H = model.hamiltonian(kfrac, grid=None if idx is None else (idx, n))
    w, v = np.linalg.eigh(H)
    return w, v.astype(cdtype, copy=False)


def _spawn_pool(nproc: int):
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=nproc, mp_context=mp.get_context("spawn"))


def default_nproc() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def fermi_level(E: np.ndarray, n_occ: float) -> float:
    """E_F at a filling of ``n_occ`` bands per k: midpoint between the last occupied
    and the first empty grid eigenvalue (a plain quantile of the grid levels)."""
    flat = np.sort(E.ravel())
    k = int(round(n_occ * E.shape[0]))
    k = min(max(k, 1), flat.size - 1)
    # never on a level: move to the nearest gap between distinct grid eigenvalues
    tol = 1e-9 * max(1.0, float(np.max(np.abs(flat))))
    for step in range(flat.size):
        for kk in (k + step, k - step):
            if 1 <= kk < flat.size and flat[kk] - flat[kk - 1] > tol:
                return float(0.5 * (flat[kk - 1] + flat[kk]))
    return float(0.5 * (flat[k - 1] + flat[k]))


# ----------------------------------------------------------------------------------------
# tight-binding models: H(k) = t0 + sum_{R in half} 2 cos(2 pi k.R) t(R),
# t(-R) = t(R) Hermitian ("Bloch-symmetric": H(k) Hermitian and even in k)
# ----------------------------------------------------------------------------------------
@dataclass
class TBModel:
    norb: int
    t0: np.ndarray                                    # [norb, norb] Hermitian
    bonds: List[Tuple[Tuple[int, int, int], np.ndarray]]  # half the bonds; partner -R implied

    def hamiltonian(self, kfrac: np.ndarray, grid=None) -> np.ndarray:
        """H(k) at fractional k.  ``grid = (idx [B,3] ints, n)``: k = idx/n exactly, with
        the phase k.R reduced in integers so that k and -k (mod G) get bitwise-identical
        Hamiltonians (exact symmetric degeneracies stay exact)."""
        B = kfrac.shape[0] if grid is None else grid[0].shape[0]
        H = np.broadcast_to(self.t0, (B, self.norb, self.norb)).astype(np.complex128)
        for R, t in self.bonds:
            if grid is None:
                ph = 2.0 * np.cos(2.0 * np.pi * (np.asarray(kfrac, dtype=np.float64) @ np.asarray(R, dtype=np.float64)))
            else:
                idx, n = grid
                L = int(np.lcm.reduce(np.asarray(n, dtype=np.int64)))
                p = (idx.astype(np.int64) * (np.asarray(R, dtype=np.int64) * (L // np.asarray(n, dtype=np.int64)))).sum(axis=1) % L
                p = np.minimum(p, L - p)
                ph = 2.0 * np.cos(2.0 * np.pi * p / L)
            H = H + ph[:, None, None] * t[None, :, :]
        return H

    def eig(self, kfrac: np.ndarray, nproc: int = 1, cdtype=np.complex128, chunk: int = 0, grid=None):
        B = kfrac.shape[0] if grid is None else grid[0].shape[0]
        if chunk <= 0:  # k points per batch: ~64 MB of Hamiltonians
            chunk = max(256, (1 << 22) // (self.norb * self.norb))
        w = np.empty((B, self.norb), dtype=np.float64)
        v = np.empty((B, self.norb, self.norb), dtype=cdtype)
        spans = [(s, min(B, s + chunk)) for s in range(0, B, chunk)]
        if nproc <= 1 or len(spans) < 2:
            for s, e in spans:
                w[s:e], v[s:e] = _eig_span(self, None if grid is not None else kfrac[s:e],
                                           None if grid is None else grid[0][s:e],
                                           None if grid is None else grid[1], cdtype)
            return w, v
        # workers build their own Hamiltonians from the k indices (only eigen-data travels
        # back) and run one LAPACK thread each
        import concurrent.futures as cf
        for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")
        with _spawn_pool(nproc) as ex:
            futs = {ex.submit(_eig_span, self, None if grid is not None else kfrac[s:e],
                              None if grid is None else grid[0][s:e], None if grid is None else grid[1],
                              cdtype): (s, e) for s, e in spans}
            for f in cf.as_completed(futs):
                s, e = futs[f]
                w[s:e], v[s:e] = f.result()
        return w, v

    def eig_grid(self, n, nproc: int = 1, cdtype=np.complex128):
        """Eigen-data at the corners of the periodic grid n (exact symmetric phases)."""
        return self.eig(None, nproc=nproc, cdtype=cdtype, grid=(corner_index(n, True), tuple(n)))


def _herm(rng, n, sigma):
    G = rng.normal(0.0, sigma, (n, n)) + 1j * rng.normal(0.0, sigma, (n, n))
    return 0.5 * (G + G.conj().T)


_SC1 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
_SC2 = [(1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]


def cr_like_model(seed: int = SEED_BASE + 2, norb: int = 9) -> TBModel:
    """9-orbital simple-cubic model: onsite diag U[-2,2] eV, first-neighbour complex
    Hermitian N(0,0.8) eV, second-neighbour N(0,0.3) eV (stand-in for Cr, Sec. III)."""
    rng = np.random.default_rng(seed)
    t0 = np.diag(rng.uniform(-2.0, 2.0, norb)).astype(np.complex128)
    bonds = [(R, _herm(rng, norb, 0.8)) for R in _SC1]
    bonds += [(R, _herm(rng, norb, 0.3)) for R in _SC2]
    return TBModel(norb, t0, bonds)


def fese_like_model(seed: int = SEED_BASE + 3) -> TBModel:
    """Tetragonal 2-site x 5-orbital model (stand-in for the two-Fe FeSe cell, Sec. III):
    site energies U[-1,1] eV, intra-cell inter-site and in-plane (x, y) hopping
    N(0,0.5) eV, out-of-plane (z) hopping N(0,0.05) eV."""
    rng = np.random.default_rng(seed)
    norb = 10
    t0 = np.diag(rng.uniform(-1.0, 1.0, norb)).astype(np.complex128)
    G = rng.normal(0.0, 0.5, (5, 5)) + 1j * rng.normal(0.0, 0.5, (5, 5))
    t0[:5, 5:] = G
    t0[5:, :5] = G.conj().T
    bonds = [((1, 0, 0), _herm(rng, norb, 0.5)), ((0, 1, 0), _herm(rng, norb, 0.5)),
             ((0, 0, 1), _herm(rng, norb, 0.05))]
    return TBModel(norb, t0, bonds)


def random_model(norb: int, seed: int, spread: float = 8.0) -> TBModel:
    """Gaussian random Hermitian onsite + nearest-neighbour model rescaled so the
    total band spread (over a 6^3 grid) is ``spread`` eV."""
    rng = np.random.default_rng(seed)
    t0 = _herm(rng, norb, 1.0)
    bonds = [(R, _herm(rng, norb, 1.0)) for R in _SC1]
    m = TBModel(norb, t0, bonds)
    w, _ = m.eig_grid((6, 6, 6))
    s = spread / float(w.max() - w.min())
    return TBModel(norb, t0 * s, [(R, t * s) for R, t in bonds])


# ----------------------------------------------------------------------------------------
# q lists
# ----------------------------------------------------------------------------------------
def path_points(nodes: Sequence[Sequence[float]], npts: int, closed_end: bool = False) -> np.ndarray:
    """``npts`` points at equal arc length along a polyline of fractional nodes; the last
    node is excluded unless ``closed_end``."""
    P = np.asarray(nodes, dtype=np.float64)
    seg = np.linalg.norm(np.diff(P, axis=0), axis=1)
    L = seg.sum()
    s = np.linspace(0.0, L, npts, endpoint=closed_end)
    out = np.empty((npts, 3))
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    for i, si in enumerate(s):
        j = min(np.searchsorted(cum, si, side="right") - 1, len(seg) - 1)
        t = (si - cum[j]) / seg[j]
        out[i] = P[j] + t * (P[j + 1] - P[j])
    return out


def explicit_q(model: TBModel, n, qfrac, nproc=1, cdtype=np.complex128, gamma_tol=1e-14):
    kf = corner_frac(n, True)
    w, v = model.eig(kf + np.asarray(qfrac)[None, :], nproc=nproc, cdtype=cdtype)
    gamma = bool(np.all(np.abs(np.asarray(qfrac) - np.round(qfrac)) < gamma_tol))
    return QPoint(Eq=w, Cq=v, gamma=gamma, frac=tuple(float(x) for x in qfrac))


# ----------------------------------------------------------------------------------------
# the five workloads (sizes overridable so tests can run them small)
# ----------------------------------------------------------------------------------------
def free_electron(n: int = 16, nq: int = 32, qmax_over_2kf: float = 1.0, axis: int = 0,
                  fill: float = 0.4) -> Workload:
    """Single band e(k) = |k|^2/2 (Hartree a.u., lattice constant 1 bohr) on the
    simple-cubic BZ [-pi, pi]^3 as an OPEN grid of n^3 cubes ((n+1)^3 corners), Fermi
    sphere filling ``fill`` of the BZ volume, |M|^2 = 1, q_j = j * 2 k_F/(nq-1) along
    ``axis``; energies at k+q are exact, |k+q|^2/2, at every corner."""
    kF = (fill * (2 * math.pi) ** 3 * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    ef = 0.5 * kF * kF
    N = n + 1
    ax = -math.pi + 2.0 * math.pi * np.arange(N) / n
    K = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    E = (0.5 * np.sum(K * K, axis=1))[:, None]
    qs = []
    if nq == 1:
        qv = np.array([0.0])
    else:
        qv = np.arange(nq) * (2.0 * kF * qmax_over_2kf) / (nq - 1)
    for qq in qv:
        Kq = K.copy()
        Kq[:, axis] += qq
        Eq = (0.5 * np.sum(Kq * Kq, axis=1))[:, None]
        frac = [0.0, 0.0, 0.0]
        frac[axis] = qq / (2 * math.pi)
        qs.append(QPoint(Eq=Eq, gamma=(qq == 0.0), frac=tuple(frac)))
    meta = dict(kF=kF, dos_ef=kF / math.pi ** 2, q_abs=qv, x=qv / (2 * kF))
    return Workload("free-electron static Lindhard", (n, n, n), False, 1, 1, E, None, ef,
                    (0, 1), True, qs, None, meta)


def cr_like(n: int = 48, nq: int = 256, nproc: int = 1, cdtype=np.complex128,
            cma: bool = False, qfracs=None) -> Workload:
    """Cr-like 9-orbital static workload: 256 q on Gamma-X-M-Gamma (equal arc length,
    off-grid, explicit k+q eigen-data), E_F at 6/9 filling."""
    m = cr_like_model()
    E, C = m.eig_grid((n, n, n), nproc=nproc, cdtype=cdtype)
    ef = fermi_level(E, 6.0)
    if qfracs is None:
        qfracs = path_points([(0, 0, 0), (0.5, 0, 0), (0.5, 0.5, 0), (0, 0, 0)], nq)
    qs = [explicit_q(m, (n, n, n), q, nproc=nproc, cdtype=cdtype) for q in qfracs]
    return Workload("Cr-like 9-orbital static", (n, n, n), True, 9, 9, E, C, ef, (0, 9), cma, qs,
                    None, dict(model=m))


def fese_like(n=(64, 64, 16), nq: int = 64, nw: int = 512, wmax: float = 2.0, nproc: int = 1,
              cdtype=np.complex128, cma: bool = False, qfracs=None) -> Workload:
    """FeSe-like dynamic workload: 10 bands, E_F at 6/10 filling, 64 q on Gamma-M
    (q_j = (j+1)/64 M, explicit k+q eigen-data), 512 omega in [0, 2] eV."""
    m = fese_like_model()
    E, C = m.eig_grid(n, nproc=nproc, cdtype=cdtype)
    ef = fermi_level(E, 6.0)
    if qfracs is None:
        qfracs = [np.array([0.5, 0.5, 0.0]) * (j + 1) / nq for j in range(nq)]
    qs = [explicit_q(m, n, q, nproc=nproc, cdtype=cdtype) for q in qfracs]
    omega = np.linspace(0.0, wmax, nw)
    return Workload("FeSe-like dynamic", tuple(n), True, 10, 10, E, C, ef, (0, 10), cma, qs,
                    omega, dict(model=m))


def _random_shifts(rng, n, nq):
    seen = set()
    out = []
    while len(out) < nq:
        s = tuple(int(x) for x in (rng.integers(0, n[0]), rng.integers(0, n[1]), rng.integers(0, n[2])))
        if s == (0, 0, 0) or s in seen:
            continue
        seen.add(s)
        out.append(s)
    return out


def band_sweep(n: int = 32, nb: int = 40, nq: int = 128, nw: int = 128, wmax: float = 2.0,
               wmin_band: int = 4, nproc: int = 1, cdtype=np.complex128) -> Workload:
    """40-band random model, 128 on-grid q each with its own band window
    w ~ U{4..40} centred on E_F: lo = clamp(n_occ - w//2, 0, nb - w)."""
    seed = SEED_BASE + 4
    m = random_model(nb, seed)
    E, C = m.eig_grid((n, n, n), nproc=nproc, cdtype=cdtype)
    nocc = nb // 2
    ef = fermi_level(E, nocc)
    rng = np.random.default_rng(seed + 1000)
    shifts = _random_shifts(rng, (n, n, n), nq)
    qs = []
    for s in shifts:
        w = int(rng.integers(wmin_band, nb + 1))
        lo = min(max(nocc - w // 2, 0), nb - w)
        qs.append(QPoint(shift=s, window=(lo, lo + w), frac=tuple(si / n for si in s)))
    omega = np.linspace(0.0, wmax, nw)
    return Workload("band-truncation sweep", (n, n, n), True, nb, nb, E, C, ef, (0, nb), False, qs,
                    omega, dict(model=m))


def large_mixed(n: int = 72, nb: int = 80, nq: int = 128, nw: int = 256, wmax: float = 2.0,
                nproc: int = 1, cdtype=np.complex64) -> Workload:
    """80-band random model on a 72^3 grid, complex64 eigenvectors, 128 on-grid q,
    256 omega in [0, 2] eV, full band window."""
    seed = SEED_BASE + 5
    m = random_model(nb, seed)
    E, C = m.eig_grid((n, n, n), nproc=nproc, cdtype=cdtype)
    ef = fermi_level(E, nb // 2)
    rng = np.random.default_rng(seed + 1000)
    qs = [QPoint(shift=s, frac=tuple(si / n for si in s)) for s in _random_shifts(rng, (n, n, n), nq)]
    omega = np.linspace(0.0, wmax, nw)
    return Workload("large mixed-precision", (n, n, n), True, nb, nb, E, C, ef, (0, nb), False, qs,
                    omega, dict(model=m))


def tiny_tb(n: int = 4, norb: int = 3, seed: int = SEED_BASE + 7, nq: int = 3, filling=None,
            explicit: bool = True, cdtype=np.complex128) -> Workload:
    """Small random model for brute-force and parity checks."""
    m = random_model(norb, seed, spread=4.0)
    E, C = m.eig_grid((n, n, n), cdtype=cdtype)
    nocc = norb / 2 if filling is None else filling
    ef = fermi_level(E, nocc)
    rng = np.random.default_rng(seed + 1)
    qs = []
    for j in range(nq):
        if explicit:
            q = rng.uniform(-0.5, 0.5, 3)
            qs.append(explicit_q(m, (n, n, n), q, cdtype=cdtype))
        else:
            s = tuple(int(x) for x in rng.integers(0, n, 3))
            qs.append(QPoint(shift=s, gamma=(s == (0, 0, 0)), frac=tuple(si / n for si in s)))
    return Workload("tiny TB", (n, n, n), True, norb, norb, E, C, ef, (0, norb), False, qs, None,
                    dict(model=m))
