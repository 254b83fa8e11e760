"""ctypes wrapper around the FP64 CPU oracle (chi0_oracle.c).

TEST INFRASTRUCTURE: only tests/, ``__graft_entry__.smoke()`` and ``bench.py``
(its cpu_baseline leg and ``--impl reference``) import this package.  The CUDA
library never loads it and shares no code with it.
"""
from __future__ import annotations

import ctypes as ct
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chi0_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_chi0.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, IEEE FP64: no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Input(ct.Structure):
    _fields_ = [
        ("n", ct.c_int * 3), ("periodic", ct.c_int), ("nb", ct.c_int), ("norb", ct.c_int),
        ("E", ct.c_void_p), ("C", ct.c_void_p), ("Eq", ct.c_void_p), ("Cq", ct.c_void_p),
        ("shift", ct.c_int * 3), ("ef", ct.c_double), ("lo", ct.c_int), ("hi", ct.c_int),
        ("cma", ct.c_int), ("gamma", ct.c_int), ("ntet", ct.c_int), ("tet", ct.c_void_p),
        ("tvol", ct.c_void_p), ("nw", ct.c_int), ("omega", ct.c_void_p), ("sign", ct.c_int),
        ("nthreads", ct.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            dp = ct.POINTER(ct.c_double)
            L.oracle_inv_weight.restype = ct.c_double
            L.oracle_inv_weight.argtypes = [dp, ct.c_int]
            L.oracle_mspline.restype = ct.c_double
            L.oracle_mspline.argtypes = [dp, ct.c_int, ct.c_double]
            L.oracle_delta_weight.restype = ct.c_double
            L.oracle_delta_weight.argtypes = [dp, ct.c_int, ct.c_double]
            L.oracle_tet_dos.restype = ct.c_double
            L.oracle_tet_dos.argtypes = [dp]
            L.oracle_carve.restype = ct.c_int
            L.oracle_carve.argtypes = [dp, dp, dp, dp, dp, dp]
            L.oracle_tet_integrals.restype = None
            L.oracle_tet_integrals.argtypes = [dp, dp, dp, ct.c_int, dp, dp, dp]
            L.oracle_chi0.restype = ct.c_int
            L.oracle_chi0.argtypes = [ct.POINTER(_Input), dp, dp]
            L.oracle_chi0_pairs.restype = ct.c_int
            L.oracle_chi0_pairs.argtypes = [ct.POINTER(_Input), dp]
            L.oracle_max_threads.restype = ct.c_int
            L.oracle_input_size.restype = ct.c_int
            assert L.oracle_input_size() == ct.sizeof(_Input), "oracle_input layout mismatch"
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _f64(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------------- single tetrahedron
def inv_weight(x, j: int) -> float:
    """(1/V) int_S lambda_j / X  for vertex values x (PV if X changes sign)."""
    return lib().oracle_inv_weight(_dp(_f64(x, 4)), int(j))


def mspline(knots, x: float) -> float:
    t = _f64(knots)
    return lib().oracle_mspline(_dp(t), t.size, float(x))


def delta_weight(d, j: int, w: float) -> float:
    return lib().oracle_delta_weight(_dp(_f64(d, 4)), int(j), float(w))


def tet_dos(a) -> float:
    return lib().oracle_tet_dos(_dp(_f64(a, 4)))


def carve(a, b, f=(1, 1, 1, 1)):
    """Final tetrahedra of the two carvings: (relative volumes [n], D [n,4], f [n,4])."""
    vol = np.zeros(9)
    D = np.zeros(36)
    F = np.zeros(36)
    n = lib().oracle_carve(_dp(_f64(a, 4)), _dp(_f64(b, 4)), _dp(_f64(f, 4)), _dp(vol), _dp(D), _dp(F))
    return vol[:n].copy(), D[:4 * n].reshape(n, 4).copy(), F[:4 * n].reshape(n, 4).copy()


def tet_integrals(a, b, f=(1, 1, 1, 1), omega=None):
    """Positive-sign integrals over a unit-volume tetrahedron: static int f*2/D, or
    (Re, Im)[w] = (int f [1/(D-w)+1/(D+w)], pi int f delta(w-D))."""
    if omega is None:
        re = np.zeros(1)
        lib().oracle_tet_integrals(_dp(_f64(a, 4)), _dp(_f64(b, 4)), _dp(_f64(f, 4)), 0, None, _dp(re), None)
        return float(re[0])
    w = _f64(omega)
    re = np.zeros(w.size)
    im = np.zeros(w.size)
    lib().oracle_tet_integrals(_dp(_f64(a, 4)), _dp(_f64(b, 4)), _dp(_f64(f, 4)), w.size, _dp(w), _dp(re), _dp(im))
    return re, im


# ---------------------------------------------------------------------- full chi0 for one q
def _input(W, q, omega, sign, nthreads, tet, tvol, window):
    """The oracle's input record for one q (and the arrays it points into)."""
    keep = []
    inp = _Input()
    inp.n[:] = list(W.n)
    inp.periodic = 1 if W.periodic else 0
    inp.nb = W.nb
    inp.norb = W.norb
    E = _f64(W.E)
    keep.append(E)
    inp.E = E.ctypes.data
    cma = bool(W.cma) or W.C is None
    if not cma:
        C = np.ascontiguousarray(W.C, dtype=np.complex128)
        keep.append(C)
        inp.C = C.ctypes.data
    if q.Eq is not None:
        Eq = _f64(q.Eq)
        keep.append(Eq)
        inp.Eq = Eq.ctypes.data
        if not cma:
            Cq = np.ascontiguousarray(q.Cq, dtype=np.complex128)
            keep.append(Cq)
            inp.Cq = Cq.ctypes.data
    inp.shift[:] = list(q.shift)
    inp.ef = float(W.ef)
    lo, hi = window if window is not None else (q.window if q.window is not None else W.window)
    inp.lo, inp.hi = int(lo), int(hi)
    inp.cma = 1 if cma else 0
    inp.gamma = 1 if q.gamma else 0
    if tet is not None:
        T = np.ascontiguousarray(tet, dtype=np.int32)
        V = _f64(tvol)
        keep += [T, V]
        inp.ntet = T.shape[0]
        inp.tet = T.ctypes.data
        inp.tvol = V.ctypes.data
    if omega is not None:
        w = _f64(omega)
        keep.append(w)
        inp.nw = w.size
        inp.omega = w.ctypes.data
    inp.sign = int(sign)
    inp.nthreads = int(nthreads)
    return inp, keep, (int(lo), int(hi))


def chi0_q(W, q, omega=None, sign: int = 0, nthreads: int = 0, tet=None, tvol=None, window=None):
    """chi0 at one q of workload W (see paper_1407_3444_gb300.workloads).

    Returns the static value (float) when ``omega`` is None and W is static, else
    (re[nw], im[nw]).  ``tet``/``tvol`` restrict the sum to a caller tetrahedron list."""
    if omega is None:
        omega = W.omega
    inp, keep, _ = _input(W, q, omega, sign, nthreads, tet, tvol, window)
    nout = 1 if omega is None else len(omega)
    re = np.zeros(nout)
    im = np.zeros(nout)
    rc = lib().oracle_chi0(ct.byref(inp), _dp(re), _dp(im))
    if rc != 0:
        raise RuntimeError("oracle_chi0 failed: %d" % rc)
    if omega is None:
        return float(re[0])
    return re, im


def chi0_pairs_q(W, q, sign: int = 0, nthreads: int = 0, tet=None, tvol=None, window=None):
    """Static chi0 at one q resolved by band pair: [w, w] array, entry (m - lo, n - lo) the
    contribution of the transitions m -> n (Sec. III, Fig. 8); the entries add up to chi0_q."""
    inp, keep, (lo, hi) = _input(W, q, None, sign, nthreads, tet, tvol, window)
    w = hi - lo
    out = np.zeros(w * w)
    rc = lib().oracle_chi0_pairs(ct.byref(inp), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle_chi0_pairs failed: %d" % rc)
    return out.reshape(w, w)


def kk_re_from_im(u, im, w):
    """Re(w) = (1/pi) PV int_0^inf Im(u) [1/(u - w) + 1/(u + w)] du for Im given on the
    ascending nodes u (u[0] = 0, Im(u[0]) = 0), linear between them and 0 past the last node
    (taken to fall to 0 over one more spacing of the last interval).  Segment by segment: on
    [a, b] with Im = alpha + beta u,  int (alpha + beta u)/(u - c) du
    = beta (b - a) + (alpha + beta c) ln|(b - c)/(a - c)|  (principal value if c in (a, b);
    the logarithms of adjacent segments at a node c = a or b cancel and are dropped)."""
    u = np.asarray(u, dtype=np.float64)
    im = np.asarray(im, dtype=np.float64)
    uu = np.append(u, u[-1] + (u[-1] - u[-2]))
    yy = np.append(im, 0.0)
    out = np.zeros(len(w))
    for i, wv in enumerate(np.asarray(w, dtype=np.float64)):
        tot = 0.0
        for c in (wv, -wv):
            for j in range(len(uu) - 1):
                a, b = uu[j], uu[j + 1]
                ya, yb = yy[j], yy[j + 1]
                beta = (yb - ya) / (b - a)
                alpha = ya - beta * a
                lb = math.log(abs(b - c)) if b != c else 0.0
                la = math.log(abs(a - c)) if a != c else 0.0
                # at a node the singular parts of the two segments cancel: drop log|0|, keep
                # the finite remainder (the value there times the log of the other end)
                tot += beta * (b - a) + (alpha + beta * c) * (lb - la)
        out[i] = tot / math.pi
    return out


def kq_interpolate(W, qfrac):
    """Energies and eigenvectors at k+q for every corner k of W's periodic mesh by linear
    interpolation from the mesh (Sec. II): k+q lies in one tetrahedron {000, e_p0, e_p0 + e_p1,
    111} of one cube (p sorts the cube-local coordinates t descending); the barycentric weights
    are (1 - t_p0, t_p0 - t_p1, t_p1 - t_p2, t_p2).  Energies: the weighted sum per band.
    Eigenvectors: per band, the corner vectors turned onto the phase of the first corner's
    (times conj(<v_0|v_i>) / |<v_0|v_i>|), summed with the weights and normalised.
    Returns (Eq [Nc, nb], Cq [Nc, norb, nb] complex128, or None without eigenvectors)."""
    n = np.array(W.n, dtype=np.int64)
    assert W.periodic
    nc = int(np.prod(n))
    i0, i1, i2 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    idx = np.stack([i0.ravel(), i1.ravel(), i2.ravel()], axis=1)          # corner c -> (i0, i1, i2)
    x = idx + np.asarray(qfrac, dtype=np.float64)[None, :] * n[None, :]
    fl = np.floor(x)
    t = x - fl
    base = np.mod(fl.astype(np.int64), n[None, :])
    E = np.asarray(W.E, dtype=np.float64)
    C = None if (W.cma or W.C is None) else np.asarray(W.C, dtype=np.complex128)
    Eq = np.empty_like(E)
    Cq = None if C is None else np.empty_like(C)
    for c in range(nc):
        tc = t[c]
        # axis order: descending t, ties to the lower axis (a stable sort of -t)
        order = sorted(range(3), key=lambda d: (-tc[d], d))
        w = [1.0 - tc[order[0]], tc[order[0]] - tc[order[1]], tc[order[1]] - tc[order[2]], tc[order[2]]]
        off = np.zeros(3, dtype=np.int64)
        corners = []
        for v in range(4):
            if v >= 1:
                off[order[v - 1]] = 1
            j = np.mod(base[c] + off, n)
            corners.append(int((j[0] * n[1] + j[1]) * n[2] + j[2]))
        Eq[c] = sum(w[v] * E[corners[v]] for v in range(4))
        if C is not None:
            v0 = C[corners[0]]                                   # [norb, nb]
            acc = np.zeros_like(v0)
            for v in range(4):
                vi = C[corners[v]]
                if v == 0:
                    ph = np.ones(vi.shape[1], dtype=np.complex128)
                else:
                    ov = np.sum(np.conj(v0) * vi, axis=0)        # <v_0|v_i> per band
                    m = np.abs(ov)
                    ph = np.where(m > 0, np.conj(ov) / np.where(m > 0, m, 1.0), 1.0)
                acc += w[v] * vi * ph[None, :]
            nrm = np.sqrt(np.sum(np.abs(acc) ** 2, axis=0))
            Cq[c] = acc / np.where(nrm > 0, nrm, 1.0)[None, :]
    return Eq, Cq


def chi0(W, omega=None, sign: int = 0, nthreads: int = 0, qs=None):
    """chi0 for every q of W: static -> [nq]; dynamic -> (re [nq, nw], im [nq, nw])."""
    qs = W.qs if qs is None else qs
    out = [chi0_q(W, q, omega=omega, sign=sign, nthreads=nthreads) for q in qs]
    if (omega if omega is not None else W.omega) is None:
        return np.array(out)
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def max_threads() -> int:
    return lib().oracle_max_threads()
