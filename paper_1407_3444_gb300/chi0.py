"""Thin ctypes binding of include/chi0.h.

The functions keep the C names (``chi0_plan``, ``chi0_static``, ``chi0_dynamic``,
``chi0_destroy`` ...) and only marshal arguments; every step of chi0 runs in the
CUDA library.  ``Plan`` is a convenience wrapper that feeds a
``workloads.Workload`` through those calls, using torch tensors as device memory
when the inputs should be resident on the GPU.  There is no CPU fallback: if
libchi0.so is missing the import of the library fails loudly.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchi0.so")

CHI0_OK = 0
CHI0_EINVAL = -1
CHI0_ENOMEM = -2
CHI0_ECUDA = -3
CHI0_ETIMEOUT = -4
CHI0_ENOTSUP = -5
CHI0_EINTERNAL = -6
CHI0_C64 = 1
CHI0_C128 = 2
CHI0_PREC_FP64 = 0
CHI0_PREC_MIXED = 1
CHI0_OVL_FP32 = 0
CHI0_OVL_BF16X3 = 1
CHI0_OVL_TF32 = 2
CHI0_OVL_BF16X6 = 3
OVERLAP_MODES = {"fp32": CHI0_OVL_FP32, "bf16x3": CHI0_OVL_BF16X3, "tf32": CHI0_OVL_TF32, "bf16x6": CHI0_OVL_BF16X6}
CHI0_SIGN_POSITIVE = 0
CHI0_SIGN_PAPER = 1
CHI0_K_OVERLAP, CHI0_K_STATIC, CHI0_K_DYNAMIC, CHI0_K_REDUCE, CHI0_K_DOS, CHI0_K_BANDS = 0, 1, 2, 3, 4, 5
CHI0_K_GRAPH = 6
CHI0_K_COUNT = 8
# frequencies per k_dynamic launch: chi0_dynamic splits longer grids into passes of this size
DYNAMIC_MAX_NW = 256


class chi0_kgrid_t(ct.Structure):
    _fields_ = [("n", ct.c_int * 3), ("periodic", ct.c_int), ("nbands", ct.c_int), ("norb", ct.c_int),
                ("energies", ct.c_void_p), ("evecs", ct.c_void_p), ("evec_dtype", ct.c_int),
                ("e_fermi", ct.c_double)]


class chi0_tetra_t(ct.Structure):
    _fields_ = [("ntet", ct.c_int), ("corners", ct.c_void_p), ("volume", ct.c_void_p)]


class chi0_band_window_t(ct.Structure):
    _fields_ = [("lo", ct.c_int), ("hi", ct.c_int)]


class chi0_q_t(ct.Structure):
    _fields_ = [("shift", ct.c_int * 3), ("e_kq", ct.c_void_p), ("c_kq", ct.c_void_p),
                ("win", chi0_band_window_t), ("gamma", ct.c_int)]


class chi0_opts_t(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("overlap", ct.c_int), ("cma", ct.c_int), ("sign", ct.c_int),
                ("tau", ct.c_double), ("inputs_on_device", ct.c_int), ("outputs_on_device", ct.c_int),
                ("stream", ct.c_void_p), ("profile", ct.c_int), ("wait_budget", ct.c_longlong),
                ("test_stall", ct.c_int), ("graph", ct.c_int), ("reserved", ct.c_int * 6)]


class chi0_stats_t(ct.Structure):
    _fields_ = [("time_ms", ct.c_double * CHI0_K_COUNT), ("launches", ct.c_longlong * CHI0_K_COUNT),
                ("calls", ct.c_longlong), ("pieces", ct.c_longlong), ("fp64_evals", ct.c_longlong),
                ("kernels", ct.c_longlong), ("queue_overflow", ct.c_longlong), ("box_pieces", ct.c_longlong)]


class chi0_tune_t(ct.Structure):
    _fields_ = [("static_variant", ct.c_int), ("static_threads", ct.c_int),
                ("static_ctas_per_sm", ct.c_int), ("dynamic_ctas_per_sm", ct.c_int),
                ("tc_corners_per_round", ct.c_int), ("candidates", ct.c_int), ("best_ms", ct.c_double),
                ("default_ms", ct.c_double)]


class Chi0Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("chi0 error %d: %s" % (code, msg))
        self.code = code


_lib = None

# every entry point declared in include/chi0.h (checked by the ABI test)
EXPORTS = ["chi0_opts_default", "chi0_plan", "chi0_static", "chi0_dynamic", "chi0_plan_stats",
           "chi0_destroy", "chi0_last_error", "chi0_version", "chi0_static_noalloc", "chi0_tune", "chi0_peak",
           "chi0_static_pairs", "chi0_dynamic_kk", "chi0_interpolate_kq", "chi0_plan_update",
           "chi0_plan_stage"]
CHI0_PEAK_FP32_FMA, CHI0_PEAK_FP64_FMA, CHI0_PEAK_TF32_MMA, CHI0_PEAK_BF16_MMA = 0, 1, 2, 3
CHI0_NOALLOC_SCRATCH_BYTES = 64 << 20


def lib():
    """Load libchi0.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libchi0.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ct.CDLL(LIB_PATH)
        L.chi0_opts_default.argtypes = [ct.POINTER(chi0_opts_t)]
        L.chi0_opts_default.restype = None
        L.chi0_plan.argtypes = [ct.POINTER(chi0_kgrid_t), ct.POINTER(chi0_tetra_t), chi0_band_window_t,
                                ct.POINTER(chi0_opts_t), ct.POINTER(ct.c_void_p)]
        L.chi0_plan.restype = ct.c_int
        L.chi0_static.argtypes = [ct.c_void_p, ct.POINTER(chi0_q_t), ct.c_int, ct.c_void_p]
        L.chi0_static.restype = ct.c_int
        L.chi0_static_pairs.argtypes = [ct.c_void_p, ct.POINTER(chi0_q_t), ct.c_int, ct.c_void_p, ct.c_void_p]
        L.chi0_static_pairs.restype = ct.c_int
        L.chi0_dynamic_kk.argtypes = [ct.c_void_p, ct.POINTER(chi0_q_t), ct.c_int, ct.c_double, ct.c_int,
                                      ct.c_void_p, ct.c_void_p]
        L.chi0_dynamic_kk.restype = ct.c_int
        L.chi0_interpolate_kq.argtypes = [ct.c_void_p, ct.POINTER(ct.c_double), ct.c_void_p, ct.c_void_p]
        L.chi0_interpolate_kq.restype = ct.c_int
        L.chi0_plan_update.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.chi0_plan_update.restype = ct.c_int
        L.chi0_plan_stage.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.chi0_plan_stage.restype = ct.c_int
        L.chi0_dynamic.argtypes = [ct.c_void_p, ct.POINTER(chi0_q_t), ct.c_int, ct.c_void_p, ct.c_int,
                                   ct.c_void_p, ct.c_void_p]
        L.chi0_dynamic.restype = ct.c_int
        L.chi0_plan_stats.argtypes = [ct.c_void_p, ct.POINTER(chi0_stats_t)]
        L.chi0_plan_stats.restype = ct.c_int
        L.chi0_destroy.argtypes = [ct.c_void_p]
        L.chi0_destroy.restype = None
        L.chi0_last_error.argtypes = [ct.c_void_p]
        L.chi0_last_error.restype = ct.c_char_p
        L.chi0_version.argtypes = []
        L.chi0_version.restype = ct.c_int
        L.chi0_static_noalloc.argtypes = [ct.POINTER(chi0_kgrid_t), chi0_band_window_t, ct.POINTER(chi0_opts_t),
                                          ct.POINTER(chi0_q_t), ct.c_int, ct.c_void_p]
        L.chi0_static_noalloc.restype = ct.c_int
        L.chi0_tune.argtypes = [ct.c_void_p, ct.POINTER(chi0_q_t), ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p,
                                ct.c_void_p, ct.POINTER(chi0_tune_t)]
        L.chi0_tune.restype = ct.c_int
        L.chi0_peak.argtypes = [ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.chi0_peak.restype = ct.c_int
        _lib = L
    return _lib


def _check(rc, plan=None):
    if rc != CHI0_OK:
        msg = lib().chi0_last_error(plan)
        raise Chi0Error(rc, msg.decode() if msg else "")


# --------------------------------------------------------------- the C entry points
def chi0_opts_default() -> chi0_opts_t:
    o = chi0_opts_t()
    lib().chi0_opts_default(ct.byref(o))
    return o


def chi0_plan(kgrid: chi0_kgrid_t, tetra: Optional[chi0_tetra_t], window: chi0_band_window_t,
              opts: chi0_opts_t) -> ct.c_void_p:
    h = ct.c_void_p()
    rc = lib().chi0_plan(ct.byref(kgrid), ct.byref(tetra) if tetra is not None else None, window,
                         ct.byref(opts), ct.byref(h))
    _check(rc, None)
    return h


def chi0_static(plan, q, nq: int, chi_ptr: int) -> None:
    _check(lib().chi0_static(plan, q, nq, chi_ptr), plan)


def chi0_static_pairs(plan, q, nq: int, chi_ptr: int, pairs_ptr: int) -> None:
    _check(lib().chi0_static_pairs(plan, q, nq, chi_ptr, pairs_ptr), plan)


def chi0_interpolate_kq(plan, qfrac, e_ptr: int, c_ptr: int) -> None:
    q = (ct.c_double * 3)(*[float(x) for x in qfrac])
    _check(lib().chi0_interpolate_kq(plan, q, e_ptr, c_ptr), plan)


def chi0_dynamic_kk(plan, q, nq: int, wmax: float, nkk: int, re_ptr: int, im_ptr: int) -> None:
    _check(lib().chi0_dynamic_kk(plan, q, nq, wmax, nkk, re_ptr, im_ptr), plan)


def chi0_dynamic(plan, q, nq: int, omega_ptr: int, nw: int, re_ptr: int, im_ptr: int) -> None:
    _check(lib().chi0_dynamic(plan, q, nq, omega_ptr, nw, re_ptr, im_ptr), plan)


def chi0_tune(plan, q, nq: int, omega_ptr, nw: int, re_ptr: int, im_ptr) -> chi0_tune_t:
    r = chi0_tune_t()
    _check(lib().chi0_tune(plan, q, nq, omega_ptr, nw, re_ptr, im_ptr, ct.byref(r)), plan)
    return r


def chi0_plan_stats(plan) -> chi0_stats_t:
    s = chi0_stats_t()
    _check(lib().chi0_plan_stats(plan, ct.byref(s)), plan)
    return s


def chi0_destroy(plan) -> None:
    lib().chi0_destroy(plan)


def chi0_last_error(plan=None) -> str:
    m = lib().chi0_last_error(plan)
    return m.decode() if m else ""


def chi0_version() -> int:
    return lib().chi0_version()


def chi0_static_noalloc(kgrid: chi0_kgrid_t, window: chi0_band_window_t, opts: chi0_opts_t, q, nq: int,
                        chi_ptr: int) -> None:
    """Static chi0 with device-resident inputs/outputs and no device allocation (the
    library's fixed work array); see include/chi0.h."""
    _check(lib().chi0_static_noalloc(ct.byref(kgrid), window, ct.byref(opts), q, nq, chi_ptr), None)


def chi0_peak(kind: int, iters: int):
    """Measured peak (TFLOP/s, ms) of one arithmetic kind on the current device."""
    tf, ms = ct.c_double(), ct.c_double()
    _check(lib().chi0_peak(int(kind), int(iters), ct.byref(tf), ct.byref(ms)), None)
    return tf.value, ms.value


# --------------------------------------------------------------- convenience wrapper
def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Staged:
    """Energies/eigenvectors of a workload (and its explicit k+q data) in one place:
    ``where='device'`` torch CUDA tensors, ``'host'`` numpy, ``'pinned'`` page-locked host
    memory.  Several plans can share one staging."""

    def __init__(self, W, where: str = "device", cma: Optional[bool] = None):
        self.where = where
        self.cma = (W.cma or W.C is None) if cma is None else cma
        self.keep = []
        self._nbytes = 0
        if where != "host":
            import torch
            self.torch = torch
        E = np.ascontiguousarray(W.E, dtype=np.float64)
        self.dtype = None
        self.evec_dtype = CHI0_C128
        C = None
        if not self.cma:
            C = np.ascontiguousarray(W.C)
            if C.dtype == np.complex64:
                self.evec_dtype = CHI0_C64
            else:
                C = C.astype(np.complex128, copy=False)
            self.dtype = C.dtype
        self.E = self.put(E)
        self.C = self.put(C) if C is not None else 0
        self.q = []
        for q in W.qs:
            if q.Eq is None:
                self.q.append((0, 0))
                continue
            e = self.put(np.ascontiguousarray(q.Eq, dtype=np.float64))
            c = 0
            if not self.cma:
                c = self.put(np.ascontiguousarray(q.Cq).astype(self.dtype, copy=False))
            self.q.append((e, c))

    def put(self, a) -> int:
        self._nbytes += a.nbytes
        if self.where == "host":
            self.keep.append(a)
            return a.ctypes.data
        t = self.torch.from_numpy(a)
        if self.where == "device":
            x = t.to("cuda")
        else:
            x = t.pin_memory()
        self.keep.append(x)
        return x.data_ptr()

    def nbytes(self) -> int:
        return self._nbytes


def DeviceInputs(W, cma=None):
    return Staged(W, "device", cma)


def HostInputs(W, pinned: bool = True, cma=None):
    return Staged(W, "pinned" if pinned else "host", cma)


class Plan:
    """chi0 for one workload through the C-ABI.

    ``device=True``: inputs are device pointers (a ``Staged`` on the device) and outputs
    land in a torch CUDA tensor.  ``device=False``: host pointers (``Staged`` on the host,
    optionally pinned); the library copies them and returns host results."""

    def __init__(self, W, precision: str = "fp64", device: bool = True, stream=None, profile: bool = False,
                 tau: float = 9.5367431640625e-07, sign: int = CHI0_SIGN_POSITIVE, tetra=None, window=None, cma=None,
                 qs: Optional[Sequence] = None, staged: Optional[Staged] = None, overlap: str = "fp32",
                 wait_budget: int = 0, test_stall: bool = False, graph: bool = False):
        self.W = W
        self.device = device
        self.keep = []
        if staged is None:
            staged = Staged(W, "device" if device else "host", cma)
        self.staged = staged
        self.cma = staged.cma
        o = chi0_opts_default()
        o.precision = CHI0_PREC_FP64 if precision == "fp64" else CHI0_PREC_MIXED
        o.cma = 1 if self.cma else 0
        o.sign = sign
        o.tau = tau
        o.overlap = OVERLAP_MODES[overlap]
        o.wait_budget = int(wait_budget)
        o.test_stall = 1 if test_stall else 0
        o.graph = 1 if graph else 0
        self.graph = bool(graph)
        self._gout = {}
        o.profile = 1 if profile else 0
        o.inputs_on_device = 1 if device else 0
        o.outputs_on_device = 1 if device else 0
        self.torch = None
        if device:
            import torch
            self.torch = torch
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            o.stream = ct.c_void_p(self.stream.cuda_stream)
        else:
            o.stream = ct.c_void_p(0 if stream is None else stream.cuda_stream)
        self.opts = o
        kg = chi0_kgrid_t()
        kg.n[:] = list(W.n)
        kg.periodic = 1 if W.periodic else 0
        kg.nbands = W.nb
        kg.norb = W.norb
        kg.e_fermi = float(W.ef)
        kg.evec_dtype = staged.evec_dtype
        kg.energies = staged.E
        kg.evecs = staged.C if not self.cma else None
        self.kgrid = kg
        tt = None
        if tetra is not None:
            corners, vols = tetra
            corners = np.ascontiguousarray(corners, dtype=np.int32)
            vols = np.ascontiguousarray(vols, dtype=np.float64)
            self.keep += [corners, vols]
            tt = chi0_tetra_t(corners.shape[0], corners.ctypes.data, vols.ctypes.data)
        lo, hi = window if window is not None else W.window
        self.h = chi0_plan(kg, tt, chi0_band_window_t(lo, hi), o)
        self.window = (lo, hi)
        if qs is None:
            self.qarr = self.make_q(W.qs, staged.q)
        else:
            pos = {id(x): i for i, x in enumerate(W.qs)}
            self.qarr = self.make_q(qs, [staged.q[pos[id(q)]] for q in qs])

    def make_q(self, qs, ptrs):
        arr = (chi0_q_t * len(qs))()
        for i, (q, (e, c)) in enumerate(zip(qs, ptrs)):
            arr[i].shift[:] = list(q.shift)
            arr[i].e_kq = e if e else None
            arr[i].c_kq = c if c else None
            w = q.window if q.window is not None else (-1, -1)
            arr[i].win = chi0_band_window_t(w[0], w[1])
            arr[i].gamma = 1 if q.gamma else 0
        return arr

    def static(self, qarr=None, out=None):
        qarr = self.qarr if qarr is None else qarr
        nq = len(qarr)
        if self.device:
            t = self.torch
            if out is None and self.graph:
                # graph mode replays a call only with the same output pointers: one buffer per
                # call shape, overwritten by the next call
                key = ("s", nq)
                if key not in self._gout:
                    self._gout[key] = t.empty(nq, dtype=t.float64, device="cuda")
                out = self._gout[key]
            o = out if out is not None else t.empty(nq, dtype=t.float64, device="cuda")
            chi0_static(self.h, qarr, nq, o.data_ptr())
            return o
        o = np.empty(nq)
        chi0_static(self.h, qarr, nq, o.ctypes.data)
        return o

    def static_pairs(self, qarr=None):
        """Static chi0 and its band-pair contributions: (chi[nq], [w_q x w_q array per q])."""
        qarr = self.qarr if qarr is None else qarr
        nq = len(qarr)
        ws = []
        for i in range(nq):
            lo, hi = (qarr[i].win.lo, qarr[i].win.hi) if qarr[i].win.lo >= 0 else self.window
            ws.append(hi - lo)
        npairs = sum(w * w for w in ws)
        if self.device:
            t = self.torch
            o = t.empty(nq, dtype=t.float64, device="cuda")
            pr = t.empty(npairs, dtype=t.float64, device="cuda")
            chi0_static_pairs(self.h, qarr, nq, o.data_ptr(), pr.data_ptr())
            o, pr = o.cpu().numpy(), pr.cpu().numpy()
        else:
            o = np.empty(nq)
            pr = np.empty(npairs)
            chi0_static_pairs(self.h, qarr, nq, o.ctypes.data, pr.ctypes.data)
        blocks, off = [], 0
        for w in ws:
            blocks.append(pr[off:off + w * w].reshape(w, w))
            off += w * w
        return o, blocks

    def update(self, staged):
        """New eigen-data (a ``Staged`` of the same shapes and placement) for this plan."""
        _check(lib().chi0_plan_update(self.h, staged.E, staged.C if not self.cma else None), self.h)
        self.staged = staged

    def stage(self, staged):
        """Eigen-data (a host ``Staged``, best pinned) for a later call: up to two staged sets
        wait, and each call takes the oldest; the copies run while the plan's stream computes.
        The plan keeps references to the last three staged sets (two waiting, one current)."""
        _check(lib().chi0_plan_stage(self.h, staged.E, staged.C if not self.cma else None), self.h)
        self._held = getattr(self, "_held", ())[-2:] + (staged,)

    def interpolate_kq(self, qfrac):
        """Energies [Nc, nb] and eigenvectors [Nc, norb, nb] at k+q by linear interpolation from
        the mesh (numpy arrays; None for the vectors of a CMA plan)."""
        W = self.W
        nc = W.ncorner
        E = np.empty((nc, W.nb))
        Cq = None
        if self.device:
            t = self.torch
            Ed = t.empty((nc, W.nb), dtype=t.float64, device="cuda")
            Cd = None
            if not self.cma:
                Cd = t.empty((nc, W.norb, W.nb), dtype=t.complex64 if self.staged.evec_dtype == CHI0_C64
                             else t.complex128, device="cuda")
            chi0_interpolate_kq(self.h, qfrac, Ed.data_ptr(), Cd.data_ptr() if Cd is not None else None)
            self.stream.synchronize()
            E = Ed.cpu().numpy()
            Cq = Cd.cpu().numpy() if Cd is not None else None
        else:
            if not self.cma:
                Cq = np.empty((nc, W.norb, W.nb), dtype=np.complex64 if self.staged.evec_dtype == CHI0_C64
                              else np.complex128)
            chi0_interpolate_kq(self.h, qfrac, E.ctypes.data, Cq.ctypes.data if Cq is not None else None)
        return E, Cq

    def dynamic_kk(self, wmax: float, nkk: int, qarr=None):
        """Kramers-Kronig route: (re, im) [nq, nkk] on u_j = j wmax / (nkk - 1)."""
        qarr = self.qarr if qarr is None else qarr
        nq = len(qarr)
        if self.device:
            t = self.torch
            re = t.empty(nq * nkk, dtype=t.float64, device="cuda")
            im = t.empty(nq * nkk, dtype=t.float64, device="cuda")
            chi0_dynamic_kk(self.h, qarr, nq, float(wmax), int(nkk), re.data_ptr(), im.data_ptr())
            return re.view(nq, nkk), im.view(nq, nkk)
        re = np.empty((nq, nkk))
        im = np.empty((nq, nkk))
        chi0_dynamic_kk(self.h, qarr, nq, float(wmax), int(nkk), re.ctypes.data, im.ctypes.data)
        return re, im

    def dynamic(self, omega, qarr=None, out=None):
        qarr = self.qarr if qarr is None else qarr
        nq = len(qarr)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        nw = om.size
        if self.device:
            t = self.torch
            if getattr(self, "_om_host", None) is None or not np.array_equal(self._om_host, om):
                self._om = t.from_numpy(om).to("cuda")
                self._om_host = om.copy()
            if out is None and self.graph:
                key = ("d", nq, nw)
                if key not in self._gout:
                    self._gout[key] = (t.empty(nq * nw, dtype=t.float64, device="cuda"),
                                       t.empty(nq * nw, dtype=t.float64, device="cuda"))
                out = self._gout[key]
            re, im = out if out is not None else (t.empty(nq * nw, dtype=t.float64, device="cuda"),
                                                  t.empty(nq * nw, dtype=t.float64, device="cuda"))
            chi0_dynamic(self.h, qarr, nq, self._om.data_ptr(), nw, re.data_ptr(), im.data_ptr())
            return re.view(nq, nw), im.view(nq, nw)
        re = np.empty((nq, nw))
        im = np.empty((nq, nw))
        chi0_dynamic(self.h, qarr, nq, om.ctypes.data, nw, re.ctypes.data, im.ctypes.data)
        return re, im

    def stats(self):
        return chi0_plan_stats(self.h)

    def tune(self, omega=None, qarr=None) -> dict:
        """chi0_tune on this plan's q points (static, or dynamic on ``omega``); returns the
        chosen launch shape and the timings.  Device plans only."""
        if not self.device:
            raise ValueError("tune() runs on device-resident plans")
        t = self.torch
        qarr = self.qarr if qarr is None else qarr
        nq = len(qarr)
        if omega is None:
            o = t.empty(nq, dtype=t.float64, device="cuda")
            r = chi0_tune(self.h, qarr, nq, None, 0, o.data_ptr(), None)
        else:
            om = t.from_numpy(np.ascontiguousarray(omega, dtype=np.float64)).to("cuda")
            re = t.empty(nq * om.numel(), dtype=t.float64, device="cuda")
            im = t.empty_like(re)
            r = chi0_tune(self.h, qarr, nq, om.data_ptr(), om.numel(), re.data_ptr(), im.data_ptr())
        return {k: getattr(r, k) for k, _ in chi0_tune_t._fields_}

    def counters(self):
        s = self.stats()
        return {"pieces": int(s.pieces), "fp64_evals": int(s.fp64_evals), "kernels": int(s.kernels),
                "queue_overflow": int(s.queue_overflow), "box_pieces": int(s.box_pieces),
                "static_launches": int(s.launches[CHI0_K_STATIC]),
                "dynamic_launches": int(s.launches[CHI0_K_DYNAMIC])}

    def close(self):
        if getattr(self, "h", None):
            chi0_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
