"""chi0_static_noalloc: static chi0 for callers that cannot allocate device memory where
they need it (allocation can synchronize the device and take unbounded time, or all
device memory belongs to the application's own pool).  It runs the static kernels with
the library's fixed work array instead of cudaMalloc'd buffers; here it is called through
the C-ABI and compared with chi0_static on the same device-resident inputs, twice in a
row (the work array keeps the previous call's contents)."""
import ctypes as ct

import numpy as np
import pytest

from paper_1407_3444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module")
def C():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_3444_gb300 import build, chi0
    build.build()
    chi0.lib()
    return chi0


def noalloc_args(C, W, staged, prec):
    kg = C.chi0_kgrid_t()
    kg.n[:] = list(W.n)
    kg.periodic = 1 if W.periodic else 0
    kg.nbands = W.nb
    kg.norb = W.norb
    kg.e_fermi = float(W.ef)
    kg.energies = staged.E
    kg.evecs = staged.C if staged.C else None
    kg.evec_dtype = staged.evec_dtype
    o = C.chi0_opts_default()
    o.precision = C.CHI0_PREC_FP64 if prec == "fp64" else C.CHI0_PREC_MIXED
    o.cma = 1 if staged.cma else 0
    o.inputs_on_device = 1
    o.outputs_on_device = 1
    import torch
    o.stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    qarr = (C.chi0_q_t * len(W.qs))()
    for i, (q, (e, c)) in enumerate(zip(W.qs, staged.q)):
        qarr[i].shift[:] = list(q.shift)
        qarr[i].e_kq = e if e else None
        qarr[i].c_kq = c if c else None
        win = q.window if q.window is not None else (-1, -1)
        qarr[i].win = C.chi0_band_window_t(*win)
        qarr[i].gamma = 1 if q.gamma else 0
    return kg, C.chi0_band_window_t(*W.window), o, qarr


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_chi0_static_on_two_calls(C, prec):
    import torch
    W = wl.tiny_tb(n=8, norb=4, nq=2, seed=wl.SEED_BASE + 60)
    W.qs += [wl.QPoint(shift=(0, 0, 0), gamma=True), wl.QPoint(shift=(3, 1, 5))]
    staged = C.DeviceInputs(W)
    P = C.Plan(W, precision=prec, device=True, staged=staged)
    ref = P.static().cpu().numpy()
    P.close()
    kg, win, opts, qarr = noalloc_args(C, W, staged, prec)
    out = torch.empty(len(W.qs), dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        C.chi0_static_noalloc(kg, win, opts, qarr, len(W.qs), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < TOL[prec], (call, got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_queue_overflow_path(C, prec):
    """A dense Fermi surface (40 bands, coarse mesh): batches queue more long-series final
    tetrahedra than the queue holds, and the overflow is evaluated in place by the carving
    warp.  The plan path's profile counter shows overflow with its 64-entry queue, so the
    16-entry queue of chi0_static_noalloc overflows too; both agree within the tolerance."""
    import torch
    W = wl.band_sweep(n=4, nb=40, nq=2, nw=4)
    W.omega = None
    W.qs = [wl.QPoint(shift=q.shift) for q in W.qs]  # full 40-band window
    staged = C.DeviceInputs(W)
    P = C.Plan(W, precision=prec, device=True, staged=staged, profile=True)
    ref = P.static().cpu().numpy()
    assert P.counters()["queue_overflow"] > 0
    P.close()
    kg, win, opts, qarr = noalloc_args(C, W, staged, prec)
    out = torch.empty(len(W.qs), dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        C.chi0_static_noalloc(kg, win, opts, qarr, len(W.qs), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref) / np.abs(ref)) < TOL[prec], (call, got, ref)


def test_noalloc_rejects_meshes_beyond_its_work_array(C):
    import torch
    E = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    kg = C.chi0_kgrid_t()
    kg.n[:] = [200, 200, 200]
    kg.periodic = 1
    kg.nbands = 9
    kg.norb = 9
    kg.e_fermi = 0.0
    kg.energies = E.data_ptr()
    kg.evecs = E.data_ptr()
    kg.evec_dtype = C.CHI0_C128
    o = C.chi0_opts_default()
    o.precision = C.CHI0_PREC_MIXED
    q = (C.chi0_q_t * 1)()
    q[0].win = C.chi0_band_window_t(-1, -1)
    with pytest.raises(C.Chi0Error) as ei:
        C.chi0_static_noalloc(kg, C.chi0_band_window_t(0, 9), o, q, 1, E.data_ptr())
    assert ei.value.code == C.CHI0_EINVAL
    assert "bytes of scratch" in str(ei.value)
