"""Tensor-core overlaps (tcgen05.mma; CHI0_OVL_BF16X6, CHI0_OVL_BF16X3 and CHI0_OVL_TF32)
through the C-ABI, against the FP64 CPU oracle and against the CUDA-core FP32 overlap on the
same inputs.

Tolerances (normwise per q, Re and Im separately): BF16 split into three pieces with six
products, or two pieces with three products, 1e-6; one TF32 product 1e-4.  The cases cover
1 to 16 corners per MMA round (band windows from 4 to 40), the 80-band window whose
three-piece tile is staged in K chunks (double-buffered), a ragged last round, explicit
complex128 and complex64 k+q data, on-grid shifts, per-q windows, static and dynamic
results, and the bounded-wait error path of both the one-stage and the chunked kernel.
"""
import numpy as np
import pytest

from paper_1407_3444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"bf16x6": 1e-6, "bf16x3": 1e-6, "tf32": 1e-4}
MODES = ["bf16x6", "bf16x3", "tf32"]


@pytest.fixture(scope="module")
def C():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_3444_gb300 import build, chi0
    build.build()
    chi0.lib()
    return chi0


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def nerr(got, ref):
    got = np.atleast_2d(np.asarray(got, dtype=np.float64))
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    scale = np.max(np.abs(ref), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return float(np.max(np.max(np.abs(got - ref), axis=1) / scale))


def static(C, W, **kw):
    P = C.Plan(W, precision="mixed", **kw)
    out = P.static().cpu().numpy()
    P.close()
    return out


def dynamic(C, W, omega, **kw):
    P = C.Plan(W, precision="mixed", **kw)
    re, im = P.dynamic(omega)
    P.close()
    return re.cpu().numpy(), im.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
def test_tc_static_explicit_kq_complex128(C, O, mode):
    # 9 bands: 8 corners per round; 11^3 = 1331 corners leave a ragged last round
    W = wl.cr_like(n=11, nq=3)
    ref = O.chi0(W)
    got = static(C, W, overlap=mode)
    assert nerr(got[:, None], ref[:, None]) < TOL[mode], (got, ref)


@pytest.mark.parametrize("mode", MODES)
def test_tc_static_and_dynamic_band_windows_on_grid(C, O, mode):
    # 40 bands, on-grid shifts, per-q windows of 4..40 bands: 1 to 14 corners per round
    W = wl.band_sweep(n=8, nb=40, nq=6, nw=16)
    omega, W.omega = W.omega, None
    ref = O.chi0(W)
    got = static(C, W, overlap=mode)
    assert nerr(got[:, None], ref[:, None]) < TOL[mode]
    W.qs = W.qs[:2]
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    gr, gi = dynamic(C, W, omega, overlap=mode)
    assert nerr(gr, np.array(ref_r)) < TOL[mode]
    assert nerr(gi, np.array(ref_i)) < TOL[mode]


@pytest.fixture(scope="module")
def eighty(O):
    """The 80-band generator (complex64 eigenvectors) on a 4^3 mesh with its oracle values:
    static on two q, dynamic on one q and six frequencies."""
    W = wl.large_mixed(n=4, nq=2, nw=6)
    omega, W.omega = W.omega, None
    ref = O.chi0(W)
    ref_r, ref_i = O.chi0_q(W, W.qs[0], omega=omega)
    return W, omega, ref, ref_r, ref_i


@pytest.mark.parametrize("mode", MODES)
def test_tc_80_bands_chunked_k(C, eighty, mode):
    """w = norb = 80 gives one corner per round; the three-piece split stages K in three
    chunks of 4, 4 and 2 K steps through two buffers (the whole tile would need 276 KB), the
    other forms in one stage."""
    W, omega, ref, ref_r, ref_i = eighty
    got = static(C, W, overlap=mode)
    assert nerr(got[:, None], ref[:, None]) < TOL[mode], (got, ref)
    a = static(C, W, overlap="fp32")
    assert nerr(got[:, None], a[:, None]) < TOL[mode]
    W1 = wl.Workload(W.name, W.n, W.periodic, W.nb, W.norb, W.E, W.C, W.ef, W.window, W.cma, W.qs[:1])
    gr, gi = dynamic(C, W1, omega, overlap=mode)
    assert nerr(gr, ref_r[None, :]) < TOL[mode]
    assert nerr(gi, ref_i[None, :]) < TOL[mode]


def test_tc_dynamic_fese_like(C, O):
    W = wl.fese_like(n=(12, 12, 4), nq=2, nw=40, qfracs=[np.array([0.5, 0.5, 0.0]) * j / 64 for j in (3, 17)])
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=W.omega) for q in W.qs])
    for mode in ("bf16x6", "bf16x3"):
        gr, gi = dynamic(C, W, W.omega, overlap=mode)
        assert nerr(gr, np.array(ref_r)) < TOL[mode]
        assert nerr(gi, np.array(ref_i)) < TOL[mode]


def test_tc_complex64_inputs(C, O):
    W = wl.tiny_tb(n=7, norb=6, nq=3, seed=wl.SEED_BASE + 61, cdtype=np.complex64)
    ref = O.chi0(W)  # the oracle promotes the same complex64 values
    got = static(C, W, overlap="bf16x3")
    assert nerr(got[:, None], ref[:, None]) < TOL["bf16x3"]


def test_tc_matches_cuda_core_overlap(C):
    W = wl.tiny_tb(n=9, norb=12, nq=3, seed=wl.SEED_BASE + 62)
    a = static(C, W, overlap="fp32")
    for mode in ("bf16x6", "bf16x3"):
        b = static(C, W, overlap=mode)
        assert nerr(b[:, None], a[:, None]) < 1e-6, mode


@pytest.mark.parametrize("case", ["one_stage", "chunked"])
def test_tc_bounded_wait_runs_out_and_plans_stay_usable(C, O, case):
    """test_stall: the kernel issues no MMA, so the wait on its mbarrier runs out of the
    budget (2e6 cycles, about a millisecond); the call reports CHI0_ETIMEOUT and the plan
    and the device stay usable.  The chunked kernel (80 bands, three pieces) gives up at its
    first chunk, while the next chunk's operands are already staged."""
    if case == "one_stage":
        W, mode = wl.tiny_tb(n=6, norb=4, nq=2, seed=wl.SEED_BASE + 63), "bf16x3"
    else:
        W, mode = wl.large_mixed(n=4, nq=1, nw=4), "bf16x6"
        W.omega = None
    P = C.Plan(W, precision="mixed", overlap=mode, test_stall=True, wait_budget=2_000_000)
    with pytest.raises(C.Chi0Error) as ei:
        P.static()
    assert ei.value.code == C.CHI0_ETIMEOUT
    P.close()
    ref = O.chi0(W)
    got = static(C, W, overlap=mode)
    assert nerr(got[:, None], ref[:, None]) < TOL[mode]
