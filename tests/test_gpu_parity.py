"""CUDA path (through the C-ABI) against the FP64 CPU oracle, element by element.

Tolerances (normwise per q, separately for Re and Im: max_w |gpu - ref| / max_w |ref|):
  * all-FP64 GPU form: 1e-12;
  * mixed precision (FP32 overlaps and weights, FP64 near-degenerate branches, FP64
    accumulation): 1e-6.
"""
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


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def nerr(got, ref):
    got = np.atleast_2d(np.asarray(got, dtype=np.float64))
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    scale = np.max(np.abs(ref), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return float(np.max(np.max(np.abs(got - ref), axis=1) / scale))


def run_static(C, W, prec, device=True, **kw):
    P = C.Plan(W, precision=prec, device=device, **kw)
    out = P.static()
    P.close()
    return out.cpu().numpy() if hasattr(out, "cpu") else out


def run_dynamic(C, W, prec, omega, device=True, **kw):
    P = C.Plan(W, precision=prec, device=device, **kw)
    re, im = P.dynamic(omega)
    P.close()
    if hasattr(re, "cpu"):
        re, im = re.cpu().numpy(), im.cpu().numpy()
    return re, im


# ------------------------------------------------------------------------ static
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_free_electron(C, O, prec):
    W = wl.free_electron(12, 7)
    ref = O.chi0(W)
    got = run_static(C, W, prec)
    assert nerr(got[:, None], ref[:, None]) < TOL[prec], (got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_tb_explicit_ragged(C, O, prec):
    # 12^3 grid: 10368 tetrahedra > one grid-stride round of warps; 5 bands
    W = wl.tiny_tb(n=12, norb=5, nq=3, seed=wl.SEED_BASE + 40)
    ref = O.chi0(W)
    got = run_static(C, W, prec)
    assert nerr(got[:, None], ref[:, None]) < TOL[prec], (got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_tb_shift_and_gamma(C, O, prec):
    W = wl.tiny_tb(n=8, norb=4, nq=0, seed=wl.SEED_BASE + 41)
    W.qs = [wl.QPoint(shift=(0, 0, 0), gamma=True), wl.QPoint(shift=(1, 0, 0)), wl.QPoint(shift=(3, 5, 7)),
            wl.QPoint(shift=(-1, 2, -3))]
    Wo = wl.Workload(W.name, W.n, W.periodic, W.nb, W.norb, W.E, W.C, W.ef, W.window, W.cma,
                     [wl.QPoint(shift=tuple(s % 8 for s in q.shift), gamma=q.gamma) for q in W.qs])
    ref = O.chi0(Wo)
    got = run_static(C, W, prec)
    assert nerr(got[:, None], ref[:, None]) < TOL[prec], (got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_per_q_windows(C, O, prec):
    W = wl.tiny_tb(n=6, norb=8, nq=0, seed=wl.SEED_BASE + 42)
    rng = np.random.default_rng(5)
    qs = []
    for j in range(6):
        w = int(rng.integers(2, 9))
        lo = min(max(4 - w // 2, 0), 8 - w)
        qs.append(wl.QPoint(shift=tuple(int(x) for x in rng.integers(0, 6, 3)), window=(lo, lo + w)))
    W.qs = qs
    ref = O.chi0(W)
    got = run_static(C, W, prec)
    assert nerr(got[:, None], ref[:, None]) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_band_pairs(C, O, prec):
    """Band-pair resolved static chi0 (chi0_static_pairs) against the oracle's pair sums: a
    general on-grid q, Gamma (the intraband pairs carry their band's DOS) and per-q windows of
    different widths (blocks back to back); each pair within the form's
    tolerance of the largest pair of its q, and the pairs of a q add up to its chi0."""
    W = wl.tiny_tb(n=8, norb=6, nq=0, seed=wl.SEED_BASE + 45)
    qs = [wl.QPoint(shift=(1, 3, 2)), wl.QPoint(shift=(0, 0, 0), gamma=True),
          wl.QPoint(shift=(2, 0, 5), window=(1, 5)), wl.QPoint(shift=(4, 4, 4), window=(2, 4))]
    W.qs = qs
    P = C.Plan(W, precision=prec, device=True)
    chi, blocks = P.static_pairs()
    P.close()
    tot_ref = O.chi0(W)
    assert nerr(chi[:, None], tot_ref[:, None]) < TOL[prec]
    for iq, q in enumerate(qs):
        ref = O.chi0_pairs_q(W, q)
        got = blocks[iq]
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= TOL[prec] * np.max(np.abs(ref)), (iq, got, ref)
        assert abs(got.sum() - chi[iq]) <= 1e-12 * abs(chi[iq]) + 1e-14, (iq, got.sum(), chi[iq])
    # host outputs give the same numbers, bitwise (fixed-point sums)
    Ph = C.Plan(W, precision=prec, device=False)
    chi_h, blocks_h = Ph.static_pairs()
    Ph.close()
    for a, b in zip(blocks, blocks_h):
        assert np.array_equal(a, b)


def test_sweep_drivers(C, O):
    """The Sec. III comparison drivers: band windows around E_F, CMA against exact |M|^2 (and
    the CMA curve shifted to 0 at the first q), and the band-pair histogram, each against the
    oracle with the same window or matrix elements (FP64, 1e-12)."""
    import dataclasses
    from paper_1407_3444_gb300 import sweeps
    W = wl.tiny_tb(n=6, norb=6, nq=0, seed=wl.SEED_BASE + 47)
    W.qs = [wl.QPoint(shift=(0, 0, 1)), wl.QPoint(shift=(1, 2, 0)), wl.QPoint(shift=(3, 3, 3))]
    tr = sweeps.band_truncation(W, W.qs, [2, 4, 6], precision="fp64")
    nocc = int(np.round(np.mean(np.sum(W.E < W.ef, axis=1))))
    for w, got in tr.items():
        lo = min(max(nocc - w // 2, 0), W.nb - w)
        ref = np.array([O.chi0_q(W, q, window=(lo, lo + w)) for q in W.qs])
        assert nerr(got[:, None], ref[:, None]) < 1e-12, (w, got, ref)
    exact, cma, shifted = sweeps.cma_vs_exact(W, W.qs, precision="fp64")
    Wc = dataclasses.replace(W, cma=True)
    assert nerr(exact[:, None], O.chi0(W)[:, None]) < 1e-12
    assert nerr(cma[:, None], O.chi0(Wc)[:, None]) < 1e-12
    assert shifted[0] == 0.0 and np.allclose(shifted, cma - cma[0], rtol=0, atol=0)
    chi, pairs = sweeps.pair_contributions(W, W.qs[1], precision="fp64")
    assert abs(pairs.sum() - chi) <= 1e-12 * abs(chi)
    assert np.max(np.abs(pairs - O.chi0_pairs_q(W, W.qs[1]))) <= 1e-12 * np.max(np.abs(pairs))


@pytest.mark.parametrize("cdt", ["c128", "c64"])
def test_interpolated_kq(C, O, cdt):
    """Off-grid q by linear interpolation of the mesh data (chi0_interpolate_kq, Sec. II)
    against the oracle's interpolation, then chi0 on the interpolated k+q data (explicit q)
    against the oracle on the same data; host and device outputs agree bitwise."""
    cdtype = np.complex64 if cdt == "c64" else np.complex128
    W = wl.tiny_tb(n=6, norb=4, nq=0, seed=wl.SEED_BASE + 54, cdtype=cdtype)
    q = (0.173, 0.061, 0.29)
    P = C.Plan(W, precision="fp64", device=True)
    Eq, Cq = P.interpolate_kq(q)
    P.close()
    Ph = C.Plan(W, precision="fp64", device=False)
    Eh, Ch = Ph.interpolate_kq(q)
    Ph.close()
    assert np.array_equal(Eq, Eh) and np.array_equal(Cq, Ch)
    Eo, Co = O.kq_interpolate(W, q)
    tol = 1e-12 if cdt == "c128" else 1e-6
    assert np.max(np.abs(Eq - Eo)) <= 1e-12 * np.max(np.abs(Eo))
    assert np.max(np.abs(Cq - Co)) <= tol, np.max(np.abs(Cq - Co))
    Wq = wl.Workload(W.name, W.n, W.periodic, W.nb, W.norb, W.E, W.C, W.ef, W.window, False,
                     [wl.QPoint(Eq=Eq, Cq=Cq.astype(W.C.dtype))])
    got = run_static(C, Wq, "fp64")
    Wo = wl.Workload(W.name, W.n, W.periodic, W.nb, W.norb, W.E, W.C.astype(np.complex128), W.ef, W.window, False,
                     [wl.QPoint(Eq=Eq, Cq=Cq.astype(np.complex128))])
    ref = O.chi0(Wo)
    assert nerr(got[:, None], ref[:, None]) < (1e-12 if cdt == "c128" else 1e-6)


@pytest.mark.parametrize("device", [True, False])
def test_plan_update_matches_a_fresh_plan(C, device):
    """chi0_plan_update: a plan built on one model's eigen-data and handed another's (same
    shapes) gives bitwise the results of a plan built on the second, static and dynamic, mixed
    (its FP32 copies rebuilt) and FP64."""
    Wa = wl.tiny_tb(n=6, norb=4, nq=0, seed=wl.SEED_BASE + 55)
    Wb = wl.tiny_tb(n=6, norb=4, nq=0, seed=wl.SEED_BASE + 56)
    Wb.ef = Wa.ef  # the plan keeps its Fermi level
    qs = [wl.QPoint(shift=(1, 0, 2)), wl.QPoint(shift=(3, 3, 1))]
    Wa.qs, Wb.qs = qs, qs
    omega = np.linspace(0.0, 2.0, 40)
    for prec in ("mixed", "fp64"):
        Pa = C.Plan(Wa, precision=prec, device=device)
        Sb = C.DeviceInputs(Wb) if device else C.HostInputs(Wb, pinned=False)
        Pa.update(Sb)
        got_s = Pa.static()
        got_d = Pa.dynamic(omega)
        Pa.close()
        Pb = C.Plan(Wb, precision=prec, device=device)
        ref_s = Pb.static()
        ref_d = Pb.dynamic(omega)
        Pb.close()
        cv = (lambda x: x.cpu().numpy()) if device else np.asarray
        assert np.array_equal(cv(got_s), cv(ref_s))
        assert np.array_equal(cv(got_d[0]), cv(ref_d[0])) and np.array_equal(cv(got_d[1]), cv(ref_d[1]))


def test_plan_stage_feeds_the_next_call(C):
    """chi0_plan_stage: calls take the staged sets oldest first and compute on them (bitwise
    the results of a plan built on each set), also with two sets waiting (the second copied
    into the buffers of the set in use before); a call with nothing staged keeps the current
    set; a third waiting set is refused; chi0_plan_update drops the staged sets; a plan with
    device inputs refuses staging."""
    Wa = wl.tiny_tb(n=6, norb=4, nq=0, seed=wl.SEED_BASE + 57)
    Wb = wl.tiny_tb(n=6, norb=4, nq=0, seed=wl.SEED_BASE + 58)
    Wb.ef = Wa.ef  # the plan keeps its Fermi level
    qs = [wl.QPoint(shift=(1, 0, 2)), wl.QPoint(shift=(2, 3, 1))]
    Wa.qs, Wb.qs = qs, qs
    omega = np.linspace(0.0, 2.0, 40)
    for prec in ("mixed", "fp64"):
        ref = {}
        for name, W in (("a", Wa), ("b", Wb)):
            P = C.Plan(W, precision=prec, device=False)
            ref[name] = (P.static(), P.dynamic(omega))
            P.close()
        Sa, Sb = C.HostInputs(Wa, pinned=True), C.HostInputs(Wb, pinned=True)
        P = C.Plan(Wa, precision=prec, device=False)
        P.stage(Sb)  # -> the alt buffers
        P.stage(Sa)  # -> the current buffers (holding a: no call reads them again)
        with pytest.raises(C.Chi0Error) as ei:
            P.stage(Sb)  # two sets wait already
        assert ei.value.code == C.CHI0_EINVAL
        d1 = P.dynamic(omega)  # takes b
        s2 = P.static()  # takes a
        d3 = P.dynamic(omega)  # nothing staged: still a
        P.stage(Sb)
        P.stage(Sb)  # into the buffers the current a sits in
        P.update(Sa)  # drops both (after their copies) and copies a
        s4 = P.static()
        seq = "babab"  # the pipeline: stage(i + 1) before call(i)
        sets = {"a": Sa, "b": Sb}
        P.stage(sets[seq[0]])
        s5 = []
        for i in range(len(seq)):
            if i + 1 < len(seq):
                P.stage(sets[seq[i + 1]])
            s5.append(P.static())
        d6 = P.dynamic(omega)  # nothing staged: the last set
        P.close()
        for got, want in ((d1, ref["b"][1]), (d3, ref["a"][1]), (d6, ref[seq[-1]][1])):
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert np.array_equal(s2, ref["a"][0]) and np.array_equal(s4, ref["a"][0])
        for got, name in zip(s5, seq):
            assert np.array_equal(got, ref[name][0])
    Pd = C.Plan(Wa, precision="mixed", device=True)
    with pytest.raises(C.Chi0Error) as ei:
        Pd.stage(C.HostInputs(Wb, pinned=False))
    assert ei.value.code == C.CHI0_EINVAL
    Pd.close()


def test_static_host_inputs_and_c64(C, O):
    W = wl.tiny_tb(n=6, norb=4, nq=2, seed=wl.SEED_BASE + 43, cdtype=np.complex64)
    ref = O.chi0(W)  # the oracle promotes the same complex64 values
    got_h = run_static(C, W, "fp64", device=False)
    got_d = run_static(C, W, "fp64", device=True)
    assert nerr(got_h[:, None], ref[:, None]) < 1e-12
    assert np.array_equal(got_h, got_d)


def test_static_custom_tetra_list(C, O):
    W = wl.tiny_tb(n=6, norb=4, nq=2, seed=wl.SEED_BASE + 44)
    rng = np.random.default_rng(3)
    tet = rng.integers(0, W.ncorner, size=(500, 4)).astype(np.int32)
    vol = rng.uniform(1e-4, 1e-3, 500)
    ref = np.array([O.chi0_q(W, q, tet=tet, tvol=vol) for q in W.qs])
    got = run_static(C, W, "fp64", tetra=(tet, vol))
    assert nerr(got[:, None], ref[:, None]) < 1e-12


def test_static_sign_and_cma(C, O):
    W = wl.tiny_tb(n=6, norb=4, nq=2, seed=wl.SEED_BASE + 45)
    pos = run_static(C, W, "fp64")
    neg = run_static(C, W, "fp64", sign=C.CHI0_SIGN_PAPER)
    assert np.array_equal(pos, -neg)
    W.cma = True
    ref = O.chi0(W)
    got = run_static(C, W, "fp64")
    assert nerr(got[:, None], ref[:, None]) < 1e-12


def test_static_deterministic(C):
    W = wl.tiny_tb(n=10, norb=5, nq=2, seed=wl.SEED_BASE + 46)
    a = run_static(C, W, "mixed")
    b = run_static(C, W, "mixed")
    assert np.array_equal(a, b)


# ------------------------------------------------------------------------ dynamic
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dynamic_tb(C, O, prec):
    W = wl.tiny_tb(n=8, norb=4, nq=2, seed=wl.SEED_BASE + 47)
    omega = np.concatenate([np.linspace(0.0, 3.0, 61), [-0.7, -1.9]])
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    gr, gi = run_dynamic(C, W, prec, omega)
    assert nerr(gr, np.array(ref_r)) < TOL[prec]
    assert nerr(gi, np.array(ref_i)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dynamic_far_field_boxes(C, O, prec):
    """A 12^3 mesh and 96 frequencies in [0, 2]: most final tetrahedra are narrow next to
    u_max/32, so their principal-value terms go to boxes of D (fine boxes inside the frequency
    range, geometric ones beyond it); every frequency against the oracle, and the counter
    shows that the boxes were used."""
    W = wl.tiny_tb(n=12, norb=4, nq=2, seed=wl.SEED_BASE + 49)
    omega = np.linspace(0.0, 2.0, 96)
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    P = C.Plan(W, precision=prec, device=True, profile=True)
    gr, gi = P.dynamic(omega)
    cnt = P.counters()
    P.close()
    assert cnt["box_pieces"] > 0.25 * cnt["pieces"], cnt
    assert nerr(gr.cpu().numpy(), np.array(ref_r)) < TOL[prec]
    assert nerr(gi.cpu().numpy(), np.array(ref_i)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dynamic_boxes_match_direct_evaluation(C, prec):
    """The same q on 64 frequencies, once as one pass (boxes stand in for far frequencies) and
    once one frequency per call (a single frequency never uses boxes): the two algorithms
    agree to the form's tolerance, negative frequencies included."""
    W = wl.tiny_tb(n=10, norb=5, nq=1, seed=wl.SEED_BASE + 50)
    omega = np.concatenate([np.linspace(0.0, 2.5, 60), [-0.3, -1.1, -2.0, 2.2]])
    P = C.Plan(W, precision=prec, device=True, profile=True)
    gr, gi = P.dynamic(omega)
    assert P.counters()["box_pieces"] > 0
    dr, di = zip(*[P.dynamic(omega[i:i + 1]) for i in range(omega.size)])
    P.close()
    dr = np.concatenate([x.cpu().numpy() for x in dr], axis=1)
    di = np.concatenate([x.cpu().numpy() for x in di], axis=1)
    assert nerr(gr.cpu().numpy(), dr) < TOL[prec]
    assert nerr(gi.cpu().numpy(), di) < TOL[prec]


def test_dynamic_many_frequencies_and_gamma(C, O):
    # 300 frequencies: two passes of the frequency loop; Gamma adds N(eF) at w = 0
    W = wl.tiny_tb(n=6, norb=3, nq=0, seed=wl.SEED_BASE + 48)
    W.qs = [wl.QPoint(shift=(0, 0, 0), gamma=True), wl.QPoint(shift=(2, 1, 0))]
    omega = np.linspace(0.0, 4.0, 300)
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    gr, gi = run_dynamic(C, W, "fp64", omega)
    assert nerr(gr, np.array(ref_r)) < 1e-12
    # at Gamma the interband |M|^2 vanish (orthogonal eigenvectors): Im is rounding noise
    # there, so Im is compared on the scale of the whole (q, w) table
    ref_i = np.array(ref_i)
    assert np.max(np.abs(gi - ref_i)) < 1e-12 * np.max(np.abs(ref_i))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dynamic_kk_route(C, O, prec):
    """Kramers-Kronig route (chi0_dynamic_kk): Im alone on a uniform grid that covers the
    spectrum (two passes: 300 nodes), against the oracle's Im at every node; Re against the
    oracle's transform of the oracle's Im (the device transform, independent code); and Re
    against the principal value of Eq. 1 within the grid's interpolation error."""
    W = wl.tiny_tb(n=8, norb=4, nq=0, seed=wl.SEED_BASE + 46)
    W.qs = [wl.QPoint(shift=(1, 2, 3)), wl.QPoint(shift=(0, 0, 0), gamma=True)]
    emax = float(W.E.max() - W.E.min()) + 0.5
    nkk = 300
    u = np.linspace(0.0, emax, nkk)
    P = C.Plan(W, precision=prec, device=True)
    re, im = P.dynamic_kk(emax, nkk)
    P.close()
    re, im = re.cpu().numpy(), im.cpu().numpy()
    ref_re, ref_im = O.chi0(W, omega=u)
    assert nerr(im[:1], ref_im[:1]) < TOL[prec], nerr(im[:1], ref_im[:1])
    # at Gamma this model has no interband weight below emax: Im is 0 up to rounding (~1e-31),
    # so the check there is absolute, against the size of Re
    assert np.max(np.abs(im[1] - ref_im[1])) < TOL[prec] * np.max(np.abs(ref_re[1]))
    kk = O.kk_re_from_im(u, ref_im[0], u)
    assert nerr(re[0], kk) < (1e-10 if prec == "fp64" else 1e-6), nerr(re[0], kk)
    # the route itself: second-order interpolation error of Im on this grid (oracle pin:
    # 1.8e-3 -> 2.5e-5 over four halvings on a 4^3 two-band model)
    assert nerr(re, ref_re) < 1e-2, nerr(re, ref_re)


def test_dynamic_free_electron_open_grid(C, O):
    W = wl.free_electron(10, 3, qmax_over_2kf=0.5)
    omega = np.linspace(0.0, 6.0, 40)
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    gr, gi = run_dynamic(C, W, "fp64", omega)
    assert nerr(gr, np.array(ref_r)) < 1e-12
    assert nerr(gi[1:], np.array(ref_i)[1:]) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_band_sweep_40_bands_windows(C, O, prec):
    """40-band random model (the band-truncation sweep's generator) on a 10^3 mesh: on-grid
    shifts with per-q windows of 4..40 bands around E_F, static and dynamic."""
    W = wl.band_sweep(n=10, nb=40, nq=4, nw=24)
    omega, W.omega = W.omega, None
    ref = O.chi0(W)
    got = run_static(C, W, prec)
    assert nerr(got[:, None], ref[:, None]) < TOL[prec]
    W.qs = W.qs[:2]
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    gr, gi = run_dynamic(C, W, prec, omega)
    assert nerr(gr, np.array(ref_r)) < TOL[prec]
    assert nerr(gi, np.array(ref_i)) < TOL[prec]


# ------------------------------------------------------------------------ graph mode
def test_graph_mode_replays_and_recaptures(C):
    """opts.graph: a call is captured into a CUDA graph and replayed by identical calls; a
    different call (other q list, dynamic instead of static) is captured anew.  Results are
    bitwise those of the plain launch sequence."""
    W = wl.tiny_tb(n=8, norb=5, nq=3, seed=wl.SEED_BASE + 64)
    ref_s = run_static(C, W, "mixed")
    omega = np.linspace(0.0, 2.0, 300)  # two frequency passes
    ref_r, ref_i = run_dynamic(C, W, "mixed", omega)
    P = C.Plan(W, precision="mixed", graph=True)
    for _ in range(3):
        got = P.static().cpu().numpy()
        assert np.array_equal(got, ref_s)
    for _ in range(2):
        gr, gi = P.dynamic(omega)
        assert np.array_equal(gr.cpu().numpy(), ref_r) and np.array_equal(gi.cpu().numpy(), ref_i)
    got = P.static().cpu().numpy()  # back to the static call: captured again
    assert np.array_equal(got, ref_s)
    k = P.counters()["kernels"]
    assert k > 0
    P.close()


# ------------------------------------------------------------------------ autotuner
def test_autotuner_picks_a_shape_and_keeps_results(C, O):
    """chi0_tune times the weight-kernel grids and the tensor-core corner packings on a call,
    keeps the fastest, and every later call still matches the oracle."""
    W = wl.band_sweep(n=8, nb=40, nq=3, nw=12)
    omega, W.omega = W.omega, None
    ref = O.chi0(W)
    P = C.Plan(W, precision="mixed", overlap="bf16x6")
    r = P.tune()
    assert r["candidates"] >= 3 and 0 < r["best_ms"] <= r["default_ms"]
    assert r["static_ctas_per_sm"] >= 1 and r["tc_corners_per_round"] >= 0  # 0: the most that fit
    got = P.static().cpu().numpy()
    assert nerr(got[:, None], ref[:, None]) < TOL["mixed"]
    W.qs = W.qs[:1]
    ref_r, ref_i = zip(*[O.chi0_q(W, q, omega=omega) for q in W.qs])
    P2 = C.Plan(W, precision="mixed", overlap="bf16x6")
    r = P2.tune(omega)
    assert r["dynamic_ctas_per_sm"] >= 1
    gr, gi = P2.dynamic(omega)
    assert nerr(gr.cpu().numpy(), np.array(ref_r)) < TOL["mixed"]
    assert nerr(gi.cpu().numpy(), np.array(ref_i)) < TOL["mixed"]
    P.close()
    P2.close()
