"""Pins of the FP64 CPU oracle against things other than itself.

Each check compares the oracle with an independent route: direct numerical
quadrature on the simplex, high-precision divided differences of the
definition, quasi-Monte-Carlo over the tetrahedron, closed forms
(free-electron Lindhard, its dynamic Im part, flat bands), sum rules and
exact symmetries.  None of them re-types the oracle's own algorithm.
"""
import math

import numpy as np
import pytest

from paper_1407_3444_gb300 import workloads as wl


# ------------------------------------------------------------------------------------------
# independent references
# ------------------------------------------------------------------------------------------
def simplex_quad(func, x, apex, n=48):
    """(1/V) * integral over the unit 3-simplex of func(lam) with collapsed (Duffy)
    coordinates; the vertex ``apex`` sits at the collapsed point so a 1/r singularity
    there is integrated smoothly."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    u, v, s = np.meshgrid(g, g, g, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]) * (1 - u) ** 2 * (1 - v)
    l_apex = u
    l_b = (1 - u) * v
    l_c = (1 - u) * (1 - v) * s
    l_d = (1 - u) * (1 - v) * (1 - s)
    others = [i for i in range(4) if i != apex]
    lam = [None] * 4
    lam[apex] = l_apex
    lam[others[0]] = l_b
    lam[others[1]] = l_c
    lam[others[2]] = l_d
    return 6.0 * np.sum(W * func(lam))


def dd_mpmath(knots, dps=220):
    """Fourth divided difference of x^3 ln|x| from its definition, in 220-digit arithmetic
    (repeated knots split by 1e-30)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    seen = {}
    kk = []
    for k in knots:
        c = seen.get(float(k), 0)
        seen[float(k)] = c + 1
        kk.append(mp.mpf(float(k)) + c * mp.mpf("1e-30"))
    s = mp.mpf(0)
    for i, ti in enumerate(kk):
        p = mp.mpf(1)
        for j, tj in enumerate(kk):
            if j != i:
                p *= ti - tj
        s += (ti ** 3 * mp.log(abs(ti)) if ti != 0 else 0) / p
    return float(s)


def sample_simplex(rng, n):
    e = rng.exponential(size=(n, 4))
    return e / e.sum(axis=1, keepdims=True)


def qmc_simplex(m, seed=0):
    from scipy.stats import qmc
    u = qmc.Sobol(d=3, scramble=True, seed=seed).random_base2(m)
    # uniform simplex from the unit cube: sorted-coordinate spacings
    s = np.sort(u, axis=1)
    return np.stack([s[:, 0], s[:, 1] - s[:, 0], s[:, 2] - s[:, 1], 1.0 - s[:, 2]], axis=1)


def lindhard(x):
    x = float(x)
    if x == 0.0:
        return 1.0
    if x == 1.0:
        return 0.5
    return 0.5 + (1 - x * x) / (4 * x) * math.log(abs((1 + x) / (1 - x)))


# ------------------------------------------------------------------------------------------
# single-tetrahedron weights
# ------------------------------------------------------------------------------------------
def test_inv_weight_vs_simplex_quadrature(oracle_mod):
    rng = np.random.default_rng(11)
    for trial in range(12):
        if trial % 3 == 0:
            x = rng.uniform(0.2, 5.0, 4)
        elif trial % 3 == 1:
            x = 1.5 + rng.uniform(-1e-2, 1e-2, 4)          # clustered knots
        else:
            x = np.array([0.0, *rng.uniform(0.3, 2.0, 3)])   # one vertex with D = 0
        apex = int(np.argmin(x))
        for j in range(4):
            ref = simplex_quad(lambda L: L[j] / (L[0] * x[0] + L[1] * x[1] + L[2] * x[2] + L[3] * x[3]), x, apex)
            got = oracle_mod.inv_weight(x, j)
            assert abs(got - ref) <= 1e-11 * abs(ref), (x, j, got, ref)


def test_inv_weight_vs_definition_all_regimes(oracle_mod):
    rng = np.random.default_rng(12)
    cases = []
    for _ in range(40):
        cases.append(rng.uniform(0.05, 4.0, 4))                        # well separated
        cases.append(2.0 + rng.uniform(-1e-6, 1e-6, 4))                 # tight cluster
        cases.append(np.array([1.0, 1.0 + 1e-9, 3.0, rng.uniform(0, 1)]))  # sub-cluster
        cases.append(np.array([0.0, 0.0, *rng.uniform(0.1, 1.0, 2)]))  # D = 0 edge
        cases.append(rng.uniform(-2.0, 3.0, 4))                         # principal value
    cases.append(np.array([1.0, 1.0, 1.0, 1.0]))
    cases.append(np.array([0.0, 2.0, 2.0, 2.0]))
    for x in cases:
        s = np.max(np.abs(x))
        for j in range(4):
            ref = dd_mpmath(list(x) + [x[j]])
            got = oracle_mod.inv_weight(x, j)
            # absolute error on the scale 1/max|x| of the weight (PV results can cancel to ~0)
            assert abs(got - ref) * s <= 2e-13 + 1e-12 * abs(ref) * s, (x, j, got, ref)


def test_inv_weight_sum_rule(oracle_mod):
    """sum_j x_j (1/V) int lambda_j / X = (1/V) int X/X = 1 (also across X = 0, PV)."""
    rng = np.random.default_rng(13)
    for _ in range(200):
        x = rng.uniform(-1.0, 4.0, 4) if _ % 2 else rng.uniform(0.0, 4.0, 4)
        tot = sum(x[j] * oracle_mod.inv_weight(x, j) for j in range(4))
        assert abs(tot - 1.0) < 1e-12


def test_inv_weight_flat(oracle_mod):
    """constant X = c: (1/V) int lambda_j / c = 1/(4c)"""
    for c in (0.3, 1.0, 7.5, -2.0):
        for j in range(4):
            assert abs(oracle_mod.inv_weight([c] * 4, j) - 0.25 / c) < 1e-15 / abs(c)


def test_mspline_vs_truncated_power_and_moments(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(14)
    for _ in range(20):
        t = np.sort(rng.uniform(0.0, 2.0, 5))
        # Curry-Schoenberg: M(x) = 4 * (. - x)_+^3 [t0..t4] for distinct knots
        for x in rng.uniform(t[0], t[-1], 5):
            s = mp.mpf(0)
            for i in range(5):
                p = mp.mpf(1)
                for j in range(5):
                    if j != i:
                        p *= mp.mpf(t[i]) - mp.mpf(t[j])
                s += max(mp.mpf(t[i]) - mp.mpf(x), 0) ** 3 / p
            assert abs(oracle_mod.mspline(t, x) - 4 * float(s)) < 1e-10 * max(1.0, 4 * abs(float(s)))
        xs = np.linspace(t[0], t[-1], 40001)
        M = np.array([oracle_mod.mspline(t, x) for x in xs])
        assert abs(np.trapezoid(M, xs) - 1.0) < 1e-6
        assert abs(np.trapezoid(M * xs, xs) - t.mean()) < 1e-6


def test_delta_weight_vs_monte_carlo(oracle_mod):
    """(1/V) int lambda_j delta(w - D): histogram of D weighted by lambda_j."""
    rng = np.random.default_rng(15)
    d = np.array([0.3, 1.1, 0.7, 1.9])
    L = sample_simplex(rng, 4_000_000)
    D = L @ d
    edges = np.linspace(0.3, 1.9, 33)
    for j in range(4):
        hist, _ = np.histogram(D, bins=edges, weights=L[:, j])
        dens = hist / len(D) / np.diff(edges)
        mids = 0.5 * (edges[1:] + edges[:-1])
        # bin average of the oracle density by fine quadrature
        ref = []
        for a, b in zip(edges[:-1], edges[1:]):
            xs = np.linspace(a, b, 41)
            ref.append(np.trapezoid([oracle_mod.delta_weight(d, j, x) for x in xs], xs) / (b - a))
        ref = np.array(ref)
        assert np.max(np.abs(dens - ref)) < 0.01 * np.max(ref), (j, dens, ref)
        del mids


# ------------------------------------------------------------------------------------------
# carving
# ------------------------------------------------------------------------------------------
def _signs(rng, nneg):
    v = rng.uniform(0.1, 1.0, 4)
    s = np.ones(4)
    s[rng.permutation(4)[:nneg]] = -1
    return v * s


def test_carving_volume_all_cases(oracle_mod):
    rng = np.random.default_rng(16)
    L = sample_simplex(rng, 2_000_000)
    for na in range(5):          # occupied corners (a < 0)
        for nb in range(5):      # empty corners (b > 0)
            a = _signs(rng, na)
            b = -_signs(rng, nb)
            vol, D, F = oracle_mod.carve(a, b)
            assert len(vol) <= 9
            if na == 0 or nb == 0:
                assert vol.sum() == 0.0
            A = L @ a
            B = L @ b
            inside = (A < 0) & (B > 0)
            p = inside.mean()
            sig = math.sqrt(max(p * (1 - p), 1e-12) / len(L))
            assert abs(vol.sum() - p) < 6 * sig + 1e-12, (na, nb, vol.sum(), p)
            # the mean of D over the region: sum_S V_S mean(d_S) vs Monte Carlo
            if p > 0.01:
                ref = np.mean(np.where(inside, B - A, 0.0))
                got = float(np.sum(vol * D.mean(axis=1)))
                assert abs(got - ref) < 0.01 * abs(ref) + 1e-4, (na, nb, got, ref)
            assert np.all(D >= 0.0)


def test_carving_single_cut_closed_forms(oracle_mod):
    """One occupied corner: volume = product of the edge fractions a0/(a0-aj); three
    occupied corners: 1 - product of the fractions from the empty corner."""
    rng = np.random.default_rng(17)
    b = np.full(4, 1.0)  # everything empty at k+q: only the first cut acts
    for _ in range(50):
        a = np.array([-rng.uniform(0.1, 1), *rng.uniform(0.1, 1, 3)])
        vol, _, _ = oracle_mod.carve(a, b)
        ref = np.prod(a[0] / (a[0] - a[1:]))
        assert abs(vol.sum() - ref) < 1e-14
        a3 = np.array([*(-rng.uniform(0.1, 1, 3)), rng.uniform(0.1, 1)])
        vol, _, _ = oracle_mod.carve(a3, b)
        ref = 1.0 - np.prod(a3[3] / (a3[3] - a3[:3]))
        assert abs(vol.sum() - ref) < 1e-14


def test_tet_static_integral_vs_qmc(oracle_mod):
    rng = np.random.default_rng(18)
    L = qmc_simplex(20, seed=3)
    for _ in range(6):
        a = rng.uniform(-1.0, 0.6, 4)
        b = rng.uniform(-0.4, 1.2, 4) + 0.8
        f = rng.uniform(0.0, 1.0, 4)
        got = oracle_mod.tet_integrals(a, b, f)
        A, B, Fv = L @ a, L @ b, L @ f
        ref = np.mean(np.where((A < 0) & (B > 0), 2.0 * Fv / np.maximum(B - A, 1e-300), 0.0))
        assert abs(got - ref) < 2e-3 * abs(ref), (got, ref)


def test_tet_dynamic_integrals_identities(oracle_mod):
    """Re at w = 0 equals the static value; Re is even in w; Im is odd (Eq. 3);
    int_0^inf Im dw = pi int_R f and int_0^inf Im/w dw = (pi/2) * static (exact)."""
    rng = np.random.default_rng(19)
    a = np.array([-0.9, -0.2, 0.3, -0.5])
    b = np.array([0.8, -0.1, 1.4, 0.6])
    f = rng.uniform(0.2, 1.0, 4)
    stat = oracle_mod.tet_integrals(a, b, f)
    re0, im0 = oracle_mod.tet_integrals(a, b, f, [0.0])
    assert abs(re0[0] - stat) < 1e-14 * abs(stat) and im0[0] == 0.0
    w = np.array([0.37, 1.3])
    rp, ip = oracle_mod.tet_integrals(a, b, f, w)
    rm, im_ = oracle_mod.tet_integrals(a, b, f, -w)
    assert np.allclose(rp, rm, rtol=0, atol=1e-14) and np.allclose(ip, -im_, rtol=0, atol=1e-14)
    dmax = float(np.max(b - a)) + 0.01
    n = 20000
    ws = (np.arange(n) + 0.5) * dmax / n
    _, im = oracle_mod.tet_integrals(a, b, f, ws)
    vol, D, F = oracle_mod.carve(a, b, f)
    int_f = float(np.sum(vol * F.mean(axis=1)))
    assert abs(np.sum(im) * dmax / n - math.pi * int_f) < 1e-4 * math.pi * int_f
    assert abs(np.sum(im / ws) * dmax / n - 0.5 * math.pi * stat) < 1e-3 * stat


# ------------------------------------------------------------------------------------------
# whole chi0: closed forms, limits and symmetries
# ------------------------------------------------------------------------------------------
def _lindhard_err(oracle_mod, n, nq=5):
    W = wl.free_electron(n, nq)
    chi = oracle_mod.chi0(W)
    N = W.meta["dos_ef"]
    return np.array([chi[i] / N - lindhard(x) for i, x in enumerate(W.meta["x"])])


def test_free_electron_lindhard_static(oracle_mod):
    """chi0/N(eF) -> 1/2 + (1-x^2)/(4x) ln|(1+x)/(1-x)|, x = q/2kF, with ~4x smaller error
    per doubling of the grid (linear interpolation, second order)."""
    e16 = _lindhard_err(oracle_mod, 16)
    e32 = _lindhard_err(oracle_mod, 32)
    assert np.all(np.abs(e32[:4]) < 3e-3), e32
    assert np.all(np.abs(e32[:4]) < np.abs(e16[:4]) / 2.5), (e16, e32)
    assert abs(e32[4]) < 1.2e-2  # x = 1 (log kink), first-order convergence there


def test_free_electron_q0_limit(oracle_mod):
    """chi0(q=0) = N(eF) (Sec. III), here k_F/pi^2 per bohr^3."""
    errs = []
    for n in (16, 32, 64):
        W = wl.free_electron(n, 1)
        errs.append(oracle_mod.chi0(W)[0] / W.meta["dos_ef"] - 1.0)
    assert abs(errs[-1]) < 5e-4
    assert abs(errs[1]) < abs(errs[0]) / 3 and abs(errs[2]) < abs(errs[1]) / 3


def test_free_electron_axis_cycle(oracle_mod):
    """The (000)-(111) cube split is symmetric under the cyclic axis permutation, so
    chi0(q x) = chi0(q y) = chi0(q z) to rounding."""
    vals = []
    for ax in range(3):
        W = wl.free_electron(12, 3, qmax_over_2kf=0.6, axis=ax)
        vals.append(oracle_mod.chi0_q(W, W.qs[2]))
    assert abs(vals[0] - vals[1]) < 1e-13 * vals[0] and abs(vals[0] - vals[2]) < 1e-13 * vals[0]


def test_free_electron_dynamic_im(oracle_mod):
    """Im chi0 of the free electron gas (Eq. 2 integrated over planes normal to q):
    (1/(4 pi q)) [(kF^2 - (w/q - q/2)^2)_+ - (kF^2 - (w/q + q/2)^2)_+]."""
    errs = []
    for n in (16, 32):
        W = wl.free_electron(n, 3, qmax_over_2kf=0.5)
        q = W.qs[1]
        qa = W.meta["q_abs"][1]
        kF = W.meta["kF"]
        w = np.array([0.3, 1.0, 2.0, 3.0])
        _, im = oracle_mod.chi0_q(W, q, omega=w)
        ref = (np.maximum(kF ** 2 - (w / qa - qa / 2) ** 2, 0) - np.maximum(kF ** 2 - (w / qa + qa / 2) ** 2, 0)) / (4 * math.pi * qa)
        errs.append(np.max(np.abs(im - ref)) / np.max(ref))
    assert errs[1] < 0.02 and errs[1] < errs[0] / 1.8, errs


def test_flat_bands_matrix_element_closed_form(oracle_mod):
    """Three flat bands -1, +1, +2 (eF = 0) with eigenvectors U at k and V at k+q: the pairs
    are (m=0, n=1) with D = 2 and (0, 2) with D = 3, so (Eq. 1, M_mn = <m,k|n,k+q>)
    chi0 = 2 [f01 2/2 + f02 2/3] and Re chi0(w) = 2 sum_n f0n (1/(D-w) + 1/(D+w))."""
    rng = np.random.default_rng(21)
    n = 3
    Nc = n ** 3

    def unitary():
        Z = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        Q, _ = np.linalg.qr(Z)
        return Q

    U, V = unitary(), unitary()
    E = np.tile([-1.0, 1.0, 2.0], (Nc, 1))
    W = wl.Workload("flat", (n, n, n), True, 3, 3, E, np.tile(U, (Nc, 1, 1)), 0.0, (0, 3), False,
                    [wl.QPoint(Eq=E.copy(), Cq=np.tile(V, (Nc, 1, 1)))])
    f = np.abs(U.conj().T @ V) ** 2          # f[m, n] = |sum_o conj(U_om) V_on|^2
    assert abs(f[0, 1] - f[1, 0]) > 1e-3 and abs(f[0, 2] - f[2, 0]) > 1e-3
    ref = 2.0 * (f[0, 1] * 2 / 2 + f[0, 2] * 2 / 3)
    got = oracle_mod.chi0_q(W, W.qs[0])
    assert abs(got - ref) < 1e-13
    w = np.array([0.5, 1.5, 2.5])
    re, im = oracle_mod.chi0_q(W, W.qs[0], omega=w)
    refw = 2.0 * (f[0, 1] * (1 / (2 - w) + 1 / (2 + w)) + f[0, 2] * (1 / (3 - w) + 1 / (3 + w)))
    assert np.allclose(re, refw, rtol=1e-13, atol=0)
    assert np.all(im == 0.0)
    # the paper's printed sign
    assert abs(oracle_mod.chi0_q(W, W.qs[0], sign=1) + ref) < 1e-13


def test_chi_even_in_q(oracle_mod):
    """t(-R) = t(R): H(k) even, so chi0(q) = chi0(-q) (inversion-symmetric mesh)."""
    m = wl.random_model(3, wl.SEED_BASE + 31, spread=4.0)
    n = 4
    kf = wl.corner_frac((n, n, n), True)
    E, C = m.eig(kf)
    ef = wl.fermi_level(E, 1.5)
    q = np.array([0.13, -0.21, 0.07])
    qp = wl.explicit_q(m, (n, n, n), q)
    qm = wl.explicit_q(m, (n, n, n), -q)
    W = wl.Workload("t", (n, n, n), True, 3, 3, E, C, ef, (0, 3), False, [qp, qm])
    a = oracle_mod.chi0_q(W, qp)
    b = oracle_mod.chi0_q(W, qm)
    assert abs(a - b) < 1e-12 * abs(a)
    ra, ia = oracle_mod.chi0_q(W, qp, omega=[0.4, 1.1])
    rb, ib = oracle_mod.chi0_q(W, qm, omega=[0.4, 1.1])
    assert np.allclose(ra, rb, rtol=1e-12, atol=0) and np.allclose(ia, ib, rtol=1e-12, atol=1e-15)


def test_diagonal_unitary_model_is_sum_of_bands(oracle_mod):
    """Eigenvectors C(k) = U fixed: |M_mn|^2 = delta_mn, so chi0 equals the sum over
    bands of the single-band (intraband) chi0 with |M|^2 = 1."""
    rng = np.random.default_rng(22)
    n = 4
    kf = wl.corner_frac((n, n, n), True)
    Z = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    U, _ = np.linalg.qr(Z)
    disp = lambda k, s: s[0] + s[1] * np.cos(2 * np.pi * k[:, 0]) + s[2] * np.cos(2 * np.pi * k[:, 1]) + s[3] * np.cos(2 * np.pi * k[:, 2])
    pars = [(-3.0, 0.4, 0.3, 0.2), (0.0, 0.5, -0.6, 0.4), (3.0, 0.3, 0.2, -0.5)]
    q = np.array([0.2, 0.05, -0.1])
    E = np.stack([disp(kf, p) for p in pars], axis=1)
    Eq = np.stack([disp(kf + q, p) for p in pars], axis=1)
    C = np.tile(U, (kf.shape[0], 1, 1))
    W = wl.Workload("diag", (n, n, n), True, 3, 3, E, C, 0.1, (0, 3), False,
                    [wl.QPoint(Eq=Eq, Cq=C.copy())])
    full = oracle_mod.chi0_q(W, W.qs[0])
    parts = 0.0
    for b in range(3):
        Wb = wl.Workload("b", (n, n, n), True, 1, 1, E[:, b:b + 1].copy(), None, 0.1, (0, 1), True,
                         [wl.QPoint(Eq=Eq[:, b:b + 1].copy())])
        parts += oracle_mod.chi0_q(Wb, Wb.qs[0])
    assert abs(full - parts) < 1e-12 * abs(parts)


def test_completeness_full_window(oracle_mod):
    """With the full band window, sum_n |M_mn|^2 = 1: chi0 with all flat-shifted empty
    bands collapses to the CMA value of one empty band per occupied band."""
    rng = np.random.default_rng(23)
    n = 3
    Nc = n ** 3
    m = wl.random_model(3, wl.SEED_BASE + 33, spread=2.0)
    kf = wl.corner_frac((n, n, n), True)
    _, C = m.eig(kf)
    _, Cq = m.eig(kf + np.array([0.11, 0.0, 0.0]))
    # occupied band 0 at -1, empty bands 1, 2 both at +1 -> D = 2 for (0,1) and (0,2)
    E = np.tile([-1.0, 1.0, 1.0], (Nc, 1))
    W = wl.Workload("c", (n, n, n), True, 3, 3, E, C, 0.0, (0, 3), False, [wl.QPoint(Eq=E.copy(), Cq=Cq)])
    got = oracle_mod.chi0_q(W, W.qs[0])
    f00 = np.mean(np.abs(np.einsum("ko,ko->k", C[:, :, 0].conj(), Cq[:, :, 0])) ** 2)
    # chi0 = 2 * sum_{n=1,2} <|M_0n|^2> * 2/2 = 2 * (1 - <|M_00|^2>)
    assert abs(got - 2.0 * (1.0 - f00)) < 1e-12


def test_brute_force_tiny_model(oracle_mod):
    """Route C: quasi-Monte-Carlo over every tetrahedron of a 2-band 3^3 model."""
    W = wl.tiny_tb(n=3, norb=2, nq=1, filling=1.0)
    q = W.qs[0]
    got = oracle_mod.chi0_q(W, q)
    L = qmc_simplex(14, seed=5)
    n = 3
    N = n
    cid = lambda i, j, k: ((i % N) * N + (j % N)) * N + (k % N)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tot = 0.0
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for p in perms:
                    o = [0, 0, 0]
                    cs = [cid(i, j, k)]
                    o[p[0]] = 1
                    cs.append(cid(i + o[0], j + o[1], k + o[2]))
                    o[p[1]] = 1
                    cs.append(cid(i + o[0], j + o[1], k + o[2]))
                    cs.append(cid(i + 1, j + 1, k + 1))
                    for mb in range(2):
                        for nb in range(2):
                            a = W.E[cs, mb] - W.ef
                            b = q.Eq[cs, nb] - W.ef
                            f = np.abs(np.einsum("co,co->c", W.C[cs, :, mb].conj(), q.Cq[cs, :, nb])) ** 2
                            A, B, F = L @ a, L @ b, L @ f
                            tot += np.mean(np.where((A < 0) & (B > 0), 2 * F / np.maximum(B - A, 1e-300), 0.0))
    ref = 2.0 * tot / (6 * n ** 3)
    assert abs(got - ref) < 3e-3 * abs(ref), (got, ref)


def test_static_vs_dynamic_at_zero_and_kk(oracle_mod):
    """Re chi0(w=0) of the dynamic route equals the static value, and the Kramers-Kronig
    integral (2/pi) int_0^inf Im(w)/w dw reproduces the static chi0."""
    W = wl.tiny_tb(n=3, norb=2, nq=1, filling=1.0)
    q = W.qs[0]
    stat = oracle_mod.chi0_q(W, q)
    re0, _ = oracle_mod.chi0_q(W, q, omega=[0.0])
    assert abs(re0[0] - stat) < 1e-13 * stat
    dmax = float(np.max(q.Eq) - np.min(W.E)) + 0.01
    nw = 3000
    ws = (np.arange(nw) + 0.5) * dmax / nw
    _, im = oracle_mod.chi0_q(W, q, omega=ws)
    kk = (2 / math.pi) * np.sum(im / ws) * dmax / nw
    assert abs(kk - stat) < 2e-3 * stat, (kk, stat)


def _carved_volume(oracle_mod, n, kF, q, L=1.0):
    """Volume of {|k|^2 < kF^2, |k+q|^2 > kF^2} in the cube [-L, L]^3 from the oracle's
    carving of the linear interpolants on n^3 cubes (6 tetrahedra each)."""
    h = 2.0 * L / n
    perm = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tot = 0.0
    for i0 in range(n):
        for i1 in range(n):
            for i2 in range(n):
                base = np.array([i0, i1, i2]) * h - L
                for p in perm:
                    o = np.zeros(3)
                    cs = [base.copy()]
                    o[p[0]] += h
                    cs.append(base + o)
                    o[p[1]] += h
                    cs.append(base + o)
                    cs.append(base + h)
                    cs = np.array(cs)
                    a = (cs ** 2).sum(1) - kF ** 2
                    b = ((cs + q) ** 2).sum(1) - kF ** 2
                    if a.min() >= 0 or b.max() <= 0:
                        continue
                    vol, _, _ = oracle_mod.carve(a, b)
                    tot += vol.sum() * h ** 3 / 6.0
    return tot


def test_fig1_worked_example_carved_volume(oracle_mod):
    """Sec. II, Fig. 1: parabolic band eps = |k|^2, q = (0.15, 0, 0), k_F = 0.77.  The doubly
    carved region is the Fermi ball minus its lens-shaped overlap with the shifted ball
    (closed form stored in tests/golden/fig1_parabolic_carving.json by make_golden.py).  The
    oracle's carving of the linear interpolants converges to it at second order."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig1_parabolic_carving.json")))
    kF, q, exact = g["kF"], np.array(g["q"]), g["carved_volume"]
    v = {n: _carved_volume(oracle_mod, n, kF, q) for n in (12, 24, 48)}
    e = {n: v[n] - exact for n in v}
    assert 3.3 < e[12] / e[24] < 4.8 and 3.3 < e[24] / e[48] < 4.8, e
    rich = (4.0 * v[48] - v[24]) / 3.0
    assert abs(rich - exact) < 3e-4 * exact, (rich, exact)


def test_chi_periodic_in_q(oracle_mod):
    """Orbitals at the cell origin (periodic gauge): H(k + G) = H(k), so chi0(q + G) = chi0(q),
    with the constant matrix element and with the full |M|^2 (CMA periodicity, Sec. III)."""
    m = wl.random_model(3, wl.SEED_BASE + 32, spread=4.0)
    n = 4
    kf = wl.corner_frac((n, n, n), True)
    E, C = m.eig(kf)
    ef = wl.fermi_level(E, 1.5)
    q = np.array([0.13, -0.21, 0.07])
    q0 = wl.explicit_q(m, (n, n, n), q)
    qG = wl.explicit_q(m, (n, n, n), q + np.array([1.0, -1.0, 2.0]))
    for cma in (True, False):
        W = wl.Workload("t", (n, n, n), True, 3, 3, E, C, ef, (0, 3), cma, [q0, qG])
        a = oracle_mod.chi0_q(W, q0)
        b = oracle_mod.chi0_q(W, qG)
        assert abs(a - b) < 1e-10 * abs(a), (cma, a, b)


def test_pairs_flat_bands_closed_form(oracle_mod):
    """Band-pair resolved static chi0 (Sec. III, Fig. 8) on three flat bands -1, +1, +2 (eF = 0)
    with eigenvectors U at k and V at k+q: only the pairs (0, 1) and (0, 2) carry weight,
    2 f01 2/2 and 2 f02 2/3 with f = |U^H V|^2 (M_mn = <m,k|n,k+q>, Eq. 1); the transposed
    entries (1, 0), (2, 0) are 0 (band 1 and 2 are empty at k), which a transposed operand or
    a swapped m/n in the accumulation index would break."""
    rng = np.random.default_rng(22)
    n = 3
    Nc = n ** 3

    def unitary():
        Z = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        Q, _ = np.linalg.qr(Z)
        return Q

    U, V = unitary(), unitary()
    E = np.tile([-1.0, 1.0, 2.0], (Nc, 1))
    W = wl.Workload("flat", (n, n, n), True, 3, 3, E, np.tile(U, (Nc, 1, 1)), 0.0, (0, 3), False,
                    [wl.QPoint(Eq=E.copy(), Cq=np.tile(V, (Nc, 1, 1)))])
    f = np.abs(U.conj().T @ V) ** 2
    P = oracle_mod.chi0_pairs_q(W, W.qs[0])
    ref = np.zeros((3, 3))
    ref[0, 1] = 2.0 * f[0, 1] * 2 / 2
    ref[0, 2] = 2.0 * f[0, 2] * 2 / 3
    assert np.allclose(P, ref, rtol=1e-13, atol=1e-15)
    assert abs(oracle_mod.chi0_pairs_q(W, W.qs[0], sign=1)[0, 2] + ref[0, 2]) < 1e-14


def test_pairs_add_up_to_chi0(oracle_mod):
    """The band-pair contributions of a q add up to its static chi0, at a general q and at
    Gamma (where the intraband pairs carry the density of states of their band, Sec. III)."""
    m = wl.random_model(4, wl.SEED_BASE + 41, spread=4.0)
    n = 4
    E, C = m.eig_grid((n, n, n))
    ef = wl.fermi_level(E, 2.0)
    qs = [wl.QPoint(shift=(1, 2, 0), frac=(0.25, 0.5, 0.0)),
          wl.QPoint(shift=(0, 0, 0), gamma=True, frac=(0.0, 0.0, 0.0))]
    W = wl.Workload("tiny", (n, n, n), True, 4, 4, E, C, ef, (0, 4), False, qs)
    for q in qs:
        P = oracle_mod.chi0_pairs_q(W, q)
        tot = oracle_mod.chi0_q(W, q)
        assert P.shape == (4, 4)
        assert abs(P.sum() - tot) <= 1e-12 * abs(tot), (P.sum(), tot)
    # at Gamma every diagonal entry is the DOS of its band (intraband transitions have no
    # region of their own there), which equals the oracle's DOS of that band alone
    Pg = oracle_mod.chi0_pairs_q(W, qs[1])
    for b in range(4):
        dos_b = oracle_mod.chi0_q(W, qs[1], window=(b, b + 1))
        assert abs(Pg[b, b] - dos_b) <= 1e-12 * max(1.0, abs(dos_b)), (b, Pg[b, b], dos_b)


def test_kk_transform_matches_cauchy_quadrature(oracle_mod):
    """The Kramers-Kronig transform of a piecewise-linear Im (Re(w) = (1/pi) PV int_0^inf Im(u)
    [1/(u - w) + 1/(u + w)] du) against scipy's Cauchy-weight quadrature of the same
    interpolant, at nodes (where adjacent segments' singular parts cancel), between nodes, at
    w = 0 and past the last node."""
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(9)
    u = np.concatenate([[0.0], np.sort(rng.uniform(0.05, 2.0, 14))])
    im = np.concatenate([[0.0], rng.uniform(-0.3, 1.0, 14)])
    uu = np.append(u, u[-1] + (u[-1] - u[-2]))
    yy = np.append(im, 0.0)

    def interp(x):
        return np.interp(x, uu, yy)

    ws = np.array([0.0, u[3], 0.5 * (u[5] + u[6]), u[-1], uu[-1] + 0.3, 0.77])
    got = oracle_mod.kk_re_from_im(u, im, ws)
    for wv, g in zip(ws, got):
        tot = 0.0
        for j in range(len(uu) - 1):
            a, b = uu[j], uu[j + 1]
            for c in (wv, -wv):
                if a < c < b:
                    v, _ = integrate.quad(interp, a, b, weight="cauchy", wvar=c, epsabs=1e-13, epsrel=1e-12)
                elif c == a or c == b:
                    # split off the node: PV over the pair of adjacent segments is taken by the
                    # symmetric limit; integrate (Im(u) - Im(c)) / (u - c) regularly plus Im(c) log
                    f = lambda x, c=c: (interp(x) - interp(c)) / (x - c) if x != c else 0.0
                    v, _ = integrate.quad(f, a, b, epsabs=1e-13, epsrel=1e-12, limit=200)
                    v += interp(c) * (math.log(abs(b - c)) if b != c else 0.0) - interp(c) * (math.log(abs(a - c)) if a != c else 0.0)
                else:
                    v, _ = integrate.quad(lambda x, c=c: interp(x) / (x - c), a, b, epsabs=1e-13, epsrel=1e-12)
                tot += v
        ref = tot / math.pi
        assert abs(g - ref) <= 1e-9 * max(1.0, abs(ref)), (wv, g, ref)


def test_kk_route_converges_to_principal_value(oracle_mod):
    """Sec. II's usual route: Re from Im by Kramers-Kronig on a grid that covers Im's whole
    support approaches the principal value of Eq. 1 as the grid is refined (two-band model)."""
    W = wl.tiny_tb(n=4, norb=2, nq=1, filling=1.0)
    q = W.qs[0]
    emax = float(W.E.max() - W.E.min()) + 0.5
    ws = np.array([0.3, 0.9, 1.7])
    re_pv, _ = oracle_mod.chi0_q(W, q, omega=ws)
    errs = []
    for m in (129, 513):
        u = np.linspace(0.0, emax, m)
        _, im = oracle_mod.chi0_q(W, q, omega=u)
        re_kk = oracle_mod.kk_re_from_im(u, im, ws)
        errs.append(np.max(np.abs(re_kk - re_pv)) / np.max(np.abs(re_pv)))
    assert errs[1] < 0.5 * errs[0] and errs[1] < 2e-2, errs


def test_kq_interpolation_on_grid_and_linear(oracle_mod):
    """Linear interpolation of the data at k+q (Sec. II): an on-grid q returns the mesh data at
    the shifted corner (eigenvectors up to their phase), and a k-linear quantity is reproduced
    exactly wherever k+q stays inside the mesh's unwrapped part."""
    W = wl.tiny_tb(n=5, norb=3, nq=0, seed=wl.SEED_BASE + 51)
    n = 5
    Eq, Cq = oracle_mod.kq_interpolate(W, (2 / n, 1 / n, 3 / n))
    idx = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)])
    sh = ((idx[:, 0] + 2) % n * n + (idx[:, 1] + 1) % n) * n + (idx[:, 2] + 3) % n
    assert np.array_equal(Eq, W.E[sh])
    ov = np.abs(np.sum(np.conj(W.C[sh]) * Cq, axis=1))       # |<v(k+q)|interpolated>| per band
    assert np.allclose(ov, 1.0, atol=1e-12)
    # k-linear energies: E = a . (i, j, k) + b per band; q small enough that no corner
    # below the last plane wraps
    a = np.array([0.3, -0.7, 1.1])
    Wl = wl.Workload("lin", (n, n, n), True, 2, 2, np.stack([idx @ a, idx @ a + 2.0], axis=1), None, 0.5,
                     (0, 2), True, [])
    q = np.array([0.13, 0.05, 0.11])
    El, _ = oracle_mod.kq_interpolate(Wl, q)
    inner = np.all(idx < n - 1, axis=1)
    ref = (idx + q[None, :] * n) @ a
    assert np.allclose(El[inner, 0], ref[inner], rtol=0, atol=1e-12)


def test_kq_interpolation_gauge_and_convergence(oracle_mod):
    """|<m,k|n,k+q>|^2 from interpolated eigenvectors does not depend on the phases the mesh's
    eigenvectors carry; interpolated eigenvectors have unit norm; interpolated energies and
    eigenvectors (up to their phase, away from avoided crossings) converge to the exact ones at
    k+q at second order in the mesh spacing (the seeded model's smooth bands)."""
    rng = np.random.default_rng(4)
    W = wl.tiny_tb(n=4, norb=3, nq=0, seed=wl.SEED_BASE + 52)
    q = (0.173, 0.061, 0.29)
    _, Cq = oracle_mod.kq_interpolate(W, q)
    ph = np.exp(2j * np.pi * rng.uniform(size=(W.C.shape[0], 1, W.C.shape[2])))
    Wp = wl.Workload(W.name, W.n, W.periodic, W.nb, W.norb, W.E, W.C * ph, W.ef, W.window, W.cma, [])
    _, Cqp = oracle_mod.kq_interpolate(Wp, q)
    M = np.abs(np.einsum("kom,kon->kmn", np.conj(W.C), Cq)) ** 2
    Mp = np.abs(np.einsum("kom,kon->kmn", np.conj(Wp.C), Cqp)) ** 2
    assert np.allclose(M, Mp, atol=1e-12)
    assert np.allclose(np.sum(np.abs(Cq) ** 2, axis=1), 1.0, atol=1e-12)
    m = wl.random_model(2, wl.SEED_BASE + 53, spread=2.0)
    errs, verrs = [], []
    for n in (8, 16):
        E, C = m.eig_grid((n, n, n))
        Wn = wl.Workload("s", (n, n, n), True, 2, 2, E, C, 0.0, (0, 2), False, [])
        Eq, Cn = oracle_mod.kq_interpolate(Wn, q)
        Qx = wl.explicit_q(m, (n, n, n), np.array(q))
        errs.append(np.max(np.abs(Eq - Qx.Eq)))
        # 1 - |<exact|interpolated>| per corner and band: its median (the largest values sit at
        # the model's avoided crossings, where the bands' gap is below the mesh's resolution)
        verrs.append(np.median(1.0 - np.abs(np.sum(np.conj(Qx.Cq) * Cn, axis=1))))
    assert errs[1] < errs[0] / 3.0, errs
    assert verrs[1] < verrs[0] / 4.0 and verrs[1] < 1e-4, verrs
