"""The seeded input generators (shared by the oracle and the CUDA path; no method arithmetic):
the readings they implement - Bloch-symmetric hopping (H(k) Hermitian and even in k, exactly
on the grid), E_F between distinct levels at the stated filling, equal-arc-length q paths,
per-q band windows around E_F - and bitwise reproducibility from the seeds."""
import numpy as np

from paper_1407_3444_gb300 import workloads as wl


def test_hamiltonian_hermitian_and_even_on_the_grid():
    m = wl.cr_like_model()
    n = (6, 6, 6)
    idx = wl.corner_index(n, True)
    H = m.hamiltonian(None, grid=(idx, n))
    assert np.array_equal(H, np.conj(np.swapaxes(H, 1, 2)))  # Hermitian, bitwise
    neg = (-idx) % np.asarray(n)
    Hm = m.hamiltonian(None, grid=(neg, n))
    assert np.array_equal(H, Hm)  # t(-R) = t(R): H(-k) = H(k) bitwise (integer phases)


def test_generators_reproduce_bitwise():
    a = wl.tiny_tb(n=4, norb=5, nq=2, seed=wl.SEED_BASE + 90)
    b = wl.tiny_tb(n=4, norb=5, nq=2, seed=wl.SEED_BASE + 90)
    assert np.array_equal(a.E, b.E) and np.array_equal(a.C, b.C) and a.ef == b.ef
    for qa, qb in zip(a.qs, b.qs):
        assert np.array_equal(qa.Eq, qb.Eq) and np.array_equal(qa.Cq, qb.Cq)


def test_fermi_level_filling_and_gap():
    E = np.sort(np.random.default_rng(3).normal(size=(500, 6)), axis=1)
    ef = wl.fermi_level(E, 2.5)
    assert not np.any(E == ef)
    frac = np.mean(E < ef) * E.shape[1]
    assert abs(frac - 2.5) < 0.01


def test_q_path_equal_arc_length():
    nodes = [(0, 0, 0), (0.5, 0, 0), (0.5, 0.5, 0), (0, 0, 0)]
    P = wl.path_points(nodes, 256)
    steps = np.linalg.norm(np.diff(P, axis=0), axis=1)
    # equal arc length except across the corners of the path, where the chord is shorter
    assert np.allclose(np.median(steps), steps[steps > 0.99 * np.median(steps)], rtol=1e-9)
    assert np.allclose(P[0], 0.0)


def test_band_sweep_windows_around_ef():
    W = wl.band_sweep(n=4, nb=40, nq=20, nw=4)
    for q in W.qs:
        lo, hi = q.window
        assert 4 <= hi - lo <= 40 and 0 <= lo and hi <= 40
        assert lo <= 20 <= hi  # the window straddles the Fermi level (half filling)
