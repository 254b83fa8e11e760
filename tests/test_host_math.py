"""The CUDA path's per-tetrahedron arithmetic (chi0_math.cuh built for the host by
tests/host_math/host_math.cpp) against the FP64 oracle on random and near-degenerate
tetrahedra.  FP64: 1e-11 per tetrahedron.  Mixed precision: 3e-5 per tetrahedron (a corner
a few 1e-5 from a Fermi surface leaves a sliver whose FP32 cut fractions carry relative
errors of that size; its volume is as small) and 1e-6 on the sum over all tetrahedra, the
normwise measure of chi0.  A CPU check of the kernel math between GPU runs; the GPU tests
remain the parity proof."""
import ctypes as ct
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("host_math") / "libhost_math.so")
    src = os.path.join(HERE, "host_math", "host_math.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", src, "-o", out], check=True)
    L = ct.CDLL(out)
    dp = ct.POINTER(ct.c_double)
    L.host_static.restype = ct.c_double
    L.host_static.argtypes = [dp, dp, dp, ct.c_int]
    L.host_dynamic_mixed.restype = None
    L.host_dynamic_mixed.argtypes = [dp, dp, dp, ct.c_int, dp, dp, dp]
    return L


def _p(x):
    return np.ascontiguousarray(x, dtype=np.float64).ctypes.data_as(ct.POINTER(ct.c_double))


def _cases(rng, n):
    out = []
    for _ in range(n):
        a = rng.normal(0.0, 1.0, 4)
        b = a + rng.uniform(0.05, 1.5) + rng.normal(0.0, 0.3, 4)  # D mostly > 0, some cuts
        f = rng.uniform(0.1, 1.0, 4)
        if a.min() < 0 and b.max() > 0:
            out.append((a, b, f))
    # clustered knots (long series, table, FP64 branch) and a vertex on both cut planes
    out.append((np.array([-0.3, -0.2, 0.1, 0.4]), np.array([0.5, 0.5000001, 0.5000002, 0.9]), np.ones(4)))
    out.append((np.array([-1.0, 0.0, 0.5, -0.25]), np.array([0.0, 0.7, 1.1, 0.3]), np.array([1, 2, 3, 4.0])))
    return out


def test_static_weights_match_oracle(H, oracle_mod):
    rng = np.random.default_rng(11)
    s_ref = s_32 = 0.0
    for a, b, f in _cases(rng, 300):
        ref = oracle_mod.tet_integrals(a, b, f)
        g64 = H.host_static(_p(a), _p(b), _p(f), 1)
        g32 = H.host_static(_p(a), _p(b), _p(f), 0)
        scale = max(abs(ref), 1e-30)
        assert abs(g64 - ref) <= 1e-11 * scale + 1e-13, (a, b, f, g64, ref)
        assert abs(g32 - ref) <= 3e-5 * scale + 1e-9, (a, b, f, g32, ref)
        s_ref += ref
        s_32 += g32
    assert abs(s_32 - s_ref) <= 1e-6 * abs(s_ref)


def test_dynamic_mixed_matches_oracle(H, oracle_mod):
    rng = np.random.default_rng(12)
    w = np.linspace(0.0, 3.0, 61)
    tr, ti, gr_s, gi_s = (np.zeros(w.size) for _ in range(4))
    for a, b, f in _cases(rng, 120):
        rr, ri = oracle_mod.tet_integrals(a, b, f, omega=w)
        gr = np.zeros(w.size)
        gi = np.zeros(w.size)
        H.host_dynamic_mixed(_p(a), _p(b), _p(f), w.size, _p(w), _p(gr), _p(gi))
        sr = max(np.max(np.abs(rr)), 1e-30)
        si = max(np.max(np.abs(ri)), sr)
        assert np.max(np.abs(gr - rr)) <= 3e-5 * sr, (a, b, f)
        assert np.max(np.abs(gi - ri)) <= 3e-5 * si, (a, b, f)
        tr += rr
        ti += ri
        gr_s += gr
        gi_s += gi
    assert np.max(np.abs(gr_s - tr)) <= 1e-6 * np.max(np.abs(tr))
    assert np.max(np.abs(gi_s - ti)) <= 1e-6 * np.max(np.abs(ti))
