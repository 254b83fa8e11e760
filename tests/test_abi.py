"""The C-ABI library builds, loads and exports every entry point of include/chi0.h;
host-side validation rejects bad arguments before touching a GPU."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1407_3444_gb300 import build, chi0
    build.build()
    return chi0


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "chi0.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(chi0_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("chi0_plan", "chi0_static", "chi0_dynamic", "chi0_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    L = ct.CDLL(lib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(L, n), n
    assert sorted(lib.EXPORTS) == declared_functions()


def test_struct_layouts_match_header(lib):
    # sizes of the ABI structs as a C compiler lays them out (x86-64 / aarch64 LP64)
    assert ct.sizeof(lib.chi0_kgrid_t) == 4 * 3 + 4 * 3 + 8 + 8 + 4 + 4 + 8
    assert ct.sizeof(lib.chi0_q_t) == 12 + 4 + 8 + 8 + 8 + 4 + 4
    assert ct.sizeof(lib.chi0_opts_t) == 4 * 4 + 8 + 4 * 2 + 8 + 4 + 4 + 8 + 32
    assert ct.sizeof(lib.chi0_stats_t) == 8 * 8 + 8 * 8 + 6 * 8


def test_opts_default(lib):
    o = lib.chi0_opts_default()
    assert o.precision == lib.CHI0_PREC_FP64 and o.sign == lib.CHI0_SIGN_POSITIVE
    assert o.cma == 0 and abs(o.tau - 2.0 ** -20) < 1e-18 and o.inputs_on_device == 0
    assert lib.chi0_version() >= 101


def _kgrid(lib, E, nb, n=(2, 2, 2)):
    kg = lib.chi0_kgrid_t()
    kg.n[:] = list(n)
    kg.periodic = 1
    kg.nbands = nb
    kg.norb = nb
    kg.energies = E.ctypes.data
    kg.evecs = None
    kg.evec_dtype = lib.CHI0_C128
    kg.e_fermi = 0.0
    return kg


def test_plan_validation_before_any_launch(lib):
    E = np.sort(np.random.default_rng(0).normal(size=(8, 3)), axis=1)
    o = lib.chi0_opts_default()
    o.cma = 1
    bad = [
        (lambda kg: setattr(kg, "nbands", 0), lib.chi0_band_window_t(0, 3)),
        (lambda kg: kg.n.__setitem__(0, 0), lib.chi0_band_window_t(0, 3)),
        (lambda kg: None, lib.chi0_band_window_t(0, 4)),
        (lambda kg: None, lib.chi0_band_window_t(2, 2)),
        (lambda kg: setattr(kg, "energies", None), lib.chi0_band_window_t(0, 3)),
    ]
    for mutate, win in bad:
        kg = _kgrid(lib, E, 3)
        mutate(kg)
        with pytest.raises(lib.Chi0Error) as ei:
            lib.chi0_plan(kg, None, win, o)
        assert ei.value.code == lib.CHI0_EINVAL
    # eigenvectors are required without CMA
    o2 = lib.chi0_opts_default()
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(_kgrid(lib, E, 3), None, lib.chi0_band_window_t(0, 3), o2)
    assert ei.value.code == lib.CHI0_EINVAL
    # descending energies are rejected
    kg = _kgrid(lib, E[:, ::-1].copy(), 3)
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(kg, None, lib.chi0_band_window_t(0, 3), o)
    assert "ascending" in str(ei.value)
    # custom tetrahedra with out-of-range corners
    corners = np.array([[0, 1, 2, 99]], dtype=np.int32)
    vols = np.array([1.0])
    tt = lib.chi0_tetra_t(1, corners.ctypes.data, vols.ctypes.data)
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(_kgrid(lib, E, 3), tt, lib.chi0_band_window_t(0, 3), o)
    assert ei.value.code == lib.CHI0_EINVAL
    # unsupported tensor-core overlap mode is reported, not silently replaced
    o3 = lib.chi0_opts_default()
    o3.cma = 1
    o3.overlap = 7
    with pytest.raises(lib.Chi0Error):
        lib.chi0_plan(_kgrid(lib, E, 3), None, lib.chi0_band_window_t(0, 3), o3)
    assert lib.chi0_last_error(None) != ""
    # tensor-core overlaps are a mixed-precision form; the stall hook needs one of them
    o4 = lib.chi0_opts_default()
    o4.cma = 1
    o4.overlap = lib.CHI0_OVL_BF16X3
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(_kgrid(lib, E, 3), None, lib.chi0_band_window_t(0, 3), o4)
    assert ei.value.code == lib.CHI0_ENOTSUP
    o5 = lib.chi0_opts_default()
    o5.cma = 1
    o5.precision = lib.CHI0_PREC_MIXED
    o5.test_stall = 1
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(_kgrid(lib, E, 3), None, lib.chi0_band_window_t(0, 3), o5)
    assert ei.value.code == lib.CHI0_EINVAL
    # graph capture and the stall hook exclude each other
    o6 = lib.chi0_opts_default()
    o6.cma = 1
    o6.precision = lib.CHI0_PREC_MIXED
    o6.overlap = lib.CHI0_OVL_BF16X6
    o6.test_stall = 1
    o6.graph = 1
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_plan(_kgrid(lib, E, 3), None, lib.chi0_band_window_t(0, 3), o6)
    assert ei.value.code == lib.CHI0_EINVAL


def test_destroy_null_is_safe(lib):
    lib.chi0_destroy(None)


def test_null_plan_calls_fail_cleanly(lib):
    q = (lib.chi0_q_t * 1)()
    out = np.zeros(1)
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_static(None, q, 1, out.ctypes.data)
    assert ei.value.code == lib.CHI0_EINVAL
    e = np.zeros(4)
    for fn in ("chi0_plan_update", "chi0_plan_stage"):  # checked before any CUDA call
        assert getattr(lib.lib(), fn)(None, e.ctypes.data, e.ctypes.data) == lib.CHI0_EINVAL


def test_noalloc_rejects_orbital_counts_beyond_the_plan_limit(lib):
    """chi0_static_noalloc caps norb like chi0_plan (65536), so that no buffer size of its
    work-array layout can wrap around; the check comes before any CUDA call."""
    kg = lib.chi0_kgrid_t()
    kg.n[:] = [4, 4, 4]
    kg.periodic = 1
    kg.nbands = 4096
    kg.norb = 1 << 20
    kg.energies = 16  # never dereferenced: validation fails first
    kg.evecs = 16
    kg.evec_dtype = lib.CHI0_C128
    o = lib.chi0_opts_default()
    o.precision = lib.CHI0_PREC_MIXED
    q = (lib.chi0_q_t * 1)()
    q[0].win = lib.chi0_band_window_t(-1, -1)
    with pytest.raises(lib.Chi0Error) as ei:
        lib.chi0_static_noalloc(kg, lib.chi0_band_window_t(0, 4096), o, q, 1, 16)
    assert ei.value.code == lib.CHI0_EINVAL
    assert "norb" in str(ei.value)
