"""Planted mistakes: each test copies the oracle, plants one plausible error in its C source or
its Python part (a wrong repeated knot, a sign, a cut fraction, a missing conjugate or
factor, a transposed band index, a dropped term of the Kramers-Kronig kernel, swapped
interpolation weights, no phase alignment), builds the copy on the CPU and checks that the
pins of test_oracle_pins.py reject it.  The real oracle is never modified."""
import importlib.util
import os
import shutil

import pytest

import test_oracle_pins as pins

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# (name, original text, planted text, pins expected to fail)
MUTANTS = [
    ("repeated_knot", "t[4] = x[j] / s;", "t[4] = x[(j + 1) % 4] / s;",
     ["test_inv_weight_vs_simplex_quadrature", "test_inv_weight_sum_rule"]),
    ("pv_sign", "r += ff[j] * (oracle_inv_weight(xm, j) + oracle_inv_weight(xp, j));",
     "r += ff[j] * (oracle_inv_weight(xm, j) - oracle_inv_weight(xp, j));",
     ["test_tet_dynamic_integrals_identities"]),
    ("cut_fraction", "double t = kp / (kp - kq);", "double t = kq / (kq - kp);",
     ["test_carving_volume_all_cases"]),
    ("second_cut_key", "return which == 0 ? v->a : -(v->a + v->D);", "return which == 0 ? v->a : -(v->D);",
     ["test_carving_volume_all_cases"]),
    ("no_conjugate", "re += x[0] * y[0] + x[1] * y[1];\n    im += x[0] * y[1] - x[1] * y[0];",
     "re += x[0] * y[0] - x[1] * y[1];\n    im += x[0] * y[1] + x[1] * y[0];",
     ["test_flat_bands_matrix_element_closed_form"]),
    ("static_factor", "acc += ff[j] * 2.0 * oracle_inv_weight(d, j);", "acc += ff[j] * oracle_inv_weight(d, j);",
     ["test_free_electron_lindhard_static", "test_tet_static_integral_vs_qmc"]),
    ("im_pi", "vs * M_PI * m);", "vs * m);",
     ["test_free_electron_dynamic_im", "test_tet_dynamic_integrals_identities"]),
    ("bands_transposed", "const double *y = Ckq + 2 * (((int64_t)ckq * in->norb + o) * nb + n);",
     "const double *y = Ckq + 2 * (((int64_t)ckq * in->norb + o) * nb + m);",
     ["test_flat_bands_matrix_element_closed_form"]),
    ("gamma_dos_dropped", "if (nw == 0 || in->omega[k] == 0.0) re_out[k] += sgn * 2.0 * acc_val(&G);",
     "if (nw == 0 || in->omega[k] == 0.0) re_out[k] += 0.0 * acc_val(&G);",
     ["test_free_electron_q0_limit"]),
    ("pairs_transposed", "acc_add(&P[((size_t)tid * w + (m - in->lo)) * w + (n - in->lo)], acc_val(&one));",
     "acc_add(&P[((size_t)tid * w + (n - in->lo)) * w + (m - in->lo)], acc_val(&one));",
     ["test_pairs_flat_bands_closed_form"]),
    ("pairs_gamma_dos_dropped", "pairs[(m - in->lo) * (w + 1)] += sgn * 2.0 * acc_val(&G);",
     "pairs[(m - in->lo) * (w + 1)] += 0.0 * acc_val(&G);",
     ["test_pairs_add_up_to_chi0"]),
    ("kk_plus_term_dropped@py", "        for c in (wv, -wv):\n            for j in range(len(uu) - 1):",
     "        for c in (wv,):\n            for j in range(len(uu) - 1):",
     ["test_kk_transform_matches_cauchy_quadrature", "test_kk_route_converges_to_principal_value"]),
    ("interp_weights_swapped@py",
     "w = [1.0 - tc[order[0]], tc[order[0]] - tc[order[1]], tc[order[1]] - tc[order[2]], tc[order[2]]]",
     "w = [1.0 - tc[order[0]], tc[order[1]] - tc[order[2]], tc[order[0]] - tc[order[1]], tc[order[2]]]",
     ["test_kq_interpolation_on_grid_and_linear"]),
    ("interp_no_phase@py", "ph = np.where(m > 0, np.conj(ov) / np.where(m > 0, m, 1.0), 1.0)",
     "ph = np.ones(vi.shape[1], dtype=np.complex128)",
     ["test_kq_interpolation_gauge_and_convergence"]),
    ("interp_not_normalised@py", "Cq[c] = acc / np.where(nrm > 0, nrm, 1.0)[None, :]", "Cq[c] = acc",
     ["test_kq_interpolation_gauge_and_convergence"]),
    ("kk_segment_expanded_at_its_start@py", "tot += beta * (b - a) + (alpha + beta * c) * (lb - la)",
     "tot += beta * (b - a) + (alpha + beta * a) * (lb - la)",
     ["test_kk_transform_matches_cauchy_quadrature"]),
]


def _mutant_module(tmp_path, name, old, new):
    """A copy of the oracle with `old` replaced by `new` in its C source, or in its Python part
    for names ending in "@py"."""
    target = "__init__.py" if name.endswith("@py") else "chi0_oracle.c"
    other = "chi0_oracle.c" if target == "__init__.py" else "__init__.py"
    src = open(os.path.join(ORACLE_DIR, target)).read()
    assert src.count(old) == 1, "planting site not unique: %r" % old
    name = name.replace("@py", "_py")
    d = tmp_path / ("oracle_mut_" + name)
    d.mkdir()
    shutil.copy(os.path.join(ORACLE_DIR, other), d / other)
    (d / target).write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_mut_" + name, str(d / "__init__.py"),
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, name, old, new, checks):
    mod = _mutant_module(tmp_path, name, old, new)
    for check in checks:
        with pytest.raises(AssertionError):
            getattr(pins, check)(mod)


def test_unmodified_copy_passes_the_same_pins(tmp_path):
    """Control: a copy built the same way without a planted mistake passes every pin used
    above, so the failures come from the mistakes."""
    mod = _mutant_module(tmp_path, "control", "t[4] = x[j] / s;", "t[4] = x[j] / s;")
    for check in sorted({c for m in MUTANTS for c in m[3]}):
        getattr(pins, check)(mod)
