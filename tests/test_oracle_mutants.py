"""The oracles' pins catch plausible mistakes: each case below plants one mistake (a dropped term, a
wrong sign, a transposed index or operand, a wrong factor, a storage-order slip) in a copy of one of the
oracle's C sources, builds the copy, points the oracle module at it and runs the pins of
test_oracle_pins.py (the chain and its adjoint), test_fd_oracle.py (on-grid derivatives) or
test_expr_oracle.py (the benchmark expressions) against it.  Every planted mistake must fail at least
one pin, and the unchanged copy must pass them all.  The committed oracle is never modified (no GPU).
"""
import os
import subprocess

import pytest

import oracle
from tests import test_expr_oracle as expr_pins
from tests import test_fd_oracle as fd_pins
from tests import test_oracle_pins as pins
from tests import test_tensor_expr_oracle as interp_pins

FORWARD_PIN_NAMES = [
    "test_inverse_worked_case_bitwise",
    "test_inverse_identity_and_library",
    "test_flat_metric_gives_zero_christoffel_and_listing1_form",
    "test_conformally_flat_closed_form",
    "test_diagonal_metric_hand_formula",
    "test_spherical_coordinates_textbook",
    "test_curvilinear_flat_space_closed_forms",
    "test_killing_field_rotation",
    "test_shift_derivative_and_eq5_from_the_lie_derivative",
    "test_metric_compatibility",
    "test_packing_convention",
]
ADJOINT_PIN_NAMES = [
    "test_adjoint_central_differences",
    "test_adjoint_all_outputs_and_dot_product_identity",
    "test_adjoint_against_torch_autograd",
]
FORWARD_PINS = [(n, getattr(pins, n)) for n in FORWARD_PIN_NAMES if n != "test_shift_derivative_and_eq5_from_the_lie_derivative"] + \
    [("test_shift_derivative_and_eq5_from_the_lie_derivative",
      lambda: pins.test_shift_derivative_and_eq5_from_the_lie_derivative(19, 25.0))]
ADJOINT_PINS = [(n, getattr(pins, n)) for n in ADJOINT_PIN_NAMES]
FD_PINS = ([("mode_exact_o%d_%d" % (o, f), lambda o=o, f=f, r=r: fd_pins.test_discrete_derivative_of_a_mode_is_exact(o, f, r))
            for o in (2, 4) for f, r in ((13, 34), (4, 6 + 3 * 4))] +
           [("convergence_o%d" % o, lambda o=o: fd_pins.test_convergence_order(o)) for o in (2, 4)] +
           [("axis_placement", fd_pins.test_axis_placement_and_copies),
            ("constants", fd_pins.test_constant_fields_have_zero_derivatives)])
EXPR_PINS = [("assign_add_outer", expr_pins.test_assign_add_outer_bitwise),
             ("einsum", expr_pins.test_contractions_against_einsum),
             ("identity_factors", expr_pins.test_contractions_with_identity_factors_are_exact),
             ("kij", expr_pins.test_kij),
             ("integers_exact", expr_pins.test_sums_and_outer_products_exact_on_integers),
             ("contractions_integers_exact", expr_pins.test_contractions_exact_on_integers),
             ("kij_rank_one", expr_pins.test_kij_minus_lapse_term_is_rank_one)]

# (id, exact text in oracle/dtg_oracle.c, replacement).  Each text occurs exactly once.
FORWARD_MUTANTS = [
    # step 1: inverse metric
    ("cofactor-sign", "C[i][j] = G[i1][j1] * G[i2][j2] - G[i1][j2] * G[i2][j1];",
     "C[i][j] = G[i1][j1] * G[i2][j2] + G[i1][j2] * G[i2][j1];"),
    ("det-wrong-cofactor", "G[0][2] * C[0][2];", "G[0][2] * C[0][1];"),
    ("det-dropped-term", "G[0][0] * C[0][0] + G[0][1] * C[0][1] + G[0][2] * C[0][2];",
     "G[0][0] * C[0][0] + G[0][1] * C[0][1];"),
    ("inverse-times-det", "H[i][j] = C[j][i] / det;", "H[i][j] = C[j][i] * det;"),
    # step 2: Eq. 6
    ("bracket-sign", "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][k][l];",
     "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) + P->D[j][k][l];"),
    ("bracket-dropped-term", "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][k][l];",
     "R->T[l][j][k] = P->D[j][l][k] - P->D[j][k][l];"),
    ("bracket-second-term-index", "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][k][l];",
     "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][j][k]) - P->D[j][k][l];"),
    ("bracket-third-term-derivative", "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][k][l];",
     "R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][l][k];"),
    ("missing-half", "R->Gam[i][j][k] = 0.5 * s;", "R->Gam[i][j][k] = s;"),
    ("contraction-transposed-bracket", "s += R->H[i][l] * R->T[l][j][k];", "s += R->H[i][l] * R->T[j][l][k];"),
    ("contraction-dropped-term", "for (int l = 0; l < 3; ++l)\n                    s += R->H[i][l] * R->T[l][j][k];",
     "for (int l = 0; l < 2; ++l)\n                    s += R->H[i][l] * R->T[l][j][k];"),
    ("contraction-metric-not-inverse", "s += R->H[i][l] * R->T[l][j][k];", "s += P->G[i][l] * R->T[l][j][k];"),
    # step 3: footnote to Listing 1
    ("shift-gamma-index", "s += R->Gam[k][i][j] * P->b[k];", "s += R->Gam[i][k][j] * P->b[k];"),
    ("shift-sign", "R->Nb[i][j] = P->B[i][j] - s;", "R->Nb[i][j] = P->B[i][j] + s;"),
    ("shift-transposed-derivative", "R->Nb[i][j] = P->B[i][j] - s;", "R->Nb[i][j] = P->B[j][i] - s;"),
    # step 4: Eq. 5
    ("eq5-K-sign", "R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];",
     "R->dtg[i][j] = (2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];"),
    ("eq5-K-factor", "R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];",
     "R->dtg[i][j] = (-1.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];"),
    ("eq5-missing-lapse", "R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];",
     "R->dtg[i][j] = (-2.0 * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];"),
    ("eq5-one-order-twice", "R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];",
     "R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[i][j]) + R->Nb[i][j];"),
    # storage convention
    ("dg-derivative-outermost", "P->D[i][j][k] = in[6 + 3 * p + k][x];", "P->D[i][j][k] = in[6 + 6 * k + p][x];"),
    ("dbeta-transposed-storage", "P->B[i][j] = in[34 + 3 * i + j][x];", "P->B[i][j] = in[34 + 3 * j + i][x];"),
    ("gamma-output-transposed", "out[6 + 6 * i + sym_index(j, k)][x] = R.Gam[i][j][k];",
     "out[6 + 6 * i + sym_index(j, k)][x] = R.Gam[j][i][k];"),
]
ADJOINT_MUTANTS = [
    ("adj-K-sign", "Kbar[p] = -2.0 * P.alpha * Wdt[p];", "Kbar[p] = 2.0 * P.alpha * Wdt[p];"),
    ("adj-shift-fold", "Nbar[j][i] += Wdt[p];", "Nbar[i][j] += Wdt[p];"),
    ("adj-beta-sign", "bbar[k] = -s;", "bbar[k] = s;"),
    ("adj-Hbar-half", "Hbar[i][l] = 0.5 * s;", "Hbar[i][l] = s;"),
    ("adj-Tbar-index", "s += R.H[i][l] * Gambar[i][sym_index(j, k)];", "s += R.H[i][l] * Gambar[l][sym_index(j, k)];"),
    ("adj-scatter-sign", "Dbar[j][k][l] -= t;", "Dbar[j][k][l] += t;"),
    ("adj-inverse-sign", "Gbar[i][j] = -s;", "Gbar[i][j] = s;"),
]


FD_MUTANTS = [
    ("fd-o2-sign", "return (v[3] - v[1]) / (2.0 * h);", "return (v[1] - v[3]) / (2.0 * h);"),
    ("fd-o2-factor", "return (v[3] - v[1]) / (2.0 * h);", "return (v[3] - v[1]) / h;"),
    ("fd-o4-outer-sign", "(8.0 * (v[3] - v[1]) - (v[4] - v[0]))", "(8.0 * (v[3] - v[1]) - (v[4] + v[0]))"),
    ("fd-o4-dropped-term", "(8.0 * (v[3] - v[1]) - (v[4] - v[0]))", "(8.0 * (v[3] - v[1]))"),
    ("fd-o4-denominator", "/ (12.0 * h);", "/ (6.0 * h);"),
    ("fd-spacing-of-axis-0", "deriv(in16[p], ix, iy, iz, k, nx, ny, nz, h[k], order)",
     "deriv(in16[p], ix, iy, iz, k, nx, ny, nz, h[0], order)"),
    ("fd-metric-axes-reversed", "deriv(in16[p], ix, iy, iz, k, nx, ny, nz, h[k], order)",
     "deriv(in16[p], ix, iy, iz, 2 - k, nx, ny, nz, h[k], order)"),
    ("fd-shift-transposed", "deriv(in16[13 + i], ix, iy, iz, j, nx, ny, nz, h[j], order)",
     "deriv(in16[13 + j], ix, iy, iz, i, nx, ny, nz, h[i], order)"),
    ("fd-K-copied-from-g", "out43[24 + p][x] = in16[6 + p][x];", "out43[24 + p][x] = in16[p][x];"),
]
EXPR_MUTANTS = [
    ("eq14-dropped-operand", "const int terms = eq - 10;", "const int terms = eq == 14 ? 3 : eq - 10;"),
    ("eq16-repeated-index", "out[9 * i + 3 * j + k][x] = (in[i][x] * in[3 + j][x]) * in[6 + k][x];",
     "out[9 * i + 3 * j + k][x] = (in[i][x] * in[3 + j][x]) * in[6 + j][x];"),
    ("eq17-repeated-index", "((in[i][x] * in[3 + j][x]) * in[6 + k][x]) * in[9 + l][x];",
     "((in[i][x] * in[3 + j][x]) * in[6 + k][x]) * in[9 + k][x];"),
    ("eq18-B-transposed", "s += in[3 * i + m][x] * in[9 + 27 * m + 9 * j + 3 * k + l][x];",
     "s += in[3 * m + i][x] * in[9 + 27 * m + 9 * j + 3 * k + l][x];"),
    ("eq18-dropped-term", "for (int m = 0; m < 3; ++m)\n                                s += in[3 * i + m][x]",
     "for (int m = 0; m < 2; ++m)\n                                s += in[3 * i + m][x]"),
    ("eq19-C-transposed", "s += (in[9 + 3 * j + nn][x] * in[3 * i + m][x]) *",
     "s += (in[9 + 3 * nn + j][x] * in[3 * i + m][x]) *"),
    ("eq20-E-slots-swapped", "in[27 + 27 * m + 9 * nn + 3 * o + l][x];", "in[27 + 27 * m + 9 * o + 3 * nn + l][x];"),
    ("eq20-D-transposed", "s += ((in[18 + 3 * k + o][x] *", "s += ((in[18 + 3 * o + k][x] *"),
    ("eq21-missing-2", "(2.0 * in[0][x]) * in[1 + expr_sym(i, j)][x]", "in[0][x] * in[1 + expr_sym(i, j)][x]"),
    ("eq21-repeated-index", "in[7 + i][x] * in[7 + j][x];", "in[7 + i][x] * in[7 + i][x];"),
]

# The tensor-index interpreter (oracle/tensor_expr.py), the runtime generator's oracle.
INTERP_PINS = [("chain_transcribed", lambda: interp_pins.test_chain_program_equals_chain_oracle("transcribed here")),
               ("chain_package", lambda: interp_pins.test_chain_program_equals_chain_oracle("shipped with the package")),
               ("expressions_bitwise", interp_pins.test_benchmark_expressions_bitwise),
               ("listings_einsum", interp_pins.test_paper_listings_against_einsum),
               ("declared_range_einsum", interp_pins.test_sum_over_a_declared_range_against_einsum)]
INTERP_MUTANTS = [
    ("interp-canonical-order", "if t[a] > t[b]:", "if t[a] < t[b]:"),
    ("interp-minus-as-plus", '"-": lambda: a - b', '"-": lambda: a + b'),
    ("interp-divide-as-multiply", '"/": lambda: a / b', '"/": lambda: a * b'),
    ("interp-unary-minus-dropped", "return -self._eval(node[1], env, values)", "return self._eval(node[1], env, values)"),
    ("interp-sum-drops-last", "for v in range(self._dim_of(node[2], letter)):",
     "for v in range(self._dim_of(node[2], letter) - 1):"),
    ("interp-sum-ignores-range", "return self.ranges.get(letter, decl.dims[s])", "return decl.dims[s]"),
    ("interp-offset-dropped", "env[ix[1]] + ix[2] for ix in node[2])", "env[ix[1]] for ix in node[2])"),
    ("interp-last-assignment-wins", "if tup not in new:", "if True:"),
]

SOURCES = ("dtg_oracle.c", "expr_oracle.c", "fd_oracle.c")


def _build_copy(tmp_path, source, old, new):
    """Compile the oracle sources with `source` edited (old -> new) into tmp_path; return the .so."""
    here = os.path.dirname(os.path.abspath(oracle.__file__))
    paths = []
    for name in SOURCES:
        src = open(os.path.join(here, name)).read()
        if name == source and old is not None:
            assert src.count(old) == 1, old
            src = src.replace(old, new)
        path = tmp_path / name
        path.write_text(src)
        paths.append(str(path))
    so = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", str(so)] + paths + ["-lm"])
    return str(so)


def _failing_pins(monkeypatch, so, battery):
    """Run the pins of `battery` ((name, callable) pairs) with the oracle module loading `so`; return the
    names of those that fail."""
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "_lib", None)
    failed = []
    for name, pin in battery:
        try:
            pin()
        except Exception:              # an assertion, or a value the pin cannot even process
            failed.append(name)
    return failed


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    so = _build_copy(tmp_path, None, None, None)
    assert _failing_pins(monkeypatch, so, FORWARD_PINS + ADJOINT_PINS + FD_PINS + EXPR_PINS) == []
    monkeypatch.setattr(interp_pins, "Program", _load_interpreter_copy(tmp_path, None, None).Program)
    assert _failing_pins(monkeypatch, so, INTERP_PINS) == []


CASES = ([("dtg_oracle.c", FORWARD_PINS) + m for m in FORWARD_MUTANTS] +
         [("dtg_oracle.c", ADJOINT_PINS) + m for m in ADJOINT_MUTANTS] +
         [("fd_oracle.c", FD_PINS) + m for m in FD_MUTANTS] +
         [("expr_oracle.c", EXPR_PINS) + m for m in EXPR_MUTANTS])


@pytest.mark.parametrize("source,battery,name,old,new", CASES, ids=[c[2] for c in CASES])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, source, battery, name, old, new):
    so = _build_copy(tmp_path, source, old, new)
    assert _failing_pins(monkeypatch, so, battery), name


def _load_interpreter_copy(tmp_path, old, new):
    """Import a copy of oracle/tensor_expr.py with old -> new applied, as a module of its own."""
    import importlib.util
    here = os.path.dirname(os.path.abspath(oracle.__file__))
    src = open(os.path.join(here, "tensor_expr.py")).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    path = tmp_path / "tensor_expr_copy.py"
    path.write_text(src)
    spec = importlib.util.spec_from_file_location("tensor_expr_copy_%d" % abs(hash(str(path))), str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", INTERP_MUTANTS, ids=[m[0] for m in INTERP_MUTANTS])
def test_planted_interpreter_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new):
    monkeypatch.setattr(interp_pins, "Program", _load_interpreter_copy(tmp_path, old, new).Program)
    failed = []
    for pin_name, pin in INTERP_PINS:
        try:
            pin()
        except Exception:
            failed.append(pin_name)
    assert failed, name
