"""The oracle's pins catch plausible mistakes: each case below plants one mistake (a dropped term, a
wrong sign, a transposed index or operand, a wrong factor, a storage-order slip) in a copy of the
oracle's C source, builds the copy, points the oracle module at it and runs the pins of
test_oracle_pins.py against it.  Every planted mistake must fail at least one pin, and the unchanged
copy must pass them all.  The committed oracle is never modified (no GPU).
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

FORWARD_PINS = [
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
ADJOINT_PINS = [
    "test_adjoint_central_differences",
    "test_adjoint_all_outputs_and_dot_product_identity",
    "test_adjoint_against_torch_autograd",
]

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


def _build_copy(tmp_path, old, new):
    """Compile the oracle sources with dtg_oracle.c edited (old -> new) into tmp_path; return the .so."""
    here = os.path.dirname(os.path.abspath(oracle.__file__))
    src = open(os.path.join(here, "dtg_oracle.c")).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    path = tmp_path / "dtg_oracle.c"
    path.write_text(src)
    so = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", str(so), str(path), os.path.join(here, "expr_oracle.c"),
                           os.path.join(here, "fd_oracle.c"), "-lm"])
    return str(so)


def _failing_pins(monkeypatch, so, names):
    """Run the named pins with the oracle module loading `so`; return the names of those that fail."""
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "_lib", None)
    failed = []
    for name in names:
        try:
            getattr(pins, name)()
        except Exception:              # an assertion, or a value the pin cannot even process
            failed.append(name)
    return failed


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    so = _build_copy(tmp_path, None, None)
    assert _failing_pins(monkeypatch, so, FORWARD_PINS + ADJOINT_PINS) == []


@pytest.mark.parametrize("name,old,new", FORWARD_MUTANTS, ids=[m[0] for m in FORWARD_MUTANTS])
def test_forward_mistake_fails_a_forward_pin(tmp_path, monkeypatch, name, old, new):
    so = _build_copy(tmp_path, old, new)
    assert _failing_pins(monkeypatch, so, FORWARD_PINS), name


@pytest.mark.parametrize("name,old,new", ADJOINT_MUTANTS, ids=[m[0] for m in ADJOINT_MUTANTS])
def test_adjoint_mistake_fails_an_adjoint_pin(tmp_path, monkeypatch, name, old, new):
    so = _build_copy(tmp_path, old, new)
    assert _failing_pins(monkeypatch, so, ADJOINT_PINS), name
