"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a temporary copy of oracle/qs_oracle.c
(on the CPU, in a scratch directory), compiles it, and runs the pin tests of
test_oracle_pins against it: at least one pin must fail.  The unmodified
source must pass them all.
"""

import os

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as P

PINS = [
    lambda: P.test_single_qubit_gate_equals_kronecker_operator(3),
    lambda: P.test_controlled_gate_equals_kronecker_operator(3),
    lambda: P.test_swap_equals_pauli_formula(3),
    lambda: P.test_qft_of_basis_state_closed_form(6),
    lambda: P.test_qft_closed_form_routines_match_the_circuit(3),
    lambda: P.test_dense_block_equals_kronecker_operator(6, 3),
    lambda: P.test_permutation_circuits_are_bit_exact(),
    lambda: P.test_reductions_brute_force(),
    lambda: P.test_gradient_closed_form_ry_z(),
    lambda: P.test_gradient_one_layer_closed_form(),
    lambda: P.test_gradient_parameter_shift_dense("ising"),
    lambda: P.test_rotation_matrices_match_matrix_exponential(),
]

# (name, exact source text, replacement, occurrence index or None for all)
MUTANTS = [
    ("transposed q12/q21", "cplx a2 = cadd(cmul(q11, a), cmul(q12, b));\n    cplx b2 = cadd(cmul(q21, a)",
     "cplx a2 = cadd(cmul(q11, a), cmul(q21, b));\n    cplx b2 = cadd(cmul(q12, a)", 0),
    ("dropped q21 term", "cplx b2 = cadd(cmul(q21, a), cmul(q22, b));", "cplx b2 = cmul(q22, b);", 0),
    ("conjugated product", "r.re = a.re * b.re - a.im * b.im;", "r.re = a.re * b.re + a.im * b.im;", None),
    ("control on |0>", "if ((i >> c) & 1u) pair_update", "if (((i >> c) & 1u) == 0) pair_update", None),
    ("stride 2^k+1", "uint64_t N = (uint64_t)1 << n, s = (uint64_t)1 << k;",
     "uint64_t N = (uint64_t)1 << n, s = (uint64_t)1 << (k ? k - 1 : 0);", None),
    ("swap condition", "if (((i >> a) & 1u) == 0 && ((i >> b) & 1u) == 1) {", "if (((i >> a) & 1u) == 0) {", None),
    ("marginal bit", "if ((i >> k) & 1u) nadd", "if (((i >> k) & 1u) == 0) nadd", None),
    ("ZZ parity", "int par = (int)(((i >> t->q0) ^ (i >> t->q1)) & 1u);", "int par = (int)((i >> t->q0) & 1u);", None),
    ("X pairing", "uint64_t j = i ^ ((uint64_t)1 << t->q0);\n            nadd", "uint64_t j = i;\n            nadd", None),
    ("RY sign", "if (kind == OR_RY) { set(m, 0, c, 0); set(m, 1, -s, 0); set(m, 2, s, 0);",
     "if (kind == OR_RY) { set(m, 0, c, 0); set(m, 1, s, 0); set(m, 2, -s, 0);", None),
    ("RZ derivative sign", "set(m, 0, -0.5 * s, -0.5 * c); set(m, 3, -0.5 * s, 0.5 * c);",
     "set(m, 0, -0.5 * s, 0.5 * c); set(m, 3, -0.5 * s, -0.5 * c);", None),
    ("gradient factor", "grads[g[j].param] += 2.0 * nval(&a);", "grads[g[j].param] += nval(&a);", None),
    ("QFT closed-form phase sign", "psi[2 * y + 1] = scale * sin(ph);", "psi[2 * y + 1] = -scale * sin(ph);", None),
    ("QFT closed-form phase product", "double ph = w * (double)((x * y) & mask);",
     "double ph = w * (double)((x + y) & mask);", None),
    ("dense block transposed", "u.re = U[2 * (r * G + c)]; u.im = U[2 * (r * G + c) + 1];",
     "u.re = U[2 * (c * G + r)]; u.im = U[2 * (c * G + r) + 1];", None),
    ("half angle", "double c = cos(0.5 * theta), s = sin(0.5 * theta);", "double c = cos(theta), s = sin(theta);", None),
]


def _mutate(src, old, new, occurrence):
    assert old in src, f"mutation anchor not found: {old!r}"
    if occurrence is None:
        return src.replace(old, new)
    idx = -1
    for _ in range(occurrence + 1):
        idx = src.index(old, idx + 1)
    return src[:idx] + new + src[idx + len(old):]


def _pins_fail(lib):
    saved = O._lib
    O._lib = lib
    failed = []
    try:
        for i, pin in enumerate(PINS):
            try:
                pin()
            except AssertionError:
                failed.append(i)
    finally:
        O._lib = saved
    return failed


def test_unmodified_oracle_passes_every_pin():
    assert _pins_fail(O._load()) == []


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, occ):
    src = open(os.path.join(os.path.dirname(O.__file__), "qs_oracle.c")).read()
    path = tmp_path / "mutant.c"
    path.write_text(_mutate(src, old, new, occ))
    lib = O.load_library(O.compile_source(str(path), str(tmp_path / "libmutant.so")))
    assert _pins_fail(lib), f"no pin caught the planted mistake: {name}"
