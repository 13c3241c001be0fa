"""Pins of the CPU FP64 oracle against things other than itself.

* Eq. 1 (Section 2): a gate on qubit k is the dense operator
  I (x) ... (x) Q (x) ... (x) I.  Qubit n-1 is the leftmost Kronecker factor and
  qubit 0 the rightmost, the only ordering consistent with the stride 2^k of
  Section 2.  The oracle's pair loops (Eq. 2 / Eq. 3 / Fig. 3) must equal the
  dense matrix-vector product built with numpy's kron for every k, (c, t).
* Closed forms: H on every qubit of |0..0>; the QFT of a basis state; GHZ.
* Invariants: norm preservation; a circuit followed by its inverse.
* Permutation circuits (X, CNOT, SWAP) move amplitudes bit-for-bit, with the
  index map computed by independent bit manipulation.
* Reductions against brute force on dense numpy arrays.
* Gradients against the closed form of RY(theta)|0> measured in Z, a
  one-layer closed form, and the parameter-shift rule evaluated with an
  independent dense simulator (scipy's matrix exponential of the generators).
"""

import math

import numpy as np
import pytest
import scipy.linalg

import qsgen as G
from oracle import oracle as O

I2 = np.eye(2, dtype=np.complex128)
P0 = np.diag([1, 0]).astype(np.complex128)
P1 = np.diag([0, 1]).astype(np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.diag([1, -1]).astype(np.complex128)


def mat2(m8):
    q = [complex(m8[2 * j], m8[2 * j + 1]) for j in range(4)]
    return np.array([[q[0], q[1]], [q[2], q[3]]], dtype=np.complex128)


def embed(n, factors):
    """Kronecker product with qubit n-1 leftmost; ``factors`` maps qubit -> 2x2."""
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, factors.get(q, I2))
    return out


def dense_gate(n, g, theta=None):
    kind = int(g["kind"])
    if kind == G.G_U1:
        return embed(n, {int(g["t"]): mat2(g["m"])})
    if kind == G.G_CU:
        c, t = int(g["c"]), int(g["t"])
        return embed(n, {c: P0}) + embed(n, {c: P1, t: mat2(g["m"])})
    if kind == G.G_SWAP:
        a, b = int(g["t"]), int(g["c"])
        # SWAP = (I + XX + YY + ZZ) / 2
        return 0.5 * (np.eye(1 << n) + embed(n, {a: PX, b: PX}) + embed(n, {a: PY, b: PY}) + embed(n, {a: PZ, b: PZ}))
    gen = {G.G_RX: PX, G.G_RY: PY, G.G_RZ: PZ}[kind]
    u = scipy.linalg.expm(-0.5j * theta[int(g["param"])] * gen)
    return embed(n, {int(g["t"]): u})


def random_state(n, rng):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def haar(rng_seed):
    return G.haar_2x2(G.SplitMix64(rng_seed))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_single_qubit_gate_equals_kronecker_operator(n):
    rng = np.random.default_rng(n)
    for k in range(n):
        g = G.gate_u1(k, haar(100 * n + k))[0]
        psi = random_state(n, rng)
        want = dense_gate(n, g) @ psi
        got = psi.copy()
        O.apply_1q(got, k, g["m"])
        assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_controlled_gate_equals_kronecker_operator(n):
    rng = np.random.default_rng(10 + n)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            g = G.gate_cu(c, t, haar(1000 * n + 10 * c + t))[0]
            psi = random_state(n, rng)
            want = dense_gate(n, g) @ psi
            got = psi.copy()
            O.apply_ctrl(got, c, t, g["m"])
            assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 5])
def test_swap_equals_pauli_formula(n):
    rng = np.random.default_rng(20 + n)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            g = G.gate_swap(a, b)[0]
            psi = random_state(n, rng)
            want = dense_gate(n, g) @ psi
            got = psi.copy()
            O.apply_swap(got, a, b)
            assert np.max(np.abs(got - want)) < 1e-14


def test_random_circuit_equals_dense_product_n8():
    n = 8
    gates, _ = G.random_circuit(n, 60, 7)
    gates = G.concat([gates, G.gate_swap(1, 6), G.gate_swap(7, 0)])
    u = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        u = dense_gate(n, g) @ u
    want = u[:, 0]
    got = O.simulate(n, gates)
    assert np.max(np.abs(got - want)) < 1e-13


def test_hadamard_layer_closed_form():
    for n in (1, 4, 9, 14):
        gates = G.concat([G.gate_u1(k, G.MAT_H) for k in range(n)])
        psi = O.simulate(n, gates)
        assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10, 13])
def test_qft_of_basis_state_closed_form(n):
    x = G.random_basis(n, 77 + n)
    psi = O.simulate(n, G.qft_circuit(n), x=x)
    y = np.arange(1 << n, dtype=np.uint64)
    # exact integer phase x*y mod 2^n before the floating-point exponential
    ph = (np.uint64(x) * y) & np.uint64((1 << n) - 1)
    want = np.exp(2j * np.pi * ph.astype(np.float64) / (1 << n)) * 2.0 ** (-n / 2)
    assert np.max(np.abs(psi - want)) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 8, 13])
def test_qft_closed_form_routines_match_the_circuit(n):
    """Both closed-form QFT routines of the oracle (the per-index Python one used
    for sampled amplitudes, and or_qft_basis that fills a whole state, serial and
    OpenMP builds) reproduce the oracle's own simulation of the QFT circuit, which
    the closed form above and the Kronecker pins fix."""
    for x in (0, 1, (1 << n) - 1, G.random_basis(n, 5 + n)):
        circ = O.simulate(n, G.qft_circuit(n), x=x)
        ys = np.arange(1 << n)
        assert np.max(np.abs(O.qft_basis_amplitudes(n, x, ys) - circ)) < 1e-13
        assert np.max(np.abs(O.qft_basis_state(n, x) - circ)) < 1e-13
        assert np.array_equal(O.qft_basis_state(n, x, parallel=True), O.qft_basis_state(n, x))


def test_openmp_build_is_bit_identical():
    """The -O3 -fopenmp build of the same source splits only the pair loops, so its
    states equal the serial build's bit for bit, for every gate kind and for
    targets on both sides of the outer/inner split (n = 16: groups < 64 from k = 10)."""
    n = 16
    gates = G.concat([G.random_circuit(n, 400, 31)[0], G.qft_circuit(n), G.gate_swap(0, n - 1),
                      G.gate_swap(n - 2, 3), G.gate_cu(n - 1, 0, G.haar_2x2(G.SplitMix64(2))),
                      G.gate_cu(0, n - 1, G.haar_2x2(G.SplitMix64(4)))])
    a = O.simulate(n, gates, x=12345)
    b = O.simulate(n, gates, x=12345, parallel=True)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_sampled_gradient_equals_the_full_gradient():
    """grad_sampled (the derivative's definition for chosen parameters, sharing
    the prefix state) reproduces or_grad, which the parameter-shift and
    closed-form pins below fix, for every parameter, in both builds."""
    for n, obs in ((5, G.ising_observable(5, 2)), (7, G.z_zz_observable(7, 3))):
        g, p = G.ansatz(n, 3)
        g = G.concat([g, G.gate_rot(G.G_RX, n - 1, p), G.gate_swap(0, n - 1)])
        th = G.angles(p + 1, 9)
        e, gr = O.grad(n, g, th, obs)
        for parallel in (False, True):
            e2, gs = O.grad_sampled(n, g, th, obs, list(range(p + 1))[::-1], parallel=parallel)
            assert abs(e2 - e) < 1e-14
            assert max(abs(gs[k] - gr[k]) for k in gs) < 1e-14


def _gate_operator(g, q):
    """The 2^q x 2^q operator of one gate record on qubits < q, from numpy.kron
    (qubit q-1 leftmost, Eq. 1 with the stride-2^k order)."""
    m = g["m"]
    Q = np.array([[m[0] + 1j * m[1], m[2] + 1j * m[3]], [m[4] + 1j * m[5], m[6] + 1j * m[7]]])
    if int(g["kind"]) == G.G_U1:
        return _embed(Q, g["t"], q)
    P0, P1 = np.diag([1.0, 0.0]), np.diag([0.0, 1.0])
    return _kron_list([P0 if k == g["c"] else np.eye(2) for k in reversed(range(q))]) + \
        _kron_list([P1 if k == g["c"] else (Q if k == g["t"] else np.eye(2)) for k in reversed(range(q))])


def _kron_list(ms):
    out = np.eye(1)
    for m in ms:
        out = np.kron(out, m)
    return out


def _embed(Q, k, q):
    return _kron_list([Q if j == k else np.eye(2) for j in reversed(range(q))])


@pytest.mark.parametrize("n,q", [(3, 1), (6, 3), (8, 6), (8, 8)])
def test_dense_block_equals_kronecker_operator(n, q):
    """or_apply_dense applies I (x) U: qubits 0..q-1 are the low bits of the index."""
    rng = np.random.default_rng(n * 10 + q)
    U = rng.standard_normal((1 << q, 1 << q)) + 1j * rng.standard_normal((1 << q, 1 << q))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    want = np.kron(np.eye(1 << (n - q)), U) @ psi
    for parallel in (False, True):
        got = O.apply_dense(psi.copy(), U, parallel=parallel)
        assert np.max(np.abs(got - want)) < 1e-12


def test_dense_block_of_a_gate_run_equals_the_run():
    """The product of a run of gates on the lowest q qubits, built from Kronecker
    operators, applied as one block reproduces the oracle's gate-by-gate run."""
    n, q = 12, 6
    rng = G.SplitMix64(77)
    gates = []
    for j in range(40):
        t = j % q
        if j % 3 == 2:
            gates.append(G.gate_cu((t + 1 + j % (q - 1)) % q, t, G.haar_2x2(rng)))
        else:
            gates.append(G.gate_u1(t, G.haar_2x2(rng)))
    gates = G.concat(gates)
    U = np.eye(1 << q, dtype=np.complex128)
    for g in gates:
        U = _gate_operator(g, q) @ U
    psi = np.random.default_rng(5).standard_normal(1 << n) + 0j
    psi /= np.linalg.norm(psi)
    want = O.run(psi.copy(), gates)
    assert np.max(np.abs(O.apply_dense(psi.copy(), U) - want)) < 1e-13


def test_qft_gate_counts_match_table3():
    rows = [tuple(map(int, ln.split())) for ln in open(_golden("qft_gate_counts.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 12
    for n, ngates in rows:
        assert len(G.qft_circuit(n, swaps=False)) == ngates
        assert len(G.qft_circuit(n, swaps=True)) == ngates + n // 2


def test_ghz_closed_form():
    for n in (2, 5, 11):
        gates = [G.gate_u1(0, G.MAT_H)] + [G.gate_cu(i, i + 1, G.MAT_X) for i in range(n - 1)]
        psi = O.simulate(n, G.concat(gates))
        want = np.zeros(1 << n, dtype=np.complex128)
        want[0] = want[-1] = 1 / math.sqrt(2)
        assert np.max(np.abs(psi - want)) < 1e-15


def test_norm_preserved_and_inverse_returns_input():
    n = 12
    rng = np.random.default_rng(3)
    psi0 = random_state(n, rng)
    gates, _ = G.random_circuit(n, 300, 11)
    gates = G.concat([gates, G.qft_circuit(n)])
    psi = O.run(psi0.copy(), gates)
    assert abs(O.norm2(psi) - 1.0) < 1e-13
    back = O.run(psi, G.inverse_circuit(gates))
    assert np.max(np.abs(back - psi0)) < 1e-13


def _perm_circuit(n, count, seed):
    rng = G.SplitMix64(seed)
    gates = []
    for _ in range(count):
        r = rng.randint(3)
        a = rng.randint(n)
        b = (a + 1 + rng.randint(n - 1)) % n
        if r == 0:
            gates.append(G.gate_u1(a, G.MAT_X))
        elif r == 1:
            gates.append(G.gate_cu(a, b, G.MAT_X))
        else:
            gates.append(G.gate_swap(a, b))
    return G.concat(gates)


def _perm_index(i, gates):
    for g in gates:
        k, t, c = int(g["kind"]), int(g["t"]), int(g["c"])
        if k == G.G_U1:
            i ^= 1 << t
        elif k == G.G_CU:
            if (i >> c) & 1:
                i ^= 1 << t
        else:
            bt, bc = (i >> t) & 1, (i >> c) & 1
            if bt != bc:
                i ^= (1 << t) | (1 << c)
    return i


def test_permutation_circuits_are_bit_exact():
    n = 9
    gates = _perm_circuit(n, 120, 5)
    rng = np.random.default_rng(9)
    # random non-zero amplitudes: every output must be a bit-identical copy of one input
    psi0 = (rng.uniform(0.5, 1.0, 1 << n) * rng.choice([-1, 1], 1 << n)
            + 1j * rng.uniform(0.5, 1.0, 1 << n) * rng.choice([-1, 1], 1 << n))
    got = O.run(psi0.copy(), gates)
    perm = np.array([_perm_index(i, gates) for i in range(1 << n)])
    want = np.empty_like(psi0)
    want[perm] = psi0
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    for x in (0, 5, 300, (1 << n) - 1):
        psi = O.simulate(n, gates, x=x)
        j = _perm_index(x, gates)
        assert psi[j] == 1.0 and np.count_nonzero(psi) == 1


def test_reductions_brute_force():
    n = 7
    rng = np.random.default_rng(4)
    psi = random_state(n, rng)
    p = np.abs(psi) ** 2
    assert np.max(np.abs(O.probs(psi) - p)) < 1e-16
    want = [p.reshape(-1, 2, 1 << k)[:, 1, :].sum() for k in range(n)]
    assert np.max(np.abs(O.marginals(psi) - want)) < 1e-15
    assert abs(O.norm2(psi) - 1.0) < 1e-14
    rows = [(G.P_Z, 2, -1, 0.7), (G.P_ZZ, 0, 5, -1.3), (G.P_X, 4, -1, 0.45), (G.P_X, 0, -1, -2.0), (G.P_ZZ, 6, 1, 0.2)]
    terms = G.terms(rows)
    h = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for kind, q0, q1, coef in rows:
        if kind == G.P_Z:
            h += coef * embed(n, {q0: PZ})
        elif kind == G.P_ZZ:
            h += coef * embed(n, {q0: PZ, q1: PZ})
        else:
            h += coef * embed(n, {q0: PX})
    want = float(np.real(np.vdot(psi, h @ psi)))
    assert abs(O.expect(psi, terms) - want) < 1e-14


def _dense_energy(n, gates, theta, h):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    for g in gates:
        psi = dense_gate(n, g, theta) @ psi
    return float(np.real(np.vdot(psi, h @ psi)))


def _dense_h(n, terms):
    h = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in terms:
        kind, q0, q1, coef = int(t["kind"]), int(t["q0"]), int(t["q1"]), float(t["coef"])
        f = {G.P_Z: {q0: PZ}, G.P_ZZ: {q0: PZ, q1: PZ}, G.P_X: {q0: PX}}[kind]
        h += coef * embed(n, f)
    return h


def test_gradient_closed_form_ry_z():
    g = G.gate_rot(G.G_RY, 0, 0)
    obs = G.terms([(G.P_Z, 0, -1, 1.0)])
    for th in (-2.5, -0.3, 0.0, 0.9, 3.0):
        e, gr = O.grad(1, g, np.array([th]), obs)
        assert abs(e - math.cos(th)) < 1e-15
        assert abs(gr[0] + math.sin(th)) < 1e-15


def test_gradient_one_layer_closed_form():
    n = 5
    gates = G.concat([G.gate_rot(G.G_RY, q, q) for q in range(n)] + [G.gate_rot(G.G_RZ, q, n + q) for q in range(n)])
    theta = G.angles(2 * n, 42)
    obs = G.z_zz_observable(n, 43)
    a = [float(t["coef"]) for t in obs if t["kind"] == G.P_Z]
    b = [float(t["coef"]) for t in obs if t["kind"] == G.P_ZZ]
    cy = np.cos(theta[:n])
    sy = np.sin(theta[:n])
    e_want = sum(a[i] * cy[i] for i in range(n)) + sum(b[i] * cy[i] * cy[i + 1] for i in range(n - 1))
    g_want = np.zeros(2 * n)
    for i in range(n):
        g_want[i] = -a[i] * sy[i]
        if i + 1 < n:
            g_want[i] += -b[i] * sy[i] * cy[i + 1]
        if i > 0:
            g_want[i] += -b[i - 1] * cy[i - 1] * sy[i]
    e, gr = O.grad(n, gates, theta, obs)
    assert abs(e - e_want) < 1e-13
    assert np.max(np.abs(gr - g_want)) < 1e-13


@pytest.mark.parametrize("observable", ["zzz", "ising"])
def test_gradient_parameter_shift_dense(observable):
    n, layers = 4, 2
    gates, p = G.ansatz(n, layers)
    gates = G.concat([gates, G.gate_rot(G.G_RX, 2, 1)])  # a shared parameter and an RX
    theta = G.angles(p, 5)
    obs = G.z_zz_observable(n, 6) if observable == "zzz" else G.ising_observable(n, 6)
    h = _dense_h(n, obs)
    e, gr = O.grad(n, gates, theta, obs)
    assert abs(e - _dense_energy(n, gates, theta, h)) < 1e-13
    # parameter shift: exact for exp(-i theta P / 2) gates, summed over a shared parameter's uses
    ps = np.zeros(p)
    for j, g in enumerate(gates):
        q = int(g["param"])
        if q < 0:
            continue
        # shift only this occurrence: give it a private copy of the parameter
        g2 = gates.copy()
        g2[j]["param"] = p
        th_p = np.append(theta, theta[q] + math.pi / 2)
        th_m = np.append(theta, theta[q] - math.pi / 2)
        ps[q] += 0.5 * (_dense_energy(n, g2, th_p, h) - _dense_energy(n, g2, th_m, h))
    assert np.max(np.abs(gr - ps)) < 1e-12
    # and central finite differences in FP64
    fd = np.zeros(p)
    hstep = 1e-6
    for q in range(p):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += hstep
        tm[q] -= hstep
        fd[q] = (_dense_energy(n, gates, tp, h) - _dense_energy(n, gates, tm, h)) / (2 * hstep)
    assert np.max(np.abs(gr - fd)) < 1e-8


def test_rotation_matrices_match_matrix_exponential():
    for kind, gen in ((G.G_RX, PX), (G.G_RY, PY), (G.G_RZ, PZ)):
        for th in (-1.1, 0.4, 2.9):
            m = O.gate_matrix(G.gate_rot(kind, 0, 0), np.array([th]))
            assert np.max(np.abs(mat2(m) - scipy.linalg.expm(-0.5j * th * gen))) < 1e-15


def test_invalid_records_are_rejected():
    psi = O.basis(3)
    with pytest.raises(ValueError):
        O.run(psi, G.gate_u1(3, G.MAT_H))
    bad = G.gate_cu(0, 1, G.MAT_X)
    bad["c"] = 1
    with pytest.raises(ValueError):
        O.run(psi, bad)
    with pytest.raises(ValueError):
        O.run(psi, G.gate_rot(G.G_RY, 0, 0))  # no angle array


def _golden(name):
    import os
    return os.path.join(os.path.dirname(__file__), "golden", name)
