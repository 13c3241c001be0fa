"""Seeded synthetic circuits, parameters and observables.

This module only *describes* inputs: gate records (kind, qubits, parameter
index, 2x2 matrix), rotation angles and Pauli-sum observables.  It never
applies a gate to a state and never evaluates an expectation value, so it
holds none of the simulation arithmetic.  Both the CPU oracle and the CUDA
path read the same records.

Gate record (80 bytes, little-endian, C layout)::

    int32 kind   G_U1 / G_CU / G_SWAP / G_RX / G_RY / G_RZ
    int32 t      target qubit (first qubit for G_SWAP)
    int32 c      control qubit (second qubit for G_SWAP), -1 if none
    int32 param  index into the angle array for G_RX/G_RY/G_RZ, -1 otherwise
    float64 m[8] row-major 2x2 matrix (q11, q12, q21, q22) as (re, im) pairs;
                 zero for G_SWAP and the parameterised kinds

The 2x2 matrix names follow the single-qubit gate of Eq. 2 (q11 q12 / q21 q22,
row = output amplitude, column = input amplitude); G_CU is the controlled-Q
gate of Eq. 3.  Qubit k is bit k of the amplitude index (the stride-2^k
convention of Section 2).

Pauli term record (24 bytes)::

    int32 kind   P_Z (coef * Z_q0) / P_ZZ (coef * Z_q0 Z_q1) / P_X (coef * X_q0)
    int32 q0, q1 (q1 = -1 unless P_ZZ), int32 pad
    float64 coef
"""

import math

import numpy as np

from .rng import SplitMix64

G_U1, G_CU, G_SWAP, G_RX, G_RY, G_RZ = 0, 1, 2, 3, 4, 5
P_Z, P_ZZ, P_X = 0, 1, 2

GATE_DTYPE = np.dtype(
    [("kind", "<i4"), ("t", "<i4"), ("c", "<i4"), ("param", "<i4"), ("m", "<f8", (8,))],
    align=True,
)
TERM_DTYPE = np.dtype(
    [("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("pad", "<i4"), ("coef", "<f8")],
    align=True,
)
assert GATE_DTYPE.itemsize == 80 and TERM_DTYPE.itemsize == 24

_R2 = 1.0 / math.sqrt(2.0)

# Fixed gate matrices (q11, q12, q21, q22) as complex numbers.
MAT_H = (_R2, _R2, _R2, -_R2)
MAT_X = (0.0, 1.0, 1.0, 0.0)
MAT_T = (1.0, 0.0, 0.0, complex(_R2, _R2))  # diag(1, e^{i pi/4})


def _pack(mat):
    out = np.zeros(8, dtype=np.float64)
    for j, z in enumerate(mat):
        z = complex(z)
        out[2 * j] = z.real
        out[2 * j + 1] = z.imag
    return out


def mat_cphase(phi: float):
    """diag(1, e^{i phi}): the target factor of a controlled-phase gate."""
    return (1.0, 0.0, 0.0, complex(math.cos(phi), math.sin(phi)))


def haar_2x2(rng: SplitMix64):
    """A Haar-distributed 2x2 unitary.

    F. Mezzadri, "How to generate random matrices from the classical compact
    groups" (Notices AMS 54, 2007): QR-factorise a complex Ginibre matrix and
    make R's diagonal positive.  For 2x2 this is Gram-Schmidt on the two
    Gaussian columns, whose R already has a positive real diagonal (the second
    projection only removes rounding left by the first).
    """
    z = [complex(rng.normal(), rng.normal()) * _R2 for _ in range(4)]  # column-major: z[0],z[1] = col 0
    c0 = (z[0], z[1])
    n0 = math.sqrt(abs(c0[0]) ** 2 + abs(c0[1]) ** 2)
    c0 = (c0[0] / n0, c0[1] / n0)
    c1 = (z[2], z[3])
    for _ in range(2):  # Gram-Schmidt twice ("twice is enough", Parlett) keeps Q unitary to rounding
        proj = c0[0].conjugate() * c1[0] + c0[1].conjugate() * c1[1]
        c1 = (c1[0] - proj * c0[0], c1[1] - proj * c0[1])
    n1 = math.sqrt(abs(c1[0]) ** 2 + abs(c1[1]) ** 2)
    c1 = (c1[0] / n1, c1[1] / n1)
    return (c0[0], c1[0], c0[1], c1[1])  # row-major q11 q12 q21 q22


def gate_u1(t, mat):
    g = np.zeros(1, dtype=GATE_DTYPE)
    g["kind"], g["t"], g["c"], g["param"] = G_U1, t, -1, -1
    g["m"][0] = _pack(mat)
    return g


def gate_cu(c, t, mat):
    if c == t:
        raise ValueError("control and target must differ")
    g = np.zeros(1, dtype=GATE_DTYPE)
    g["kind"], g["t"], g["c"], g["param"] = G_CU, t, c, -1
    g["m"][0] = _pack(mat)
    return g


def gate_swap(a, b):
    if a == b:
        raise ValueError("swap needs two distinct qubits")
    g = np.zeros(1, dtype=GATE_DTYPE)
    g["kind"], g["t"], g["c"], g["param"] = G_SWAP, a, b, -1
    return g


def gate_rot(kind, t, param):
    if kind not in (G_RX, G_RY, G_RZ):
        raise ValueError("rotation kind must be G_RX, G_RY or G_RZ")
    g = np.zeros(1, dtype=GATE_DTYPE)
    g["kind"], g["t"], g["c"], g["param"] = kind, t, -1, param
    return g


def concat(gates):
    if not gates:
        return np.zeros(0, dtype=GATE_DTYPE)
    return np.concatenate(gates).astype(GATE_DTYPE, copy=False)


def random_circuit(n: int, n_gates: int, seed: int):
    """Random circuit with the gate mix of the n=20/30/33/34 workloads.

    With probability 0.7 a single-qubit gate, its type uniform over
    {H, X, T, Haar 2x2}, on a uniform qubit; otherwise a controlled gate,
    uniform over {CNOT, controlled-phase with phi ~ U[0, 2pi)}, on a uniform
    ordered pair c != t.  Returns (gate records, list of gate names).
    """
    if n < 2:
        raise ValueError("random circuits need n >= 2")
    rng = SplitMix64(seed)
    gates, names = [], []
    for _ in range(n_gates):
        if rng.uniform() < 0.7:
            k = rng.randint(n)
            which = rng.randint(4)
            if which == 0:
                gates.append(gate_u1(k, MAT_H)); names.append("H")
            elif which == 1:
                gates.append(gate_u1(k, MAT_X)); names.append("X")
            elif which == 2:
                gates.append(gate_u1(k, MAT_T)); names.append("T")
            else:
                gates.append(gate_u1(k, haar_2x2(rng))); names.append("HAAR")
        else:
            c = rng.randint(n)
            t = rng.randint(n - 1)
            if t >= c:
                t += 1
            if rng.randint(2) == 0:
                gates.append(gate_cu(c, t, MAT_X)); names.append("CNOT")
            else:
                phi = rng.uniform_range(0.0, 2.0 * math.pi)
                gates.append(gate_cu(c, t, mat_cphase(phi))); names.append("CPHASE")
    return concat(gates), names


def qft_circuit(n: int, swaps: bool = True):
    """Quantum Fourier transform on n qubits, little-endian.

    Textbook circuit (Nielsen & Chuang, Section 5.1) with the most significant
    bit on qubit n-1: for j = n-1 .. 0, H on j, then for m = j-1 .. 0 a
    controlled phase pi / 2^(j-m) with control m and target j; then, if
    ``swaps``, SWAP(j, n-1-j) for j < n/2.  Without the swaps this is
    n(n+1)/2 gates, the count of the QFT table in Section 5.5.
    """
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(gate_u1(j, MAT_H))
        for m in range(j - 1, -1, -1):
            gates.append(gate_cu(m, j, mat_cphase(math.pi / 2.0 ** (j - m))))
    if swaps:
        for j in range(n // 2):
            gates.append(gate_swap(j, n - 1 - j))
    return concat(gates)


def dagger_matrix(m8):
    """Conjugate transpose of a packed 2x2 matrix (an input transformation)."""
    q = [complex(m8[2 * j], m8[2 * j + 1]) for j in range(4)]
    return (q[0].conjugate(), q[2].conjugate(), q[1].conjugate(), q[3].conjugate())


def inverse_circuit(gates):
    """The inverse circuit of fixed gates: reversed order, each matrix daggered."""
    out = []
    for g in gates[::-1]:
        k = int(g["kind"])
        if k == G_U1:
            out.append(gate_u1(int(g["t"]), dagger_matrix(g["m"])))
        elif k == G_CU:
            out.append(gate_cu(int(g["c"]), int(g["t"]), dagger_matrix(g["m"])))
        elif k == G_SWAP:
            out.append(gate_swap(int(g["t"]), int(g["c"])))
        else:
            raise ValueError("inverse_circuit takes fixed gates only")
    return concat(out)


def ansatz(n: int, layers: int):
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, RZ(theta)
    on every qubit, then the CNOT ladder (i, i+1) for i = 0 .. n-2.

    2n parameters and 3n-1 gates per layer; parameter indices run in gate order.
    """
    gates = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(gate_rot(G_RY, q, p)); p += 1
        for q in range(n):
            gates.append(gate_rot(G_RZ, q, p)); p += 1
        for q in range(n - 1):
            gates.append(gate_cu(q, q + 1, MAT_X))
    return concat(gates), p


def angles(n_params: int, seed: int):
    rng = SplitMix64(seed)
    return np.array([rng.uniform_range(-math.pi, math.pi) for _ in range(n_params)], dtype=np.float64)


def _terms(rows):
    t = np.zeros(len(rows), dtype=TERM_DTYPE)
    for i, (kind, q0, q1, coef) in enumerate(rows):
        t[i]["kind"], t[i]["q0"], t[i]["q1"], t[i]["coef"] = kind, q0, q1, coef
    return t


def z_zz_observable(n: int, seed: int):
    """H = sum_i a_i Z_i + sum_{i<n-1} b_i Z_i Z_{i+1} with a, b ~ N(0, 1); open chain."""
    rng = SplitMix64(seed)
    rows = [(P_Z, i, -1, rng.normal()) for i in range(n)]
    rows += [(P_ZZ, i, i + 1, rng.normal()) for i in range(n - 1)]
    return _terms(rows)


def ising_observable(n: int, seed: int):
    """H = sum_{i<n-1} J_i Z_i Z_{i+1} + sum_i h_i X_i with J, h ~ N(0, 1); open chain."""
    rng = SplitMix64(seed)
    rows = [(P_ZZ, i, i + 1, rng.normal()) for i in range(n - 1)]
    rows += [(P_X, i, -1, rng.normal()) for i in range(n)]
    return _terms(rows)


def terms(rows):
    """Pauli sum from (kind, q0, q1, coef) tuples."""
    return _terms(rows)


def batch_instances(seed: int, count: int = 512, n_min: int = 10, n_max: int = 22, layers: int = 8):
    """Batched variational workload: ``count`` instances with n ~ U{n_min..n_max},
    the ansatz with ``layers`` layers, angles ~ U[-pi, pi] and a Z + ZZ observable.

    Returns a list of dicts {n, gates, theta, terms}.
    """
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = n_min + rng.randint(n_max - n_min + 1)
        gates, p = ansatz(n, layers)
        sub = rng.next_u64()
        theta = angles(p, sub)
        obs = z_zz_observable(n, sub ^ 0x5DEECE66D)
        out.append({"n": n, "gates": gates, "theta": theta, "terms": obs})
    return out


def random_basis(n: int, seed: int) -> int:
    return SplitMix64(seed).next_u64() >> (64 - n) if n > 0 else 0


# Seeds of the five synthetic workloads (n=20 random; n=30 QFT + random;
# n=33/34 random and its n=26 error run; batched ansatz; n=28 adjoint).
SEEDS = {"random20": 1000, "qft30": 1001, "random33": 1002, "batch512": 1003, "adjoint28": 1004}
