"""Seeded input generators: determinism, published vectors, distributions."""

import os

import numpy as np

import qsgen as G


def test_splitmix64_published_vector():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(ln, 16) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    r = G.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == want


def test_haar_matrices_are_unitary():
    rng = G.SplitMix64(5)
    for _ in range(200):
        q = np.array(G.haar_2x2(rng)).reshape(2, 2)
        assert np.max(np.abs(q.conj().T @ q - np.eye(2))) < 1e-15


def test_haar_first_row_modulus_is_uniform():
    # For Haar 2x2 unitaries |q11|^2 is uniform on [0, 1].
    rng = G.SplitMix64(6)
    v = np.array([abs(G.haar_2x2(rng)[0]) ** 2 for _ in range(4000)])
    hist, _ = np.histogram(v, bins=4, range=(0, 1))
    assert np.all(np.abs(hist - 1000) < 150)


def test_random_circuit_mix_and_validity():
    n = 30
    gates, names = G.random_circuit(n, 20000, 1)
    frac_1q = np.mean(gates["kind"] == G.G_U1)
    assert abs(frac_1q - 0.7) < 0.02
    for nm in ("H", "X", "T", "HAAR"):
        assert abs(names.count(nm) / 20000 - 0.175) < 0.02
    for nm in ("CNOT", "CPHASE"):
        assert abs(names.count(nm) / 20000 - 0.15) < 0.02
    assert gates["t"].min() >= 0 and gates["t"].max() == n - 1
    cu = gates[gates["kind"] == G.G_CU]
    assert np.all(cu["c"] != cu["t"]) and cu["c"].min() == 0 and cu["c"].max() == n - 1


def test_generators_are_deterministic():
    a, _ = G.random_circuit(20, 200, 1000)
    b, _ = G.random_circuit(20, 200, 1000)
    assert a.tobytes() == b.tobytes()
    x = G.batch_instances(1003, count=8)
    y = G.batch_instances(1003, count=8)
    for p, q in zip(x, y):
        assert p["n"] == q["n"] and p["gates"].tobytes() == q["gates"].tobytes()
        assert np.array_equal(p["theta"], q["theta"]) and p["terms"].tobytes() == q["terms"].tobytes()


def test_ansatz_shape():
    g, p = G.ansatz(28, 20)
    assert p == 1120 and len(g) == 1660
    g, p = G.ansatz(10, 8)
    assert p == 16 * 10 and len(g) == 8 * (3 * 10 - 1)
