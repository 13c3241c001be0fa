"""The dense tensor-core block (qs_apply_dense) against the oracle's plain
definition (or_apply_dense: y = U x on every group of 2^q amplitudes).

complex64 states; bound 1e-5 max-abs (the complex64 bound of the path), with
the input rounded to complex64 on both sides.  Covers q = 1..6 (q < 6 widened
to I (x) U), tiles with ragged row counts (n = 6..13: fewer than the 128 rows
of one tile), many tiles per CTA, two calls in a row on one state, a gate run
folded into one block, and the n = 30 state on sampled rows."""

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1601_07195_gb300 import qs as _qs
    _qs.load()
    return _qs


def haar(d, seed):
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_c64_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex64)


@pytest.mark.parametrize("n", [6, 7, 9, 13, 14, 21])
@pytest.mark.parametrize("q", [6, 3, 1])
def test_dense_block_matches_oracle(qs, n, q):
    psi = rand_c64_state(n, 10 * n + q)
    U1, U2 = haar(1 << q, n + 100 * q), haar(1 << q, n + 100 * q + 1)
    want = psi.astype(np.complex128)
    O.apply_dense(want, U1)
    O.apply_dense(want, U2)
    with qs.State.create(n, qs.QS_C64) as s:
        s.from_numpy(psi)
        s.apply_dense(U1)
        s.apply_dense(U2)  # a second call reuses the state's operand buffers
        got = s.to_numpy()
    assert np.max(np.abs(got - want)) < TOL


def test_gate_run_as_one_block(qs):
    """40 gates on qubits 0..5 multiplied into U on the host (Kronecker
    operators) and applied as one block reproduce the oracle's gate-by-gate run."""
    n, q = 16, 6
    rng = G.SplitMix64(5)
    gates = []
    for j in range(40):
        t = j % q
        gates.append(G.gate_cu((t + 1 + j % 5) % q, t, G.haar_2x2(rng)) if j % 3 == 2 else G.gate_u1(t, G.haar_2x2(rng)))
    gates = G.concat(gates)
    U = np.eye(1 << q, dtype=np.complex128)
    for g in gates:
        m = g["m"]
        Q = np.array([[m[0] + 1j * m[1], m[2] + 1j * m[3]], [m[4] + 1j * m[5], m[6] + 1j * m[7]]])
        ops = [np.eye(2)] * q
        if int(g["kind"]) == G.G_U1:
            op = np.eye(1)
            for k in reversed(range(q)):
                op = np.kron(op, Q if k == g["t"] else np.eye(2))
        else:
            p0, p1 = np.eye(1), np.eye(1)
            for k in reversed(range(q)):
                p0 = np.kron(p0, np.diag([1.0, 0.0]) if k == g["c"] else np.eye(2))
                p1 = np.kron(p1, np.diag([0.0, 1.0]) if k == g["c"] else (Q if k == g["t"] else np.eye(2)))
            op = p0 + p1
        U = op @ U
    psi = rand_c64_state(n, 3)
    want = O.run(psi.astype(np.complex128), gates)
    with qs.State.create(n, qs.QS_C64) as s:
        s.from_numpy(psi)
        s.apply_dense(U)
        got = s.to_numpy()
    assert np.max(np.abs(got - want)) < TOL


def test_full_size_n30_sampled_rows(qs):
    """n = 30 (8 GiB complex64): the block on QFT|x>, 4096 sampled 64-amplitude
    rows compared with the oracle applied to those rows alone."""
    n = 30
    x = G.random_basis(n, 17)
    U = haar(64, 9)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.integers(0, 1 << (n - 6), 4093), [0, 1, (1 << (n - 6)) - 1]]))
    with qs.State.create(n, qs.QS_C64) as s:
        s.init_basis(x)
        s.run(G.qft_circuit(n))
        before = np.concatenate([s.to_numpy(int(r) * 64, 64) for r in rows])
        s.apply_dense(U)
        after = np.concatenate([s.to_numpy(int(r) * 64, 64) for r in rows])
    # the oracle takes whole states: the sampled rows side by side, zero rows up to a power of two
    want = np.zeros(64 * (1 << int(np.ceil(np.log2(len(rows))))), dtype=np.complex128)
    want[:before.size] = before
    O.apply_dense(want, U)
    assert np.max(np.abs(after - want[:before.size])) < TOL


def test_dense_block_rejections(qs):
    with qs.State.create(8, qs.QS_C128) as s:
        with pytest.raises(qs.QSError) as e:
            s.apply_dense(np.eye(64))
        assert e.value.status == qs.QS_EDTYPE
    with qs.State.create(5, qs.QS_C64) as s:
        with pytest.raises(qs.QSError) as e:
            s.apply_dense(np.eye(4))
        assert e.value.status == qs.QS_EINVAL
    with qs.State.create(8, qs.QS_C64) as s:
        with pytest.raises(qs.QSError):
            s.apply_dense(np.eye(128))  # q = 7
        bad = np.eye(8, dtype=np.complex128)
        bad[0, 0] = np.nan
        with pytest.raises(qs.QSError):
            s.apply_dense(bad)


def _low_run(length, seed):
    rng = G.SplitMix64(seed)
    out = []
    for j in range(length):
        t = j % 6
        if j % 7 == 6:
            out.append(G.gate_swap(t, (t + 2) % 6))
        elif j % 3 == 2:
            out.append(G.gate_cu((t + 1) % 6, t, G.haar_2x2(rng)))
        else:
            out.append(G.gate_u1(t, G.haar_2x2(rng)))
    return G.concat(out)


@pytest.mark.parametrize("graph", [False, True])
def test_dense_plan_matches_oracle(qs, graph):
    """complex64 plans: long runs on qubits 0..5 run as tensor-core passes between
    ordinary tile passes; the state matches the oracle, eager and replayed as a
    CUDA graph (twice)."""
    import torch
    n = 18
    r1, _ = G.random_circuit(n, 60, 21)
    r2, _ = G.random_circuit(n, 60, 22)
    gates = G.concat([r1, _low_run(40, 7), r2, _low_run(64, 8), G.gate_u1(12, G.MAT_H)])
    psi = rand_c64_state(n, 5)
    want = O.run(psi.astype(np.complex128), gates)
    stream = torch.cuda.Stream()
    with qs.State.create(n, qs.QS_C64, stream=stream) as s:
        s.from_numpy(psi)
        flags = qs.PLAN_GRAPH if graph else qs.PLAN_DEFAULT
        p = s.plan(gates, flags=flags)
        kinds = [ps["kind"] for ps in p.passes()]
        assert kinds.count("dense") == 2 and "tile" in kinds
        p.execute()
        stream.synchronize()
        got = s.to_numpy()
        assert np.max(np.abs(got - want)) < TOL
        if graph:  # a second replay applies the circuit again
            p.execute()
            stream.synchronize()
            O.run(want, gates)
            assert np.max(np.abs(s.to_numpy() - want)) < 2 * TOL
        p.close()
