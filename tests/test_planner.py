"""Host logic of the planner, on the CPU (dry-run plans allocate no device memory).

* every gate lands in exactly one pass;
* a tile pass holds at most 2^b amplitudes' worth of qubits and contains the
  mixing qubits of each of its gates (target, both swap qubits; none for
  diagonal gates);
* the execution order only moves a gate ahead of gates it commutes with
  (disjoint qubits, or both diagonal), and the oracle applying the gates in
  execution order reproduces the circuit-order state.
"""

import ctypes

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O
from paper_1601_07195_gb300 import qs


def fake_state(n, dt):
    h = ctypes.c_void_p()
    assert qs.load().qs_wrap(ctypes.c_void_p(1 << 30), n, dt, None, ctypes.byref(h)) == qs.QS_OK
    return qs.State(h.value, n, dt)


def is_diag(g):
    k = int(g["kind"])
    if k == G.G_SWAP:
        return False
    if k == G.G_RZ:
        return True
    if k in (G.G_RX, G.G_RY):
        return False
    m = g["m"]
    return m[2] == 0 and m[3] == 0 and m[4] == 0 and m[5] == 0


def support(g):
    s = {int(g["t"])}
    if int(g["c"]) >= 0:
        s.add(int(g["c"]))
    return s


def mixing(g):
    if int(g["kind"]) == G.G_SWAP:
        return support(g)
    return set() if is_diag(g) else {int(g["t"])}


def commute(a, b):
    return not (support(a) & support(b)) or (is_diag(a) and is_diag(b))


CASES = {
    "random20": lambda: (20, G.random_circuit(20, 200, 1000)[0], None),
    "qft30+random": lambda: (30, G.concat([G.qft_circuit(30), G.random_circuit(30, 1000, 1001)[0]]), None),
    "ansatz12": lambda: (12, G.ansatz(12, 4)[0], G.angles(96, 1)),
    "qft7": lambda: (7, G.qft_circuit(7), None),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("tile_bits", [0, 2, 5, 8, 11])
def test_plan_is_a_valid_reordering(case, dt, tile_bits):
    n, gates, theta = CASES[case]()
    st = fake_state(n, dt)
    p = qs.Plan(st, gates, theta, flags=qs.PLAN_DRY_RUN, tile_bits=tile_bits)
    passes = p.passes()
    order = [g for ps in passes for g in ps["gates"]]
    assert sorted(order) == list(range(len(gates)))
    b = tile_bits if tile_bits else 12
    b = min(b, n)
    for ps in passes:
        if ps["kind"] == "tile":
            assert bin(ps["mask"]).count("1") == b
            for j in ps["gates"]:
                assert all((ps["mask"] >> q) & 1 for q in mixing(gates[j]))
        elif ps["kind"] == "dense":  # complex64: a run of consecutive gates on qubits 0..5
            assert dt == qs.QS_C64 and ps["mask"] == 0x3F and ps["n_gates"] >= 10
            assert ps["gates"] == list(range(ps["gates"][0], ps["gates"][0] + ps["n_gates"]))
            assert all(int(gates[j]["t"]) < 6 and int(gates[j]["c"]) < 6 for j in ps["gates"])
        else:
            assert ps["n_gates"] == 1
    pos = {g: i for i, g in enumerate(order)}
    for a in range(len(gates)):
        for c in range(a + 1, min(len(gates), a + 600)):
            if pos[c] < pos[a]:
                assert commute(gates[a], gates[c]), (a, c)
    with pytest.raises(qs.QSError):
        p.execute()  # dry-run plans never launch
    p.close()
    st.close()


def test_execution_order_reproduces_the_state():
    n = 12
    gates = G.concat([G.qft_circuit(n), G.random_circuit(n, 400, 3)[0]])
    st = fake_state(n, 1)
    p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN, tile_bits=6)
    order = [g for ps in p.passes() for g in ps["gates"]]
    assert order != list(range(len(gates)))  # the planner did move gates
    a = O.simulate(n, gates, x=5)
    b = O.simulate(n, gates[order], x=5)
    assert np.max(np.abs(a - b)) < 1e-13


def test_fusion_reduces_passes_for_the_n30_workload():
    n = 30
    gates = G.concat([G.qft_circuit(n), G.random_circuit(n, 1000, 1001)[0]])
    st = fake_state(n, 1)
    fused = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN).stats()
    unfused = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_FUSION).stats()
    assert unfused["passes"] == len(gates)
    assert fused["passes"] < len(gates) / 4


def test_no_fusion_keeps_circuit_order():
    n, gates, _ = CASES["random20"]()
    st = fake_state(n, 1)
    p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_FUSION)
    assert [g for ps in p.passes() for g in ps["gates"]] == list(range(len(gates)))


def test_tuning_table_roundtrip_and_planner_uses_it():
    from paper_1601_07195_gb300 import autotune as A
    assert A.tune_get(qs.QS_C64, 17) == (12, 4)  # built-in default
    A.tune_set(qs.QS_C64, 17, 9, 3)
    assert A.tune_get(qs.QS_C64, 17) == (9, 3)
    st = fake_state(17, qs.QS_C64)
    p = qs.Plan(st, G.random_circuit(17, 100, 2)[0], flags=qs.PLAN_DRY_RUN)
    assert all(bin(x["mask"]).count("1") == 9 for x in p.passes() if x["kind"] == "tile")
    A.tune_set(qs.QS_C64, 17, 12, 4)
    with pytest.raises(qs.QSError):
        A.tune_set(qs.QS_C64, 17, 20, 3)


def test_autotune_cache_file_roundtrip(tmp_path, monkeypatch):
    from paper_1601_07195_gb300 import autotune as A
    cache = tmp_path / "tune.json"
    import json
    cache.write_text(json.dumps({"FAKE GPU": {"c128/21": {"tile_bits": 11, "run_bits": 4, "ms": 1.0, "gates": 10}}}))
    assert A.apply_cache(str(cache), device="FAKE GPU") == 1
    assert A.tune_get(qs.QS_C128, 21) == (11, 4)
    assert A.apply_cache(str(cache), device="OTHER") == 0


def test_balanced_real_counts():
    """qs_plan_pass_balanced: complex128 double-float plans apply real gates whose
    entries share one magnitude (H, HX, XH, ZH) in balanced form; RY-type real
    gates, complex64 and native-FP64 plans report none."""
    n = 14
    r2 = 1 / np.sqrt(2)
    gates = G.concat([G.gate_u1(3, G.MAT_H), G.gate_u1(5, (r2, r2, -r2, r2)), G.gate_u1(6, G.MAT_H),
                      G.gate_rot(G.G_RY, 7, 0), G.gate_cu(1, 8, G.MAT_H), G.gate_u1(9, G.MAT_X)])
    theta = np.array([0.3])

    def totals(dt, flags=0):
        p = qs.Plan(fake_state(n, dt), gates, theta, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_MERGE | flags)
        bal = np.sum([p.balanced(i) for i in range(p.stats()["passes"])], axis=0)
        real = sum(int(p.op_counts(i)[0][1]) + int(p.op_counts(i)[1][1]) for i in range(p.stats()["passes"]))
        return tuple(int(v) for v in bal), real

    # 3 single-qubit + 1 controlled H-like, plus RY
    assert totals(qs.QS_C128, qs.PLAN_NO_PRP) == ((3, 1), 5)
    # by default two of the single-qubit ones leave their scalar out (qs_plan_pass_prp),
    # the third keeps it times theirs
    assert totals(qs.QS_C128) == ((1, 1), 5)
    p = qs.Plan(fake_state(n, qs.QS_C128), gates, theta, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_MERGE)
    assert sum(p.scalar_free(i)[1] for i in range(p.stats()["passes"])) == 2
    assert totals(qs.QS_C64)[0] == (0, 0)
    assert totals(qs.QS_C128, qs.PLAN_ARITH_F64)[0] == (0, 0)


def _random_mixed_circuit(n, count, seed):
    """Single-qubit gates of every class, controlled gates, swaps and rotations."""
    rng = G.SplitMix64(seed)
    out = []
    for _ in range(count):
        a = rng.randint(n)
        b = (a + 1 + rng.randint(n - 1)) % n
        k = rng.randint(9)
        if k == 0:
            out.append(G.gate_u1(a, G.haar_2x2(rng)))
        elif k == 1:
            out.append(G.gate_u1(a, G.MAT_H))
        elif k == 2:
            out.append(G.gate_u1(a, G.MAT_T))
        elif k == 3:
            out.append(G.gate_u1(a, G.MAT_X))
        elif k == 4:
            out.append(G.gate_cu(a, b, G.MAT_X))
        elif k == 5:
            out.append(G.gate_cu(a, b, G.mat_cphase(rng.uniform_range(0.0, 6.0))))
        elif k == 6:
            out.append(G.gate_swap(a, b))
        elif k == 7:
            out.append(G.gate_rot(G.G_RZ, a, 0))
        else:
            out.append(G.gate_cu(a, b, G.haar_2x2(rng)))
    return G.concat(out)


def test_random_plans_are_valid_reorderings():
    """Property test over random circuits, qubit counts and tile shapes: every
    gate is planned once, each tile pass holds its gates' mixing qubits, a gate
    only moves ahead of gates it commutes with, and the oracle applying the
    gates in execution order reproduces the circuit-order state."""
    hyp = pytest.importorskip("hypothesis")
    st_ = hyp.strategies

    @hyp.settings(max_examples=200, deadline=None, derandomize=True)
    @hyp.given(n=st_.integers(2, 10), count=st_.integers(1, 160), seed=st_.integers(0, 10 ** 6),
               b=st_.integers(2, 12), b0=st_.integers(0, 6), dt=st_.sampled_from([0, 1]))
    def check(n, count, seed, b, b0, dt):
        gates = _random_mixed_circuit(n, count, seed)
        theta = np.array([0.7])
        st = fake_state(n, dt)
        p = qs.Plan(st, gates, theta, flags=qs.PLAN_DRY_RUN, tile_bits=b | (min(b0, b) << 8))
        passes = p.passes()
        order = [g for ps in passes for g in ps["gates"]]
        assert sorted(order) == list(range(len(gates)))
        for ps in passes:
            if ps["kind"] == "tile":
                assert bin(ps["mask"]).count("1") == min(b, n)
                for j in ps["gates"]:
                    assert all((ps["mask"] >> q) & 1 for q in mixing(gates[j]))
        pos = {g: i for i, g in enumerate(order)}
        for a in range(len(gates)):
            for c in range(a + 1, len(gates)):
                if pos[c] < pos[a]:
                    assert commute(gates[a], gates[c]), (a, c)
        x = seed % (1 << n)
        want = O.simulate(n, gates, theta=theta, x=x)
        got = O.simulate(n, gates[order], theta=theta, x=x)
        assert np.max(np.abs(want - got)) < 1e-12
        p.close()
        st.close()

    check()


def test_prp_counts_keeper_and_scale_bound():
    """complex128 plans apply general single-qubit unitaries in phase-shear-phase
    form except one per pass that takes the pass's scalars (when no diagonal,
    anti-diagonal or non-unitary general update can); non-unitary matrices keep
    the full product; the scalars' product stays above 2^-24; complex64 plans and
    PLAN_NO_PRP apply none."""
    rng = G.SplitMix64(5)
    st = fake_state(10, qs.QS_C128)
    haar = [G.gate_u1(q, G.haar_2x2(rng)) for q in range(5)]

    def counts(gates, flags=0, state=st):
        p = qs.Plan(state, G.concat(gates), flags=qs.PLAN_DRY_RUN | flags)
        n = p.stats()["passes"]
        out = (n, sum(p.prp(i) for i in range(n)), sum(int(p.op_counts(i)[0][0]) for i in range(n)))
        p.close()
        return out

    assert counts(haar) == (1, 4, 5)
    diag = G.gate_u1(7, (np.exp(0.3j), 0.0, 0.0, np.exp(-0.2j)))
    assert counts(haar + [diag]) == (1, 5, 5)
    bad = G.gate_u1(6, (0.5, 0.5j, 0.5, 0.4))  # not unitary: keeps the full product and takes the scalars
    assert counts(haar + [bad]) == (1, 5, 6)
    assert counts(haar + [diag], flags=qs.PLAN_NO_PRP)[1] == 0
    assert counts(haar + [diag], state=fake_state(10, qs.QS_C64))[1] == 0
    # 160 unitaries on qubits 0..3 that cannot merge (a controlled X between
    # neighbours on the same qubit): one pass, some kept general by the bound
    long = []
    for k in range(160):
        long.append(G.gate_u1(k % 4, G.haar_2x2(rng)))
        long.append(G.gate_cu((k + 1) % 4, k % 4, G.MAT_X))
    n, prp, general = counts(long + [diag])
    assert n == 1 and general == 160 and 40 <= prp < 159


def test_balanced_without_scalar_counts():
    """H-like gates (four entries of one magnitude) leave q11 out in complex128
    plans: all of them when a general or diagonal update of the pass takes the
    scalars, all but the last when only they are present (it keeps its scalar
    times the others'); gates whose rows differ in magnitude keep theirs."""
    st = fake_state(10, qs.QS_C128)
    H = G.MAT_H
    hx = (G.MAT_H[1], G.MAT_H[0], G.MAT_H[3], G.MAT_H[2])  # H X
    rows = (0.6, 0.6, 0.8, -0.8)  # balanced, rows of different magnitude

    def forms(gates, flags=0):
        p = qs.Plan(st, G.concat(gates), flags=qs.PLAN_DRY_RUN | flags)
        n = p.stats()["passes"]
        out = (n, [sum(p.scalar_free(i)[k] for i in range(n)) for k in range(2)],
               sum(p.balanced(i)[0] for i in range(n)))
        p.close()
        return out

    hs = [G.gate_u1(q, H) for q in range(5)] + [G.gate_u1(5, hx)]
    assert forms(hs) == (1, [0, 5], 1)
    diag = G.gate_u1(7, (np.exp(0.3j), 0.0, 0.0, np.exp(-0.2j)))
    assert forms(hs + [diag]) == (1, [0, 6], 0)
    assert forms(hs + [G.gate_u1(8, G.haar_2x2(G.SplitMix64(3)))]) == (1, [0, 6], 0)
    assert forms(hs + [G.gate_u1(6, rows)]) == (1, [0, 5], 2)
    assert forms(hs, flags=qs.PLAN_NO_PRP) == (1, [0, 0], 6)


def test_trailing_phase_hand_over_counts():
    """A phase-shear-phase update hands its trailing phase diag(1, z) to the next
    update of the pass on the same qubit when that one is general, diagonal or
    anti-diagonal and only updates that commute with the phase (controlled ones
    with the qubit as control, diagonal controlled ones) lie in between; an H-like,
    X or controlled-X-target update in between stops it."""
    rng = G.SplitMix64(17)
    st = fake_state(10, qs.QS_C128)
    diag = G.gate_u1(7, (np.exp(0.3j), 0.0, 0.0, np.exp(-0.2j)))

    def nz(gates):
        p = qs.Plan(st, G.concat(gates + [diag]), flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_MERGE)
        n = p.stats()["passes"]
        out = [sum(p.scalar_free(i)[k] for i in range(n)) for k in (0, 2)]
        p.close()
        return out

    u = lambda q: G.gate_u1(q, G.haar_2x2(rng))
    cz = G.gate_cu(1, 0, (1.0, 0.0, 0.0, -1.0))
    cx_ctl = G.gate_cu(0, 1, G.MAT_X)   # qubit 0 as control: commutes
    cx_tgt = G.gate_cu(1, 0, G.MAT_X)   # qubit 0 as target: stops
    t0 = G.gate_u1(0, G.MAT_T)
    assert nz([u(0), cz, cx_ctl, u(0)]) == [2, 1]
    assert nz([u(0), cz, t0]) == [1, 1]
    assert nz([u(0), cx_tgt, u(0)]) == [2, 0]
    assert nz([u(0), G.gate_u1(0, G.MAT_H), u(0)]) == [2, 0]
    assert nz([u(0), G.gate_u1(0, G.MAT_X), u(0)]) == [2, 0]
    assert nz([u(0), u(1), u(0)]) == [3, 1]


def test_plan_arguments_on_the_host():
    """Plan creation on a dry-run state: an empty circuit gives an empty plan;
    a negative count, a NULL gate array, an out-of-range or repeated qubit, an
    unknown kind, a rotation without its angle and a tile of more than 14 bits
    are rejected with QS_EINVAL and a message; a run of more low qubits than
    tile bits is clamped to the tile."""
    lib = qs.load()
    st = fake_state(10, qs.QS_C128)
    p = qs.Plan(st, G.concat([]), flags=qs.PLAN_DRY_RUN)
    assert p.stats() == {"passes": 0, "tile_passes": 0, "launches": 0, "device_ops": 0}
    p.close()

    def create(gates, n=None, theta=None, tile_bits=0):
        g = np.ascontiguousarray(gates, dtype=qs.GATE_DTYPE)
        th = np.ascontiguousarray(theta if theta is not None else np.zeros(0), dtype=np.float64)
        out = ctypes.c_void_p()
        rc = lib.qs_plan_create(st.handle, g.ctypes.data if n != "null" else None,
                                len(g) if n in (None, "null") else n,
                                th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if th.size else None, th.size,
                                qs.PLAN_DRY_RUN, tile_bits, ctypes.byref(out))
        if rc == qs.QS_OK:
            lib.qs_plan_destroy(out)
        return rc, lib.qs_last_error().decode()

    h = G.gate_u1(0, G.MAT_H)
    assert create(h, n=-1) == (qs.QS_EINVAL, "negative gate count")
    assert create(h, n="null")[0] == qs.QS_EINVAL
    bad = h.copy()
    bad["t"] = 10
    assert create(bad) == (qs.QS_EINVAL, "gate 0: qubit out of range")
    cu = G.gate_cu(1, 2, G.MAT_X)
    cu["c"] = 2
    assert create(cu)[0] == qs.QS_EINVAL
    sw = G.gate_swap(1, 2)
    sw["c"] = 1
    assert create(sw)[0] == qs.QS_EINVAL
    kind = h.copy()
    kind["kind"] = 9
    assert create(kind) == (qs.QS_EINVAL, "gate 0: unknown kind")
    assert create(G.gate_rot(G.G_RY, 0, 0))[0] == qs.QS_EINVAL              # no angles
    assert create(G.gate_rot(G.G_RY, 0, 3), theta=np.array([0.1]))[0] == qs.QS_EINVAL
    assert create(h, tile_bits=15)[0] == qs.QS_EINVAL
    assert create(h, tile_bits=12 | (13 << 8))[0] == qs.QS_OK
    assert create(h, tile_bits=1)[0] == qs.QS_OK


def _low_run(length, seed):
    """`length` gates on qubits 0..5: Haar single-qubit gates, controlled Haar gates, swaps."""
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


def test_dense_runs_become_dense_passes():
    """complex64 plans: runs of >= 10 consecutive gates on qubits 0..5 become one
    dense pass each, in circuit order, with every other gate planned around
    them; a 9-gate run stays in tile passes; every gate lands once.  The pass's
    matrix is the ordered product of its gates (numpy.kron operators)."""
    n = 14
    r1, _ = G.random_circuit(n, 40, 3)
    r2, _ = G.random_circuit(n, 30, 4)
    gates = G.concat([r1, _low_run(24, 1), r2, G.gate_u1(9, G.MAT_H), _low_run(9, 2), G.gate_u1(9, G.MAT_H),
                      _low_run(10, 5)])
    st = fake_state(n, qs.QS_C64)
    p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN)
    passes = p.passes()
    dense = [ps for ps in passes if ps["kind"] == "dense"]
    low = [int(g["t"]) < 6 and int(g["c"]) < 6 for g in gates]  # maximal runs of gates on qubits 0..5
    want, i = [], 0
    while i < len(gates):
        j = i
        while j < len(gates) and low[j]:
            j += 1
        if j - i >= 10:
            want.append(list(range(i, j)))
        i = max(j, i + 1)
    assert len(want) == 2 and want[0][0] <= 40 and want[0][-1] >= 63 and want[1][-1] == len(gates) - 1
    assert [ps["gates"] for ps in dense] == want
    assert all(ps["mask"] == 0x3F for ps in dense)
    seen = sorted(j for ps in passes for j in ps["gates"])
    assert seen == list(range(len(gates)))
    # passes before a dense pass hold only earlier gates, passes after it only later ones
    for i, ps in enumerate(passes):
        if ps["kind"] != "dense":
            continue
        lo, hi = ps["gates"][0], ps["gates"][-1]
        assert all(max(q["gates"]) < lo for q in passes[:i]) and all(min(q["gates"]) > hi for q in passes[i + 1:])
    for i, ps in enumerate(passes):
        if ps["kind"] == "dense":
            U = np.eye(64, dtype=np.complex128)
            for j in ps["gates"]:
                U = _low_operator(gates[j]) @ U
            assert np.max(np.abs(p.dense_matrix(i) - U)) < 1e-13
        else:
            with pytest.raises(qs.QSError):
                p.dense_matrix(i)
    p.close()
    # with QS_PLAN_NO_DENSE, or for complex128, no dense pass
    p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_DENSE)
    assert all(ps["kind"] != "dense" for ps in p.passes())
    p.close()
    p = qs.Plan(fake_state(n, qs.QS_C128), gates, flags=qs.PLAN_DRY_RUN)
    assert all(ps["kind"] != "dense" for ps in p.passes())
    p.close()


def _low_operator(g):
    """The 64 x 64 operator of one gate record on qubits 0..5 (qubit 5 leftmost)."""
    m = g["m"]
    Q = np.array([[m[0] + 1j * m[1], m[2] + 1j * m[3]], [m[4] + 1j * m[5], m[6] + 1j * m[7]]])
    kind, t, c = int(g["kind"]), int(g["t"]), int(g["c"])
    def kron(fs):
        out = np.eye(1)
        for f in fs:
            out = np.kron(out, f)
        return out
    if kind == G.G_SWAP:
        P = np.zeros((64, 64))
        for i in range(64):
            j = i
            if ((i >> t) & 1) != ((i >> c) & 1):
                j = i ^ (1 << t) ^ (1 << c)
            P[j, i] = 1.0
        return P
    if kind == G.G_U1:
        return kron([Q if k == t else np.eye(2) for k in reversed(range(6))])
    return (kron([np.diag([1.0, 0.0]) if k == c else np.eye(2) for k in reversed(range(6))])
            + kron([np.diag([0.0, 1.0]) if k == c else (Q if k == t else np.eye(2)) for k in reversed(range(6))]))
