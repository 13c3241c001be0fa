"""The planner's arithmetic, on the CPU: the tile records of complex128
double-float plans (dry-run plans, no device memory), applied by the host
reading in record_interp.py, reproduce the oracle's state.

This checks what the planner writes into the records: matrix products of
adjacent same-qubit gates, phase-run tables (per-tile-bit and outside
factors), the balanced, phase-shear-phase and scalar-free forms, the scalars
those forms leave out and the record that takes them, trailing phases moved
to a later record, and the pass order.  The kernels that read the records
are checked against the oracle by the GPU tests.
"""

import ctypes

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O
from paper_1601_07195_gb300 import qs
from tests.record_interp import run_plan

TOL = 1e-12


def fake_state(n, dt=qs.QS_C128):
    h = ctypes.c_void_p()
    assert qs.load().qs_wrap(ctypes.c_void_p(1 << 30), n, dt, None, ctypes.byref(h)) == qs.QS_OK
    return qs.State(h.value, n, dt)


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def mixed_circuit(n, count, seed):
    """Every gate class, controlled gates, swaps, rotations, runs of phase gates
    around one qubit, nearly diagonal and non-unitary general matrices."""
    rng = G.SplitMix64(seed)
    out = []
    for _ in range(count):
        a = rng.randint(n)
        b = (a + 1 + rng.randint(n - 1)) % n
        k = rng.randint(13)
        if k <= 1:
            out.append(G.gate_u1(a, G.haar_2x2(rng)))
        elif k == 2:
            h = G.MAT_H
            out.append(G.gate_u1(a, (h, (h[1], h[0], h[3], h[2]), (h[0], h[1], -h[2], -h[3]))[rng.randint(3)]))
        elif k == 3:
            out.append(G.gate_u1(a, G.MAT_T))
        elif k == 4:
            out.append(G.gate_u1(a, G.MAT_X))
        elif k == 5:
            out.append(G.gate_cu(a, b, G.MAT_X))
        elif k == 6:  # a run of controlled phases around qubit a
            for _ in range(1 + rng.randint(6)):
                c = (a + 1 + rng.randint(n - 1)) % n
                out.append(G.gate_cu(c, a, G.mat_cphase(rng.uniform_range(0.0, 6.0))))
        elif k == 7:
            out.append(G.gate_swap(a, b))
        elif k == 8:
            out.append(G.gate_rot(G.G_RZ, a, 0))
        elif k == 9:
            out.append(G.gate_rot(G.G_RY, a, 1))
        elif k == 10:
            out.append(G.gate_cu(a, b, G.haar_2x2(rng)))
        elif k == 11:  # nearly diagonal unitary
            e = 10.0 ** -(3 + rng.randint(9))
            p = np.exp(1j * rng.uniform_range(0.0, 6.0))
            out.append(G.gate_u1(a, (p * np.cos(e), -p * np.sin(e), np.sin(e), np.cos(e))))
        else:  # general, not unitary
            u = G.haar_2x2(rng)
            out.append(G.gate_u1(a, (0.8 * u[0], 0.8 * u[1], u[2], u[3])))
    return G.concat(out)


def check(n, gates, theta, flags, tile_bits, seed, dt=qs.QS_C128, tol=TOL):
    psi = rand_state(n, seed)
    want = O.run(psi.copy(), gates, theta)
    p = qs.Plan(fake_state(n, dt), gates, theta, flags=qs.PLAN_DRY_RUN | flags, tile_bits=tile_bits)
    try:
        got = run_plan(p, psi, gates, theta)
        forms = np.sum([p.scalar_free(i) for i in range(p.stats()["passes"])], axis=0)
    finally:
        p.close()
    err = np.max(np.abs(got - want))
    assert err < tol, (flags, tile_bits, err)
    return forms


FLAGS = [qs.PLAN_DEFAULT, qs.PLAN_NO_PRP, qs.PLAN_NO_MERGE, qs.PLAN_NO_PHASE_RUNS,
         qs.PLAN_NO_MERGE | qs.PLAN_NO_PHASE_RUNS | qs.PLAN_NO_PRP]


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("n,tile_bits", [(3, 0), (6, 4 | (2 << 8)), (9, 6 | (3 << 8)), (12, 0), (13, 8 | (1 << 8))])
def test_records_reproduce_oracle(n, tile_bits, flags):
    gates = mixed_circuit(n, 260, 500 + n)
    theta = np.array([0.7, -1.3])
    forms = check(n, gates, theta, flags, tile_bits, 41 + n)
    if flags in (qs.PLAN_DEFAULT, qs.PLAN_NO_MERGE, qs.PLAN_NO_PHASE_RUNS) and n >= 6:
        assert forms[0] > 0 and forms[1] > 0 and forms[2] > 0  # every form taken
    if flags & qs.PLAN_NO_PRP:
        assert not np.any(forms)


def _drun_count(p):
    count = 0
    for i in range(p.stats()["passes"]):
        recs, _, _ = p.records(i)
        count += int(np.sum(recs["kind"] == 5)) if len(recs) else 0
    return count


def diag_circuit(n, count, seed, outside_from):
    """Runs of phase gates of every kind a diagonal run takes: phases on one qubit,
    controlled phases between tile qubits of one half (low qubits 0..1, or
    2..3), and between qubits below `outside_from` and qubits at or above it
    (which the tile shapes below leave outside); between runs, a Haar gate, so
    that passes hold several runs."""
    rng = G.SplitMix64(seed)
    out = []
    for _ in range(count):
        for _ in range(4 + rng.randint(9)):
            k = rng.randint(5)
            phi = rng.uniform_range(0.0, 6.0)
            lo, hi = rng.randint(outside_from), outside_from + rng.randint(n - outside_from)
            if k == 0:
                out.append(G.gate_u1((lo, hi)[rng.randint(2)], G.mat_cphase(phi)))  # a phase on one qubit
            elif k == 1:
                out.append(G.gate_cu(lo, hi, G.mat_cphase(phi)))
            elif k == 2:
                out.append(G.gate_cu(hi, lo, G.mat_cphase(phi)))
            elif k == 3:
                a = rng.randint(2)
                out.append(G.gate_cu(a, 1 - a, G.mat_cphase(phi)))
            else:
                h2 = (outside_from + rng.randint(n - outside_from), outside_from + rng.randint(n - outside_from))
                if h2[0] != h2[1]:
                    out.append(G.gate_cu(h2[0], h2[1], G.mat_cphase(phi)))
        out.append(G.gate_u1(rng.randint(n), G.haar_2x2(rng)))
    return G.concat(out)


@pytest.mark.parametrize("dt,tol", [(qs.QS_C128, TOL), (qs.QS_C64, 1e-5)])
@pytest.mark.parametrize("n,tile_bits", [(9, 4 | (2 << 8)), (12, 6 | (2 << 8)), (14, 8 | (3 << 8))])
def test_diagonal_runs_reproduce_oracle(n, tile_bits, dt, tol):
    """Runs of phase gates whose phase separates over the two halves of the tile
    bits become one diagonal-run record set (kind 5): bit terms with and without
    an outside condition, pair terms inside one half, scalar terms of outside
    qubits.  Applied on the host they give the oracle's state; without them
    (QS_PLAN_NO_DIAG_RUNS) there are none and the state is the same."""
    gates = diag_circuit(n, 12, 900 + n, outside_from=4)
    psi = rand_state(n, 3 + n)
    want = O.run(psi.copy(), gates)
    for flags, expect_runs in ((qs.PLAN_DEFAULT, True), (qs.PLAN_NO_DIAG_RUNS, False)):
        p = qs.Plan(fake_state(n, dt), gates, flags=qs.PLAN_DRY_RUN | flags, tile_bits=tile_bits)
        try:
            assert (_drun_count(p) > 0) == expect_runs
            got = run_plan(p, psi, gates)
        finally:
            p.close()
        assert np.max(np.abs(got - want)) < tol, (flags, np.max(np.abs(got - want)))


@pytest.mark.parametrize("n,tile_bits", [(12, 6 | (2 << 8)), (16, 8 | (4 << 8))])
def test_inverse_qft_diagonal_runs(n, tile_bits):
    """The inverse QFT's controlled phases whose target lies outside the tile
    form diagonal runs; the records reproduce the oracle's inverse QFT of a
    random state, and the plan holds fewer records than without the runs."""
    gates = G.inverse_circuit(G.qft_circuit(n))
    psi = rand_state(n, 17 + n)
    want = O.run(psi.copy(), gates)
    ops = {}
    for flags in (qs.PLAN_DEFAULT, qs.PLAN_NO_DIAG_RUNS):
        p = qs.Plan(fake_state(n), gates, flags=qs.PLAN_DRY_RUN | flags, tile_bits=tile_bits)
        try:
            if flags == qs.PLAN_DEFAULT:
                assert _drun_count(p) > 0
            ops[flags] = p.stats()["device_ops"]
            got = run_plan(p, psi, gates)
        finally:
            p.close()
        assert np.max(np.abs(got - want)) < TOL, flags
    assert ops[qs.PLAN_DEFAULT] < ops[qs.PLAN_NO_DIAG_RUNS]


def test_diagonal_run_op_counts():
    """A pass whose only records are one diagonal run reports it as two
    single-qubit diagonal updates (two complex products on every amplitude),
    and as one device op; without the runs the same gates count one by one."""
    n = 10
    gates = G.concat([G.gate_u1(q, G.mat_cphase(0.1 * q + 0.3)) for q in range(6)])  # phases, no shared qubit
    p = qs.Plan(fake_state(n), gates, flags=qs.PLAN_DRY_RUN, tile_bits=8 | (4 << 8))
    try:
        assert _drun_count(p) == 1
        counts = sum(p.op_counts(i) for i in range(p.stats()["passes"]))
        assert counts[0][2] == 2 and counts.sum() == 2 and p.stats()["device_ops"] == 1
    finally:
        p.close()
    p = qs.Plan(fake_state(n), gates, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_DIAG_RUNS, tile_bits=8 | (4 << 8))
    try:
        assert _drun_count(p) == 0 and p.stats()["device_ops"] == 6
    finally:
        p.close()


@pytest.mark.parametrize("n", [10, 14])
def test_records_qft_and_random_workload_shape(n):
    """The benchmark's circuit shape (QFT of a basis state, then random gates),
    smaller: phase runs from the QFT's controlled-phase chains, swaps, H gates."""
    r, _ = G.random_circuit(n, 300, 77 + n)
    gates = G.concat([G.qft_circuit(n), r])
    check(n, gates, None, qs.PLAN_DEFAULT, 0, 3 + n)


def test_records_long_pass_scale_bound():
    """One pass of 160 unitaries on qubits 0..3 that cannot merge (a controlled X
    between neighbours on the same qubit), so the product of the scalars left out
    reaches the 2^-24 bound and later candidates keep their own."""
    rng = G.SplitMix64(8)
    out = []
    for k in range(160):
        out.append(G.gate_u1(k % 4, G.haar_2x2(rng)))
        out.append(G.gate_cu((k + 1) % 4, k % 4, G.MAT_X))
        out.append(G.gate_u1((k + 2) % 4, G.MAT_H))
    gates = G.concat(out)
    forms = check(8, gates, None, qs.PLAN_DEFAULT, 0, 9)
    assert 0 < forms[0] < 159


@pytest.mark.parametrize("n,tile_bits", [(6, 4 | (2 << 8)), (12, 0), (13, 8 | (1 << 8))])
@pytest.mark.parametrize("dt,flags,tol", [(qs.QS_C64, qs.PLAN_DEFAULT, 1e-5),
                                          (qs.QS_C64, qs.PLAN_NO_MERGE | qs.PLAN_NO_PHASE_RUNS, 1e-5),
                                          (qs.QS_C128, qs.PLAN_ARITH_F64, TOL)])
def test_native_records_reproduce_oracle(n, tile_bits, dt, flags, tol):
    """Native records (complex64 floats, complex128 doubles): products, phase-run
    slots and outside-tile factors in those formats; no scalar-free forms."""
    gates = mixed_circuit(n, 260, 600 + n)
    forms = check(n, gates, np.array([0.7, -1.3]), flags, tile_bits, 43 + n, dt=dt, tol=tol)
    assert not np.any(forms)


def test_records_match_qs_records_layout():
    """RECORD_DTYPE is the 96-byte layout include/qs_records.h states."""
    assert qs.RECORD_DTYPE.itemsize == 96
    n = 8
    p = qs.Plan(fake_state(n), G.concat([G.gate_u1(0, G.MAT_H), G.gate_u1(1, G.MAT_T)]),
                flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_PRP)
    recs, tq, fmt = p.records(0)
    p.close()
    assert fmt == 1 and list(recs["kind"]) == [0, 0] and list(recs["tq"]) == [0, 1] and len(tq) == 8
    assert list(recs["cls"]) == [6, 3]  # balanced real (H), diagonal with q11 = 1 (T)
    assert float(recs["c"][1][12]) + float(recs["c"][1][13]) == pytest.approx(np.cos(np.pi / 4), abs=1e-15)
    for dt, flags, want_fmt in ((qs.QS_C64, 0, 2), (qs.QS_C128, qs.PLAN_ARITH_F64, 3)):
        p = qs.Plan(fake_state(n, dt), G.concat([G.gate_u1(0, G.MAT_H), G.gate_u1(1, G.MAT_T)]),
                    flags=qs.PLAN_DRY_RUN | flags)
        recs, tq, fmt = p.records(0)
        p.close()
        assert fmt == want_fmt and recs.dtype.itemsize == (64 if fmt == 2 else 96)
        assert list(recs["cls"]) == [1, 3] and recs["m"][1][6] == pytest.approx(np.cos(np.pi / 4), rel=1e-7)


def test_record_view_arguments():
    """qs_plan_pass_records: a NULL count or an out-of-range pass is QS_EINVAL,
    a buffer smaller than the pass is QS_EINVAL and left untouched, single-gate
    passes have no records."""
    lib = qs.load()
    n = 12
    gates = G.concat([G.gate_u1(0, G.MAT_H), G.gate_u1(1, G.MAT_T), G.gate_u1(2, G.haar_2x2(G.SplitMix64(4)))])
    p = qs.Plan(fake_state(n), gates, flags=qs.PLAN_DRY_RUN)
    cnt = ctypes.c_int()
    assert lib.qs_plan_pass_records(p._h, 0, None, 0, None, None, None, None) == qs.QS_EINVAL
    assert lib.qs_plan_pass_records(p._h, 5, None, 0, ctypes.byref(cnt), None, None, None) == qs.QS_EINVAL
    assert lib.qs_plan_pass_records(p._h, 0, None, 0, ctypes.byref(cnt), None, None, None) == qs.QS_OK
    assert cnt.value == 3
    buf = np.full(2, 7, dtype=qs.RECORD_DTYPE)
    assert lib.qs_plan_pass_records(p._h, 0, buf.ctypes.data, 2, ctypes.byref(cnt), None, None, None) == qs.QS_EINVAL
    assert np.all(buf["kind"] == 7)
    p.close()
    single = qs.Plan(fake_state(n), G.gate_u1(11, G.haar_2x2(G.SplitMix64(5))), flags=qs.PLAN_DRY_RUN)
    assert single.passes()[0]["kind"] == "single"
    recs, tq, fmt = single.records(0)
    single.close()
    assert len(recs) == 0 and tq == []


def test_random_plans_records_reproduce_oracle():
    """Property test over random circuits, qubit counts, tile shapes, plan flags
    and record formats: the records of every pass, applied on the host,
    reproduce the oracle's state."""
    hyp = pytest.importorskip("hypothesis")
    st_ = hyp.strategies
    flag_sets = [qs.PLAN_DEFAULT, qs.PLAN_NO_PRP, qs.PLAN_NO_MERGE, qs.PLAN_NO_PHASE_RUNS, qs.PLAN_NO_FUSION]
    modes = [(qs.QS_C128, 0, TOL), (qs.QS_C128, qs.PLAN_ARITH_F64, TOL), (qs.QS_C64, 0, 1e-5)]

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(n=st_.integers(2, 10), count=st_.integers(1, 150), seed=st_.integers(0, 10 ** 6),
               b=st_.integers(1, 12), b0=st_.integers(0, 6), flags=st_.sampled_from(flag_sets),
               mode=st_.sampled_from(modes))
    def prop(n, count, seed, b, b0, flags, mode):
        dt, arith, tol = mode
        gates = mixed_circuit(n, count, seed)
        check(n, gates, np.array([0.7, -1.3]), flags | arith, b | (min(b0, b) << 8), seed % 997, dt=dt, tol=tol)

    prop()


def test_random_plans_with_diagonal_runs_reproduce_oracle():
    """Property test over circuits that interleave runs of phase gates (every
    diagonal-run term kind) with other gates, random tile shapes, flags and
    record formats: the records, diagonal runs included, reproduce the oracle."""
    hyp = pytest.importorskip("hypothesis")
    st_ = hyp.strategies
    flag_sets = [qs.PLAN_DEFAULT, qs.PLAN_NO_PHASE_RUNS, qs.PLAN_NO_DIAG_RUNS, qs.PLAN_NO_MERGE]
    modes = [(qs.QS_C128, 0, TOL), (qs.QS_C128, qs.PLAN_ARITH_F64, TOL), (qs.QS_C64, 0, 1e-5)]

    @hyp.settings(max_examples=80, deadline=None, derandomize=True)
    @hyp.given(n=st_.integers(4, 11), runs=st_.integers(1, 8), seed=st_.integers(0, 10 ** 6),
               b=st_.integers(2, 10), b0=st_.integers(0, 4), flags=st_.sampled_from(flag_sets),
               mode=st_.sampled_from(modes))
    def prop(n, runs, seed, b, b0, flags, mode):
        dt, arith, tol = mode
        gates = G.concat([mixed_circuit(n, 20, seed), diag_circuit(n, runs, seed + 1, outside_from=n // 2),
                          mixed_circuit(n, 10, seed + 2)])
        check(n, gates, np.array([0.7, -1.3]), flags | arith, b | (min(b0, b) << 8), seed % 991, dt=dt, tol=tol)

    prop()


def test_dense_passes_reproduce_oracle():
    """complex64 plans with runs of >= 10 gates on qubits 0..5: the dense passes'
    64 x 64 matrices (formed by the planner in FP64) together with the other
    passes' records reproduce the oracle (dense products checked to rounding of
    the float records around them)."""
    from tests.test_planner import _low_run
    for n, seed in ((8, 1), (11, 2), (14, 3)):
        r1, _ = G.random_circuit(n, 40, seed)
        r2, _ = G.random_circuit(n, 40, seed + 10)
        gates = G.concat([_low_run(12, seed), r1, _low_run(30, seed + 1), r2, _low_run(10, seed + 2)])
        st = fake_state(n, qs.QS_C64)
        p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN)
        assert sum(ps["kind"] == "dense" for ps in p.passes()) >= 3
        p.close()
        check(n, gates, None, qs.PLAN_DEFAULT, 0, seed, dt=qs.QS_C64, tol=1e-5)
