"""GPU parity at the sizes of the benchmarked workloads, against the OpenMP build
of the CPU FP64 oracle (the same source as the serial build, bit-identical
states, run on every host core).

- n = 30, the timed step of the benchmark: QFT of a random basis state followed
  by the 1000-gate random circuit, through the same planned launch sequence the
  benchmark times (default flags and tile shape).  All 2^30 amplitudes are
  compared with the oracle state, which starts from the closed form of QFT|x>
  (pinned against the oracle's simulation of the QFT circuit) and then applies
  the 1000 random gates.
- Batched adjoint gradients at the variational workload's sizes (n = 16, 19,
  22; L = 8; two instances of one structure per size, so each size runs as a
  grouped tile tier with two members), and the n = 28 Ising workload (L = 20,
  1120 angles): energies and a sample of gradient entries against the oracle's
  definition of the derivative, every entry of complex64 against complex128.

Bounds: 1e-12 (complex128) and 1e-5 (complex64) max-abs for amplitudes,
energies and gradients.
"""

import json
import os

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = {1: 1e-12, 0: 1e-5}


def _log(err):
    path = os.environ.get("QS_ERRLOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0],
                                 "err": float(err)}) + "\n")
    return err


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1601_07195_gb300 import qs as _qs
    _qs.load()
    return _qs


@pytest.fixture(scope="module")
def n30_reference():
    """Oracle state of the n = 30 benchmark step (16 GiB on the host)."""
    n = 30
    x = G.random_basis(n, G.SEEDS["qft30"])
    r, _ = G.random_circuit(n, 1000, G.SEEDS["qft30"])
    psi = O.qft_basis_state(n, x, parallel=True)
    O.run(psi, r, parallel=True)
    return n, x, G.concat([G.qft_circuit(n), r]), psi


@pytest.mark.parametrize("dt,dense", [(1, False), (0, True), (0, False)])
def test_benchmark_step_n30_every_amplitude(qs, n30_reference, dt, dense):
    """complex64 plans run the QFT's last 21 gates (all on qubits 0..5) as one
    tensor-core pass unless planned with QS_PLAN_NO_DENSE (dense = False)."""
    n, x, gates, want = n30_reference
    chunk = 1 << 24
    err = 0.0
    with qs.State.create(n, dt) as s:
        s.init_basis(x)
        p = s.plan(gates, flags=qs.PLAN_DEFAULT if dense else qs.PLAN_NO_DENSE)
        kinds = [ps["kind"] for ps in p.passes()]
        assert kinds.count("dense") == (1 if dense else 0) and "single" not in kinds
        p.execute()
        for off in range(0, 1 << n, chunk):
            got = s.to_numpy(off, chunk)
            err = max(err, float(np.max(np.abs(got - want[off:off + chunk]))))
        p.close()
    assert _log(err) < TOL[dt]


def _variational(n, layers, seeds, ising=False):
    g, p = G.ansatz(n, layers)
    out = []
    for s in seeds:
        obs = G.ising_observable(n, s + 1) if ising else G.z_zz_observable(n, s + 1)
        out.append({"n": n, "gates": g, "theta": G.angles(p, s), "terms": obs})
    return out


def _sample(p, layers, n):
    """Parameters from the first, a middle and the last layer (2n per layer)."""
    per = 2 * n
    pick = [0, per - 1, per * (layers // 2) + n // 2, per * (layers - 1), p - 1]
    return sorted(set(pick))


def test_batched_gradients_at_workload_sizes(qs):
    insts = []
    for n in (16, 19, 22):
        insts += _variational(n, 8, (500 + n, 600 + n))
    res = {}
    for dt in (1, 0):
        b = qs.Batch(insts, dt)
        st = b.stats()
        assert st["small"] == 0 and st["groups"] == 3  # one grouped tier of two members per size
        res[dt] = b.execute()
        b.close()
    for i, inst in enumerate(insts):
        n, p = inst["n"], len(inst["theta"])
        e_ref, g_ref = O.grad_sampled(n, inst["gates"], inst["theta"], inst["terms"], _sample(p, 8, n), parallel=True)
        for dt in (1, 0):
            e, gr = res[dt]
            assert _log(abs(e[i] - e_ref)) < TOL[dt], (n, dt)
            assert _log(max(abs(gr[i][k] - v) for k, v in g_ref.items())) < TOL[dt], (n, dt)
        assert _log(float(np.max(np.abs(res[0][1][i] - res[1][1][i])))) < TOL[0]


def test_adjoint_n28_ising(qs):
    """The n = 28 gradient workload (L = 20, ZZ + X Ising), complex64 with FP64
    reductions and complex128."""
    n, layers = 28, 20
    inst = _variational(n, layers, (G.SEEDS["adjoint28"],), ising=True)
    p = len(inst[0]["theta"])
    out = {}
    for dt in (0, 1):
        b = qs.Batch(inst, dt)
        out[dt] = b.execute()
        b.close()
    pick = [p - 1, p - n - 1, p - 2 * n, p - 3 * n + 5]  # the last layers (each angle costs its gate's suffix)
    e_ref, g_ref = O.grad_sampled(n, inst[0]["gates"], inst[0]["theta"], inst[0]["terms"], pick, parallel=True)
    for dt in (0, 1):
        e, gr = out[dt]
        assert _log(abs(e[0] - e_ref)) < TOL[dt], dt
        assert _log(max(abs(gr[0][k] - v) for k, v in g_ref.items())) < TOL[dt], dt
    assert _log(float(np.max(np.abs(out[0][1][0] - out[1][1][0])))) < TOL[0]


@pytest.mark.parametrize("n,dt", [(33, 1), (34, 0)])
def test_largest_states_circuit_then_inverse(qs, n, dt):
    """n = 33 complex128 and n = 34 complex64 (128 GiB each), the 500-gate circuit
    family of the largest workload, planned and run, then its inverse: the state
    returns to the basis state |x>.  Checked on 4099 sampled amplitudes (including
    |x> itself and the ends) and the FP64 norm; no oracle state fits these sizes."""
    import torch
    free = torch.cuda.mem_get_info()[0]
    if free < (8 << n) * (2 if dt == 1 else 1) + (4 << 30):
        pytest.skip("not enough free device memory for this state")
    r, _ = G.random_circuit(n, 500, G.SEEDS["random33"])
    x = G.random_basis(n, 33)
    rng = np.random.default_rng(n)
    ys = np.unique(np.concatenate([rng.integers(0, 1 << n, 4096), [0, x, (1 << n) - 1]]))
    with qs.State.create(n, dt) as s:
        s.init_basis(x)
        for gates in (r, G.inverse_circuit(r)):
            p = s.plan(gates)
            p.execute()
            p.close()
        vals = np.array([s.to_numpy(int(y), 1)[0] for y in ys])
        nrm = s.norm()
    want = (ys == x).astype(np.complex128)
    assert _log(float(np.max(np.abs(vals - want)))) < TOL[dt]
    assert _log(abs(nrm - 1.0)) < (1e-11 if dt == 1 else 1e-4)
