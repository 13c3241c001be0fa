"""PyTorch plumbing on the GPU: the autograd Function over the adjoint sweep,
and states that live in torch tensors on non-default streams, both checked
against the CPU FP64 oracle."""

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_qs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1601_07195_gb300 import qs
    qs.load()
    return torch, qs


def _instances():
    out = []
    for i, n in enumerate((3, 6, 11, 14, 14)):  # persistent small-instance kernel and a grouped tile tier
        g, p = G.ansatz(n, 2)
        obs = G.z_zz_observable(n, 60 + i) if i % 2 else G.ising_observable(n, 60 + i)
        out.append({"n": n, "gates": g, "theta": G.angles(p, 70 + i), "terms": obs})
    return out


@pytest.mark.parametrize("dt", [1, 0])
def test_autograd_function_matches_oracle_gradients(torch_qs, dt):
    """loss = sum_i w_i E_i(theta); torch.autograd.grad gives w_i dE_i/dtheta for
    every angle of instance i.  Bounds: the gradient-parity bounds of the batched
    adjoint tests (complex128 1e-12, complex64 1e-4 per unit weight)."""
    torch, qs = torch_qs
    from paper_1601_07195_gb300 import autograd as QA
    insts = _instances()
    batch = QA.make_batch(insts, dt)
    for dev in ("cpu", "cuda"):
        theta = torch.tensor(np.concatenate([x["theta"] for x in insts]), dtype=torch.float64, device=dev,
                             requires_grad=True)
        w = torch.tensor([1.0, -2.0, 0.5, 3.0, 0.25], dtype=torch.float64, device=dev)
        e = QA.energies(batch, theta)
        assert e.device == theta.device and e.shape == (len(insts),)
        (gth,) = torch.autograd.grad((w * e).sum(), theta)
        off = 0
        tol = 1e-12 if dt == 1 else 1e-4
        for i, inst in enumerate(insts):
            e_ref, g_ref = O.grad(inst["n"], inst["gates"], inst["theta"], inst["terms"])
            p = len(inst["theta"])
            assert abs(float(e[i]) - e_ref) < tol
            got = gth[off:off + p].cpu().numpy()
            assert np.max(np.abs(got - float(w[i]) * g_ref)) < tol * max(1.0, abs(float(w[i])))
            off += p
    batch.close()


def test_autograd_gradcheck_complex128(torch_qs):
    """torch.autograd.gradcheck: central differences of the GPU energies (through
    the same Function) agree with its adjoint gradients."""
    torch, qs = torch_qs
    from paper_1601_07195_gb300 import autograd as QA
    g, p = G.ansatz(4, 2)
    inst = [{"n": 4, "gates": g, "theta": G.angles(p, 5), "terms": G.ising_observable(4, 6)},
            {"n": 3, "gates": G.ansatz(3, 1)[0], "theta": G.angles(6, 7), "terms": G.z_zz_observable(3, 8)}]
    batch = QA.make_batch(inst, qs.QS_C128)
    theta = torch.tensor(np.concatenate([x["theta"] for x in inst]), dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda th: QA.energies(batch, th), (theta,), eps=1e-6, atol=1e-7, rtol=1e-6)
    batch.close()


@pytest.mark.parametrize("dt", [1, 0])
def test_state_in_torch_tensor_on_side_streams(torch_qs, dt):
    """A state wrapped in a torch tensor (no copy) runs its gates on a non-default
    stream, then on a second one after set_stream; the tensor itself holds the
    result, which matches the oracle (1e-12 complex128, 1e-5 complex64)."""
    torch, qs = torch_qs
    n = 14
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    tdt = torch.complex128 if dt == 1 else torch.complex64
    t = torch.from_numpy(psi).to(tdt).cuda()
    want = t.cpu().numpy().astype(np.complex128)
    g1, _ = G.random_circuit(n, 150, 41)
    g2, _ = G.random_circuit(n, 150, 42)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    st = qs.State.wrap_tensor(t, stream=s1)
    st.run(g1)
    st.set_stream(s2)
    s2.wait_stream(s1)
    st.run(g2)
    s2.synchronize()
    O.run(want, G.concat([g1, g2]))
    got = t.cpu().numpy()
    assert np.max(np.abs(got - want)) < (1e-12 if dt == 1 else 1e-5)
    assert abs(st.norm() - O.norm2(want)) < (1e-12 if dt == 1 else 1e-5)
    st.close()


def test_wrap_rejects_host_memory(torch_qs):
    torch, qs = torch_qs
    host = torch.zeros(1 << 6, dtype=torch.complex128)
    import ctypes
    h = ctypes.c_void_p()
    assert qs.load().qs_wrap(ctypes.c_void_p(host.data_ptr()), 6, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_EINVAL


def test_host_buffer_round_trip(torch_qs):
    """qs_host_alloc memory (huge pages, page-locked) as the source and target of
    state copies: a state copied in, run, and copied out matches the oracle."""
    torch, qs = torch_qs
    n = 16
    rng = np.random.default_rng(9)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    gates, _ = G.random_circuit(n, 120, 77)
    buf = qs.HostBuffer(1 << n, np.complex128)
    buf.array[:] = psi
    with qs.State.create(n, qs.QS_C128) as s:
        s.copy_in_ptr(buf.ptr, 1 << n)
        s.run(gates)
        buf.array[:] = 0
        import ctypes
        assert qs.load().qs_copy_out(s.handle, 0, 1 << n, ctypes.c_void_p(buf.ptr)) == qs.QS_OK
    want = O.run(psi.copy(), gates)
    assert np.max(np.abs(buf.array - want)) < 1e-12
    buf.close()
