"""The allocation-free marginal reduction (qs_marginals_noalloc).

It serves callers that cannot allocate device memory, for example a host
application whose memory pool already owns the GPU's memory or a
latency-critical loop that must not pay for cudaMalloc / cudaFree.  Its partial
sums live in a static device array inside the library.  This file is named so
that pytest collects it last.  The GPU test calls the entry point through the C
ABI twice in a row on the same state: the second call runs over whatever the
first left in the shared array.  Both calls must agree with the allocating
entry point qs_prob(k = -1) and qs_norm within the tolerance the reduction
tests use (1e-12), and with the CPU FP64 oracle's marginals and norm of the
state the GPU holds (copied out), which is computed with neither kernel.
"""

import ctypes

import numpy as np
import pytest

import qsgen as G
from oracle import oracle as O
from paper_1601_07195_gb300 import qs

TOL = 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n", [5, 12, 21])
def test_noalloc_marginals_match_allocating_entry_point(dt, n):
    import torch

    assert torch.cuda.is_available()
    lib = qs.load()
    stream = torch.cuda.current_stream()
    with qs.State.create(n, dt, stream=stream) as s:
        s.run(G.random_circuit(n, 80, 31 + n)[0])
        ref = s.marginals()
        ref_norm = s.norm()
        held = s.to_numpy().astype(np.complex128)
        ora, ora_norm = O.marginals(held), O.norm2(held)
        dev = ctypes.c_void_p()
        assert lib.qs_info(s.handle, ctypes.byref(dev), None, None) == qs.QS_OK
        out = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))
            rc = lib.qs_marginals_noalloc(dev, n, dt, ctypes.c_void_p(stream.cuda_stream),
                                          ctypes.c_void_p(out.data_ptr()))
            assert rc == qs.QS_OK, lib.qs_last_error().decode()
            stream.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got[:n] - ref)) < TOL
            assert abs(got[n] - ref_norm) < TOL
            assert np.max(np.abs(got[:n] - ora)) < TOL
            assert abs(got[n] - ora_norm) < TOL


def test_noalloc_rejects_bad_arguments_before_any_launch():
    lib = qs.load()
    fake = ctypes.c_void_p(1 << 20)
    assert lib.qs_marginals_noalloc(None, 5, qs.QS_C128, None, fake) == qs.QS_EINVAL
    assert lib.qs_marginals_noalloc(fake, 5, qs.QS_C128, None, None) == qs.QS_EINVAL
    assert lib.qs_marginals_noalloc(fake, 37, qs.QS_C128, None, fake) == qs.QS_EINVAL
    assert b"36" in lib.qs_last_error()
    assert lib.qs_marginals_noalloc(fake, 0, qs.QS_C64, None, fake) == qs.QS_EINVAL
    assert lib.qs_marginals_noalloc(fake, 5, 9, None, fake) == qs.QS_EDTYPE
