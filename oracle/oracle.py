"""Python front end of the CPU FP64 oracle (qs_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import this module; the product path
never does.  It shares no code with the CUDA library: it compiles its own C
file with gcc (``-O2 -ffp-contract=off``) into ``oracle/_build`` and calls it
through ctypes.  States are numpy complex128 arrays, whose memory layout is the
interleaved (re, im) layout the C routines expect.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


_OMP_LIB_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_omp_lib = None


def compile_source(src: str, out: str, parallel: bool = False) -> str:
    """gcc -O2 -ffp-contract=off: separately rounded IEEE double operations.
    parallel=True: the same source with -O3 -fopenmp (its pair loops split over
    the host's cores; the same operations on every pair, so the same bits)."""
    tmp = out + f".tmp{os.getpid()}"
    opt = ["-O3", "-fopenmp"] if parallel else ["-O2"]
    subprocess.check_call(
        ["gcc", "-std=c99", *opt, "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
         src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False, parallel: bool = True) -> str:
    """Compile qs_oracle.c into a shared library (plain gcc, no vector extensions),
    and (parallel=True) its OpenMP build beside it."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            compile_source(_SRC, _LIB_PATH)
        if parallel and (force or not os.path.exists(_OMP_LIB_PATH)
                         or os.path.getmtime(_OMP_LIB_PATH) < os.path.getmtime(_SRC)):
            compile_source(_SRC, _OMP_LIB_PATH, parallel=True)
    return _LIB_PATH


def load_library(path):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build(parallel=False))
    return _lib


def _load_omp():
    global _omp_lib
    if _omp_lib is None:
        build(parallel=True)
        _omp_lib = load_library(_OMP_LIB_PATH)
    return _omp_lib


def threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else every core the process may run on)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.split(",")[0].isdigit():
        return int(env.split(",")[0])
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _declare(lib):
    lib.or_init_basis.argtypes = [_dp, ctypes.c_int, ctypes.c_uint64]
    lib.or_apply_1q.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
    lib.or_apply_ctrl.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.or_apply_swap.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.or_run.argtypes = [_dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int]
    lib.or_run.restype = ctypes.c_int
    lib.or_gate_matrix.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_norm2.argtypes = [_dp, ctypes.c_int]
    lib.or_norm2.restype = ctypes.c_double
    lib.or_marginals.argtypes = [_dp, ctypes.c_int, _dp]
    lib.or_probs.argtypes = [_dp, ctypes.c_int, _dp]
    lib.or_expect.argtypes = [_dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    lib.or_expect.restype = ctypes.c_double
    lib.or_grad.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                            ctypes.c_void_p, ctypes.c_int, _dp, _dp]
    lib.or_grad.restype = ctypes.c_int
    lib.or_qft_basis.argtypes = [_dp, ctypes.c_int, ctypes.c_uint64]
    lib.or_apply_hamiltonian.argtypes = [_dp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _dp]
    lib.or_apply_hamiltonian.restype = ctypes.c_int
    lib.or_dot_re.argtypes = [_dp, _dp, ctypes.c_int]
    lib.or_dot_re.restype = ctypes.c_double
    lib.or_apply_gate.argtypes = [_dp, ctypes.c_int, ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_int]
    lib.or_apply_gate.restype = ctypes.c_int
    lib.or_apply_dense.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _state(psi):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("oracle states are C-contiguous complex128 arrays")
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


def _m8(m):
    m = np.ascontiguousarray(m, dtype=np.float64).reshape(8)
    return m


def basis(n: int, x: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().or_init_basis(_ptr(psi.view(np.float64)), n, x)
    return psi


def apply_1q(psi, k, m8):
    n = _state(psi)
    if not 0 <= k < n:
        raise ValueError("qubit out of range")
    m = _m8(m8)
    _load().or_apply_1q(_ptr(psi.view(np.float64)), n, k, _ptr(m))


def apply_ctrl(psi, c, t, m8):
    n = _state(psi)
    if not (0 <= c < n and 0 <= t < n and c != t):
        raise ValueError("bad control/target")
    m = _m8(m8)
    _load().or_apply_ctrl(_ptr(psi.view(np.float64)), n, c, t, _ptr(m))


def apply_swap(psi, a, b):
    n = _state(psi)
    if not (0 <= a < n and 0 <= b < n and a != b):
        raise ValueError("bad swap qubits")
    _load().or_apply_swap(_ptr(psi.view(np.float64)), n, a, b)


def apply_dense(psi, U, parallel=False):
    """y = U x on every group of 2^q consecutive amplitudes (U: 2^q x 2^q complex,
    acting on qubits 0..q-1), in place."""
    n = _state(psi)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    q = int(U.shape[0]).bit_length() - 1
    if U.shape != (1 << q, 1 << q) or not 1 <= q <= min(n, 10):
        raise ValueError("U must be 2^q x 2^q with 1 <= q <= min(n, 10)")
    (_load_omp() if parallel else _load()).or_apply_dense(_ptr(psi.view(np.float64)), n, q, _ptr(U.view(np.float64)))
    return psi


def run(psi, gates, theta=None, parallel=False):
    """Apply the gate records in order, in place (parallel=True: the OpenMP build,
    bit-identical result on all host cores)."""
    n = _state(psi)
    gates = np.ascontiguousarray(gates)
    th = np.ascontiguousarray(theta if theta is not None else np.zeros(0), dtype=np.float64)
    lib = _load_omp() if parallel else _load()
    rc = lib.or_run(_ptr(psi.view(np.float64)), n, gates.ctypes.data, len(gates),
                    _ptr(th) if th.size else None, int(th.size))
    if rc != 0:
        raise ValueError("invalid gate record")
    return psi


def simulate(n, gates, theta=None, x=0, parallel=False):
    return run(basis(n, x), gates, theta, parallel=parallel)


def qft_basis_state(n, x, parallel=False):
    """The whole state QFT|x> from its closed form (or_qft_basis): amplitude y is
    2^(-n/2) exp(2 pi i (x y mod 2^n) / 2^n), the product reduced exactly in
    64-bit integers (n <= 32)."""
    if not 1 <= n <= 32 or not 0 <= int(x) < (1 << n):
        raise ValueError("need 1 <= n <= 32 and 0 <= x < 2^n")
    psi = np.empty(1 << n, dtype=np.complex128)
    (_load_omp() if parallel else _load()).or_qft_basis(_ptr(psi.view(np.float64)), n, int(x))
    return psi


def gate_matrix(gate, theta=None):
    th = np.ascontiguousarray(theta if theta is not None else np.zeros(1), dtype=np.float64)
    g = np.ascontiguousarray(np.atleast_1d(gate))
    out = np.zeros(8, dtype=np.float64)
    _load().or_gate_matrix(g.ctypes.data, _ptr(th), _ptr(out))
    return out


def norm2(psi):
    n = _state(psi)
    return _load().or_norm2(_ptr(psi.view(np.float64)), n)


def marginals(psi):
    n = _state(psi)
    out = np.zeros(n, dtype=np.float64)
    _load().or_marginals(_ptr(psi.view(np.float64)), n, _ptr(out))
    return out


def probs(psi):
    n = _state(psi)
    out = np.zeros(1 << n, dtype=np.float64)
    _load().or_probs(_ptr(psi.view(np.float64)), n, _ptr(out))
    return out


def expect(psi, terms):
    n = _state(psi)
    terms = np.ascontiguousarray(terms)
    v = _load().or_expect(_ptr(psi.view(np.float64)), n, terms.ctypes.data, len(terms))
    if np.isnan(v):
        raise ValueError("invalid Pauli term")
    return v


def grad(n, gates, theta, terms):
    """(energy, gradient) of <psi(theta)|H|psi(theta)> from the definition of the derivative."""
    gates = np.ascontiguousarray(gates)
    terms = np.ascontiguousarray(terms)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    e = np.zeros(1, dtype=np.float64)
    g = np.zeros(max(1, th.size), dtype=np.float64)
    rc = _load().or_grad(n, gates.ctypes.data, len(gates), _ptr(th), int(th.size),
                         terms.ctypes.data, len(terms), _ptr(e), _ptr(g))
    if rc != 0:
        raise ValueError("invalid gradient input")
    return float(e[0]), g[: th.size].copy()


def grad_sampled(n, gates, theta, terms, params, parallel=False):
    """(energy, {p: dE/dtheta_p}) for the listed parameters only, from the same
    definition as or_grad: dE/dtheta_p = 2 Re <H psi | U_P..U_{j+1} (dU_j/dtheta)
    U_{j-1}..U_1 |0>> for the rotation gate j that carries p.  One forward run
    keeps the prefix state U_{j-1}..U_1 |0> of each listed parameter in turn, so
    a parameter costs only its gate's suffix.  Each listed parameter must belong
    to exactly one rotation gate."""
    gates = np.ascontiguousarray(gates)
    terms = np.ascontiguousarray(terms)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lib = _load_omp() if parallel else _load()
    where = {}
    for j, g in enumerate(gates):
        if int(g["kind"]) in (3, 4, 5):
            where.setdefault(int(g["param"]), []).append(j)
    for p in params:
        if len(where.get(int(p), [])) != 1:
            raise ValueError(f"parameter {p} is not carried by exactly one rotation gate")
    order = sorted({int(p) for p in params}, key=lambda p: where[p][0])

    def apply(psi, j, deriv=0):
        rc = lib.or_apply_gate(_ptr(psi.view(np.float64)), n, gates[j:j + 1].ctypes.data, _ptr(th), int(th.size), deriv)
        if rc != 0:
            raise ValueError("invalid gate record")

    prefix = basis(n, 0)
    done = 0
    partial = {}
    for p in order:
        j = where[p][0]
        for i in range(done, j):
            apply(prefix, i)
        done = j
        d = prefix.copy()
        apply(d, j, deriv=1)
        for i in range(j + 1, len(gates)):
            apply(d, i)
        partial[p] = d
    for i in range(done, len(gates)):
        apply(prefix, i)
    hpsi = np.empty_like(prefix)
    if lib.or_apply_hamiltonian(_ptr(prefix.view(np.float64)), n, terms.ctypes.data, len(terms),
                                _ptr(hpsi.view(np.float64))) != 0:
        raise ValueError("invalid Pauli term")
    energy = lib.or_dot_re(_ptr(prefix.view(np.float64)), _ptr(hpsi.view(np.float64)), n)
    grads = {p: 2.0 * lib.or_dot_re(_ptr(hpsi.view(np.float64)), _ptr(d.view(np.float64)), n)
             for p, d in partial.items()}
    return energy, grads


def qft_basis_amplitudes(n, x, ys):
    """Closed form of the quantum Fourier transform of |x> at indices ys:
    2^(-n/2) exp(2 pi i (x y mod 2^n) / 2^n), the modular product taken in exact
    integer arithmetic before the floating-point exponential."""
    ys = np.asarray(ys, dtype=np.uint64)
    mod = (1 << n) - 1
    ph = np.array([(int(x) * int(y)) & mod for y in ys], dtype=np.float64)
    return np.exp(2j * np.pi * ph / float(1 << n)) * 2.0 ** (-n / 2)
