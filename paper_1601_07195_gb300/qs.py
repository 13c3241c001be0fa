"""Thin ctypes binding of the C ABI in include/qs.h (argument marshalling only).

Every computation runs in libqs.so on the GPU.  There is no CPU fallback: if
the library is missing or fails to load, importing a function raises.
PyTorch supplies device memory and streams (``State.wrap_tensor``); states
created by ``State.create`` own their device memory.
"""

import ctypes
import os

import numpy as np

from . import build as _build

QS_C64, QS_C128 = 0, 1
QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EDTYPE = range(6)
QS_G_U1, QS_G_CU, QS_G_SWAP, QS_G_RX, QS_G_RY, QS_G_RZ = range(6)
QS_P_Z, QS_P_ZZ, QS_P_X = range(3)
PLAN_DEFAULT, PLAN_NO_FUSION, PLAN_GRAPH, PLAN_ARITH_F64, PLAN_DRY_RUN, PLAN_NO_MERGE = 0, 1, 2, 4, 8, 16
PLAN_NO_PHASE_RUNS = 32
PLAN_NO_PRP = 64
PLAN_NO_DENSE = 128
PLAN_NO_DIAG_RUNS = 256
LANES_OFF, LANES_AUTO, LANES_ON = 0, 1, 2  # qs_set_lanes

# one tile-pass record (include/qs_records.h): double-float (complex128 plans),
# float (complex64) and double (complex128 with PLAN_ARITH_F64) formats
_REC_HEAD = [("kind", "<i4"), ("cls", "<i4"), ("tb", "<i4"), ("tq", "<i4"), ("cb", "<i4"), ("cq", "<i4"),
             ("pad", "<i4", (2,))]
RECORD_DTYPE = np.dtype(_REC_HEAD + [("c", "<f4", (16,))])
RECORD_DTYPES = {1: RECORD_DTYPE, 2: np.dtype(_REC_HEAD + [("m", "<f4", (8,))]),
                 3: np.dtype(_REC_HEAD + [("m", "<f8", (8,))])}

_STATUS = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ENOMEM", 3: "QS_ECUDA", 4: "QS_ETIMEOUT", 5: "QS_EDTYPE"}

GATE_DTYPE = np.dtype([("kind", "<i4"), ("t", "<i4"), ("c", "<i4"), ("param", "<i4"), ("m", "<f8", (8,))], align=True)
TERM_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("pad", "<i4"), ("coef", "<f8")], align=True)


class QSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_gates", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("n_params", ctypes.c_int32), ("theta", ctypes.c_void_p),
                ("n_terms", ctypes.c_int32), ("terms", ctypes.c_void_p)]


_lib = None
_vp, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "qs_create": [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)],
    "qs_wrap": [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)],
    "qs_destroy": [_vp],
    "qs_set_stream": [_vp, _vp],
    "qs_set_arith": [_vp, ctypes.c_int],
    "qs_set_lanes": [_vp, ctypes.c_int],
    "qs_info": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "qs_init_basis": [_vp, ctypes.c_uint64],
    "qs_copy_out": [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp],
    "qs_copy_in": [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp],
    "qs_host_alloc": [ctypes.c_size_t, ctypes.POINTER(_vp)],
    "qs_host_free": [_vp],
    "qs_apply_1q": [_vp, ctypes.c_int, _dp],
    "qs_apply_ctrl": [_vp, ctypes.c_int, ctypes.c_int, _dp],
    "qs_apply_swap": [_vp, ctypes.c_int, ctypes.c_int],
    "qs_apply_dense": [_vp, ctypes.c_int, _dp],
    "qs_plan_create": [_vp, _vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "qs_plan_execute": [_vp],
    "qs_plan_stats": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                     ctypes.POINTER(ctypes.c_uint64)],
    "qs_plan_pass_gates": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass_dense": [_vp, ctypes.c_int, _dp],
    "qs_plan_device_ops": [_vp, ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass_op_counts": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass_balanced": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass_prp": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "qs_plan_pass_records": [_vp, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "qs_plan_set_timing": [_vp, ctypes.c_int],
    "qs_plan_pass_times": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)],
    "qs_plan_destroy": [_vp],
    "qs_run": [_vp, _vp, ctypes.c_int, _dp, ctypes.c_int],
    "qs_norm": [_vp, _dp],
    "qs_prob": [_vp, ctypes.c_int, _dp],
    "qs_probs": [_vp, _dp],
    "qs_expect": [_vp, _vp, ctypes.c_int, _dp],
    "qs_grad": [_vp, ctypes.c_int, ctypes.c_int, _vp, _dp, _dp],
    "qs_marginals_noalloc": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "qs_batch_create": [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(_vp)],
    "qs_batch_execute": [_vp, _dp, _dp, _dp],
    "qs_batch_stats": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "qs_batch_destroy": [_vp],
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqs.so (building it first when the toolkit is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libqs.so not found at {path}; run paper_1601_07195_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.qs_last_error.restype = ctypes.c_char_p
    lib.qs_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != QS_OK:
        raise QSError(status, load().qs_last_error().decode())


def _m8(m):
    a = np.ascontiguousarray(m, dtype=np.float64).reshape(8)
    return a, a.ctypes.data_as(_dp)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


class HostBuffer:
    """Page-locked host memory from qs_host_alloc (huge pages, registered):
    ``array`` is a numpy view of ``count`` elements of ``dtype``."""

    def __init__(self, count, dtype=np.complex128):
        dtype = np.dtype(dtype)
        p = _vp()
        _check(load().qs_host_alloc(count * dtype.itemsize, ctypes.byref(p)))
        self._p = p
        self.array = np.ctypeslib.as_array((ctypes.c_char * (count * dtype.itemsize)).from_address(p.value)
                                           ).view(dtype)

    @property
    def ptr(self):
        return self._p.value

    def huge_page_fraction(self):
        """Share of the buffer backed by transparent huge pages (Linux /proc/self/smaps;
        None where that is not readable)."""
        lo, size = self._p.value, self.array.nbytes
        try:
            with open("/proc/self/smaps") as fh:
                inside, total = False, 0
                for line in fh:
                    head = line.split()[0]
                    if "-" in head and not head.endswith(":"):
                        a, b = (int(v, 16) for v in head.split("-"))
                        inside = a < lo + size and b > lo
                    elif inside and head == "AnonHugePages:":
                        total += int(line.split()[1]) * 1024
            return min(1.0, total / size)
        except (OSError, ValueError):
            return None

    def close(self):
        if self._p is not None and self._p.value:
            self.array = None
            _check(load().qs_host_free(self._p))
        self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """A 2^n-amplitude state on the GPU, handled through the C ABI."""

    def __init__(self, handle, n, dtype, keepalive=None):
        self._h = ctypes.c_void_p(handle)
        self.n = n
        self.dtype = dtype
        self._keepalive = keepalive

    @classmethod
    def create(cls, n, dtype=QS_C128, stream=None):
        h = _vp()
        _check(load().qs_create(n, dtype, _stream_handle(stream), ctypes.byref(h)))
        return cls(h.value, n, dtype)

    @classmethod
    def wrap_tensor(cls, tensor, stream=None):
        """Wrap a CUDA tensor of dtype complex128/complex64 and 2^n elements (no copy)."""
        import torch
        if not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("need a contiguous CUDA tensor")
        dt = {torch.complex128: QS_C128, torch.complex64: QS_C64}[tensor.dtype]
        n = tensor.numel().bit_length() - 1
        if tensor.numel() != 1 << n:
            raise ValueError("tensor length must be a power of two")
        if stream is None:
            stream = torch.cuda.current_stream(tensor.device)
        h = _vp()
        with torch.cuda.device(tensor.device):  # the state belongs to the tensor's device
            _check(load().qs_wrap(tensor.data_ptr(), n, dt, _stream_handle(stream), ctypes.byref(h)))
        return cls(h.value, n, dt, keepalive=tensor)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            load().qs_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- data movement
    def init_basis(self, x=0):
        _check(load().qs_init_basis(self._h, x))

    @property
    def np_dtype(self):
        return np.complex128 if self.dtype == QS_C128 else np.complex64

    def to_numpy(self, off=0, cnt=None):
        cnt = (1 << self.n) - off if cnt is None else cnt
        out = np.empty(cnt, dtype=self.np_dtype)
        _check(load().qs_copy_out(self._h, off, cnt, out.ctypes.data))
        return out

    def from_numpy(self, arr, off=0):
        a = np.ascontiguousarray(arr, dtype=self.np_dtype)
        _check(load().qs_copy_in(self._h, off, a.size, a.ctypes.data))

    def copy_in_ptr(self, host_ptr, cnt, off=0):
        """Copy cnt amplitudes from a host address (ideally pinned) into the state."""
        _check(load().qs_copy_in(self._h, off, cnt, ctypes.c_void_p(host_ptr)))

    def set_stream(self, stream):
        _check(load().qs_set_stream(self._h, _stream_handle(stream)))

    def set_arith(self, native_f64):
        """complex128 single-gate calls: native FP64 (True) or double-float (False, default)."""
        _check(load().qs_set_arith(self._h, 1 if native_f64 else 0))

    def set_lanes(self, mode):
        """Single-gate calls on targets 0..4: LANES_AUTO (default, the measured choice),
        LANES_OFF (pair kernel) or LANES_ON (lane exchange by warp shuffles)."""
        _check(load().qs_set_lanes(self._h, int(mode)))

    # ---- gates
    def apply_1q(self, k, m8):
        a, p = _m8(m8)
        _check(load().qs_apply_1q(self._h, k, p))

    def apply_ctrl(self, c, t, m8):
        a, p = _m8(m8)
        _check(load().qs_apply_ctrl(self._h, c, t, p))

    def apply_swap(self, a, b):
        _check(load().qs_apply_swap(self._h, a, b))

    def apply_dense(self, U):
        """Dense 2^q x 2^q complex matrix on qubits 0..q-1 (complex64 states, tensor cores)."""
        u = np.ascontiguousarray(U, dtype=np.complex128)
        q = int(u.shape[0]).bit_length() - 1
        if u.ndim != 2 or u.shape != (1 << q, 1 << q):
            raise ValueError("U must be a 2^q x 2^q matrix")
        _check(load().qs_apply_dense(self._h, q, u.view(np.float64).ctypes.data_as(_dp)))

    def run(self, gates, theta=None):
        g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
        th = np.ascontiguousarray(theta if theta is not None else np.zeros(0), dtype=np.float64)
        _check(load().qs_run(self._h, g.ctypes.data, len(g), th.ctypes.data_as(_dp) if th.size else None, th.size))

    def plan(self, gates, theta=None, flags=PLAN_DEFAULT, tile_bits=0):
        return Plan(self, gates, theta, flags, tile_bits)

    # ---- reductions
    def norm(self):
        out = ctypes.c_double()
        _check(load().qs_norm(self._h, ctypes.byref(out)))
        return out.value

    def prob(self, k):
        out = ctypes.c_double()
        _check(load().qs_prob(self._h, k, ctypes.byref(out)))
        return out.value

    def marginals(self):
        out = np.zeros(self.n, dtype=np.float64)
        _check(load().qs_prob(self._h, -1, out.ctypes.data_as(_dp)))
        return out

    def marginals_and_norm(self):
        """(the n marginals, sum_i |alpha_i|^2) from one read of the state."""
        out = np.zeros(self.n + 1, dtype=np.float64)
        _check(load().qs_prob(self._h, -2, out.ctypes.data_as(_dp)))
        return out[:self.n], float(out[self.n])

    def probs(self):
        out = np.empty(1 << self.n, dtype=np.float64)
        _check(load().qs_probs(self._h, out.ctypes.data_as(_dp)))
        return out

    def expect(self, terms):
        t = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        out = ctypes.c_double()
        _check(load().qs_expect(self._h, t.ctypes.data, len(t), ctypes.byref(out)))
        return out.value


class Plan:
    """A planned circuit (fused tile passes + single-gate passes) bound to a state."""

    def __init__(self, state, gates, theta=None, flags=PLAN_DEFAULT, tile_bits=0):
        g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
        th = np.ascontiguousarray(theta if theta is not None else np.zeros(0), dtype=np.float64)
        h = _vp()
        _check(load().qs_plan_create(state.handle, g.ctypes.data, len(g), th.ctypes.data_as(_dp) if th.size else None,
                                     th.size, flags, tile_bits, ctypes.byref(h)))
        self._h = h
        self.state = state
        self.n_gates = len(g)

    def execute(self):
        _check(load().qs_plan_execute(self._h))

    def stats(self):
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().qs_plan_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        _check(load().qs_plan_device_ops(self._h, ctypes.byref(d)))
        return {"passes": a.value, "tile_passes": b.value, "launches": c.value, "device_ops": d.value}

    def passes(self):
        out = []
        for i in range(self.stats()["passes"]):
            k, ng, mask = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint64()
            _check(load().qs_plan_pass(self._h, i, ctypes.byref(k), ctypes.byref(ng), ctypes.byref(mask)))
            pos = (ctypes.c_int * max(1, ng.value))()
            _check(load().qs_plan_pass_gates(self._h, i, pos))
            out.append({"kind": {0: "single", 1: "tile", 2: "dense"}[k.value], "n_gates": ng.value, "mask": mask.value,
                        "gates": list(pos[:ng.value])})
        return out

    def dense_matrix(self, i):
        """64 x 64 complex matrix of dense pass i (kind "dense")."""
        out = np.zeros(2 * 64 * 64, dtype=np.float64)
        _check(load().qs_plan_pass_dense(self._h, i, out.ctypes.data_as(_dp)))
        return out.view(np.complex128).reshape(64, 64)

    def set_timing(self, records):
        _check(load().qs_plan_set_timing(self._h, records))

    def pass_times(self, record=0):
        n = self.stats()["passes"]
        out = (ctypes.c_float * max(1, n))()
        _check(load().qs_plan_pass_times(self._h, record, out))
        return np.array(out[:n], dtype=np.float64)

    def op_counts(self, i):
        """3x6 array: ops of pass i by (single-qubit, controlled, swap) x gate class; a fused run of
        phase gates around one qubit counts as one single-qubit diagonal op, a diagonal run as two."""
        buf = (ctypes.c_int * 18)()
        _check(load().qs_plan_pass_op_counts(self._h, i, buf))
        return np.array(buf[:], dtype=np.int64).reshape(3, 6)

    def balanced(self, i):
        """(single-qubit, controlled) real updates of pass i applied in balanced form
        (complex128 double-float plans; see qs_plan_pass_balanced)."""
        buf = (ctypes.c_int * 2)()
        _check(load().qs_plan_pass_balanced(self._h, i, buf))
        return int(buf[0]), int(buf[1])

    def scalar_free(self, i):
        """(general, real, general without the trailing phase) single-qubit updates of
        pass i applied with a scalar left out: phase-shear-phase form, balanced real
        without q11, and of the first those whose trailing phase a later update took
        (complex128 double-float plans; see QS_PLAN_NO_PRP and qs_plan_pass_prp)."""
        buf = (ctypes.c_int * 3)()
        _check(load().qs_plan_pass_prp(self._h, i, buf))
        return int(buf[0]), int(buf[1]), int(buf[2])

    def records(self, i):
        """(records, tile qubits, format) of pass i as its tile kernel reads them
        (RECORD_DTYPES[format], layouts in include/qs_records.h)."""
        n, b, fmt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        tq = (ctypes.c_int * 14)()
        _check(load().qs_plan_pass_records(self._h, i, None, 0, ctypes.byref(n), tq, ctypes.byref(b),
                                           ctypes.byref(fmt)))
        out = np.zeros(n.value, dtype=RECORD_DTYPES[fmt.value])
        if n.value:
            _check(load().qs_plan_pass_records(self._h, i, out.ctypes.data, n.value, ctypes.byref(n), None, None,
                                               None))
        return out, list(tq[:b.value]), fmt.value

    def prp(self, i):
        """General single-qubit updates of pass i applied in phase-shear-phase form."""
        return self.scalar_free(i)[0]

    def close(self):
        """Free the plan (raises QSError(QS_ETIMEOUT) if a dense pass's bounded wait gave up)."""
        h, self._h = self._h, None
        if h is not None and h.value:
            _check(load().qs_plan_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _instance_array(instances):
    keep = []
    arr = (Instance * len(instances))()
    for i, inst in enumerate(instances):
        g = np.ascontiguousarray(inst["gates"], dtype=GATE_DTYPE)
        th = np.ascontiguousarray(inst["theta"], dtype=np.float64)
        tm = np.ascontiguousarray(inst["terms"], dtype=TERM_DTYPE)
        keep += [g, th, tm]
        arr[i] = Instance(inst["n"], len(g), g.ctypes.data, th.size, th.ctypes.data, len(tm), tm.ctypes.data)
    return arr, keep


class Batch:
    """A planned batch of variational instances (qs_batch_*): energies and
    adjoint gradients, replayed as one CUDA graph with new angles."""

    def __init__(self, instances, dtype=QS_C128, stream=None, graph=True):
        arr, keep = _instance_array(instances)
        h = _vp()
        _check(load().qs_batch_create(ctypes.cast(arr, _vp), len(instances), dtype, _stream_handle(stream),
                                      0 if graph else 1, ctypes.byref(h)))
        self._h = h
        self.sizes = [len(inst["theta"]) for inst in instances]

    def execute(self, thetas=None):
        lib = load()
        th = None
        if thetas is not None:
            th = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64) for t in thetas]))
            if th.size != sum(self.sizes):
                raise ValueError("angle count does not match the batch")
        energies = np.zeros(len(self.sizes), dtype=np.float64)
        grads = np.zeros(max(1, sum(self.sizes)), dtype=np.float64)
        _check(lib.qs_batch_execute(self._h, th.ctypes.data_as(_dp) if th is not None else None,
                                    energies.ctypes.data_as(_dp), grads.ctypes.data_as(_dp)))
        out, off = [], 0
        for p in self.sizes:
            out.append(grads[off:off + p].copy())
            off += p
        return energies, out

    def stats(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().qs_batch_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"small": a.value, "groups": b.value, "launches": c.value}

    def close(self):
        if self._h is not None and self._h.value:
            load().qs_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grad(instances, dtype=QS_C128, stream=None):
    """Energies and adjoint gradients of a batch of instances (dicts n, gates, theta, terms)."""
    lib = load()
    keep = []
    arr = (Instance * len(instances))()
    total = 0
    for i, inst in enumerate(instances):
        g = np.ascontiguousarray(inst["gates"], dtype=GATE_DTYPE)
        th = np.ascontiguousarray(inst["theta"], dtype=np.float64)
        tm = np.ascontiguousarray(inst["terms"], dtype=TERM_DTYPE)
        keep += [g, th, tm]
        arr[i] = Instance(inst["n"], len(g), g.ctypes.data, th.size, th.ctypes.data, len(tm), tm.ctypes.data)
        total += th.size
    energies = np.zeros(len(instances), dtype=np.float64)
    grads = np.zeros(max(1, total), dtype=np.float64)
    _check(lib.qs_grad(ctypes.cast(arr, _vp), len(instances), dtype, _stream_handle(stream),
                       energies.ctypes.data_as(_dp), grads.ctypes.data_as(_dp)))
    out, off = [], 0
    for inst in instances:
        p = len(inst["theta"])
        out.append(grads[off:off + p].copy())
        off += p
    return energies, out
