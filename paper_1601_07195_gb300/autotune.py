"""Tile-shape autotuner front end: runs the library's qs_autotune on a
synthetic circuit and keeps the winners in a JSON cache keyed by GPU name,
dtype and qubit count, which `apply_cache` loads into the planner
(qs_tune_set) in later processes.

The measurement itself is native (qs_autotune times every tile shape that
fits shared memory with CUDA events); this module only chooses the sample
circuit and persists the result.
"""

import ctypes
import json
import os

import numpy as np

from . import qs

DEFAULT_CACHE = os.environ.get("QS_AUTOTUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "qs_autotune.json"))

_lib_extra = {
    "qs_tune_set": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "qs_tune_get": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "qs_autotune": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                    ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                    ctypes.POINTER(ctypes.c_float)],
}


def _lib():
    lib = qs.load()
    for name, args in _lib_extra.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib


def device_key():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def tune_set(dtype, n, tile_bits, run_bits):
    qs._check(_lib().qs_tune_set(dtype, n, tile_bits, run_bits))


def tune_get(dtype, n):
    b, b0 = ctypes.c_int(), ctypes.c_int()
    qs._check(_lib().qs_tune_get(dtype, n, ctypes.byref(b), ctypes.byref(b0)))
    return b.value, b0.value


def tune(n, dtype, gates=None, reps=2, cache=DEFAULT_CACHE, stream=None):
    """Autotune the tile shape for (dtype, n) on `gates` (default: a 300-gate
    random circuit with the random-circuit mix) and store it in the cache."""
    import qsgen as G
    if gates is None:
        gates, _ = G.random_circuit(n, 300, 77)
    g = np.ascontiguousarray(gates, dtype=qs.GATE_DTYPE)
    b, b0, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    with qs.State.create(n, dtype, stream=stream) as st:
        qs._check(_lib().qs_autotune(st.handle, g.ctypes.data, len(g), None, 0, reps, ctypes.byref(b),
                                     ctypes.byref(b0), ctypes.byref(ms)))
    entry = {"tile_bits": b.value, "run_bits": b0.value, "ms": ms.value, "gates": len(g)}
    if cache:
        data = load_cache(cache)
        data.setdefault(device_key(), {})[f"{'c128' if dtype == qs.QS_C128 else 'c64'}/{n}"] = entry
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return entry


def load_cache(cache=DEFAULT_CACHE):
    try:
        with open(cache) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def apply_cache(cache=DEFAULT_CACHE, device=None):
    """Load this GPU's tuned shapes into the planner; returns how many were applied."""
    data = load_cache(cache)
    dev = device if device is not None else device_key()
    count = 0
    for key, e in data.get(dev, {}).items():
        dt, n = key.split("/")
        tune_set(qs.QS_C128 if dt == "c128" else qs.QS_C64, int(n), int(e["tile_bits"]), int(e["run_bits"]))
        count += 1
    return count
