#!/usr/bin/env python3
"""Benchmark of the state-vector gate engine on one GB300 (replicas on N GPUs).

Workload: n = 30 qubits, complex128 (16 GiB state): the quantum Fourier
transform of a random basis state (30 H + 435 controlled phase + 15 swaps)
followed by a 1000-gate random circuit (H / X / T / Haar 2x2 on random qubits,
CNOT / controlled phase on random pairs), seeds as in qsgen.SEEDS["qft30"].

One step = |x> initialisation, every gate of the circuit through the planned
launch sequence (fused tile passes and single-gate passes), and the FP64
readout of the norm and all 30 marginals (one read pass for both).  The plan is built once before the
timed region (host work, reported as plan_ms).

value = algorithmic bytes of the step / step time, in the paper's convention
(Section 5.3: the memory traffic each gate needs on its own, summed over the
gates, divided by the run time).  Bytes per gate (n qubits, s bytes per
amplitude): 2*2^n*s for a single-qubit gate, 2^n*s for T-like diagonal gates
(only |1> amplitudes change), controlled gates and swaps, 2^(n-1)*s for a
controlled phase; 2^n*s per reduction pass and for the initialisation.

--impl reference times the CPU FP64 oracle (the only other implementation of
this path) on a bounded sample of the same workload.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qsgen as G  # noqa: E402

METRIC = "gate-apply GB/s vs HBM peak at 30q; batched adjoint-gradient circuits/sec"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 2 DFMA (4 flop) per clock x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--no-secondary", action="store_true", help="skip the batched-gradient measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64 comparison step")
    ap.add_argument("--no-dense-leg", action="store_true", help="skip the tensor-core dense-block measurement")
    ap.add_argument("--parts", default="gate1q,ctrl,iqft", help="sweeps: which of gate1q, ctrl, iqft to run")
    ap.add_argument("--no-dense", action="store_true",
                    help="complex64: plan with QS_PLAN_NO_DENSE (no tensor-core passes for runs on qubits 0..5)")
    ap.add_argument("--workload", default="qft30", choices=["qft30", "random33", "adjoint28", "sweeps", "batch512", "dense"],
                    help="qft30: the headline n=30 step; random33: n=33 complex128 / n=34 complex64 500-gate "
                         "circuits and the n=26 error table; adjoint28: n=28 complex64 adjoint vs parameter shift; "
                         "dense: the tensor-core 64x64 block vs the SIMT tile pass on gate runs on qubits 0..5")
    return ap.parse_args()


# ---- workload and its algorithmic cost ------------------------------------------

def workload(n):
    x = G.random_basis(n, G.SEEDS["qft30"])
    r, _ = G.random_circuit(n, 1000, G.SEEDS["qft30"])
    return x, G.concat([G.qft_circuit(n), r])


def gate_class(g):
    m = g["m"]
    if m[0] == 0 and m[1] == 0 and m[6] == 0 and m[7] == 0 and m[2] == 1 and m[3] == 0 and m[4] == 1 and m[5] == 0:
        return "perm"
    if m[2] == 0 and m[3] == 0 and m[4] == 0 and m[5] == 0:
        return "diag1" if (m[0] == 1 and m[1] == 0) else "diag"
    if m[0] == 0 and m[1] == 0 and m[6] == 0 and m[7] == 0:
        return "antidiag"
    if m[1] == 0 and m[3] == 0 and m[5] == 0 and m[7] == 0:
        return "real"
    return "general"


# FP64 flops per amplitude the class's update touches (FMA = 2 flops)
_FLOPS = {"general": 14.0, "real": 6.0, "diag": 6.0, "diag1": 6.0, "antidiag": 6.0, "perm": 0.0}
# FP32 flops per touched amplitude of the double-float update (csrc/df.cuh):
# df_mul = 1 FMUL + 3 FFMA = 7 flops; TwoSum = 6; dot2 = 2 df_mul + TwoSum + 2 adds = 22;
# dot4 = 4 df_mul + 3 TwoSum + 6 adds = 52 (pairs stay unnormalised); a complex output = 2 dots.
_DF_FLOPS = {"general": 104.0, "real": 44.0, "diag": 44.0, "diag1": 44.0, "antidiag": 44.0, "perm": 0.0}
# a balanced real gate (H-like, qs_plan_pass_balanced): per component an exact
# sum (1 FMUL + TwoSum + 1 FFMA + 1 add = 10) and one product (7): 34 per amplitude
_DF_FLOPS_BALANCED = 34.0
# a general single-qubit unitary in phase-shear-phase form (qs_plan_pass_prp): two
# complex products on the |1> amplitude (2 x 22 flops each) and a shear, per
# component one product and one sum (15): 148 per pair, 74 per amplitude
_DF_FLOPS_PRP = 74.0
# a balanced real gate without its scalar (qs_plan_pass_prp counts[1]): per component
# an exact signed sum (10), times +-1 for the second row (1 more): 44 per pair, 22 per amplitude
_DF_FLOPS_BALANCED_FREE = 22.0
# phase-shear-phase without the trailing product by z (qs_plan_pass_prp counts[2]): 148 - 44 per pair
_DF_FLOPS_PRP_NZ = 52.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
FFMA_MEASURED_TFLOPS = 74.2  # a dependent-chain-free FFMA loop on this GPU (152 SMs, 2.07 GHz)
ISSUE_PEAK_PER_S = 152 * 4 * 2.07e9  # 152 SMs x 4 schedulers x 1 warp instruction per clock
HBM_FALLBACK_GBS = 6800.0  # used only when no measured copy bandwidth is available

# Counters of one launch of each tile kernel from an ncu capture of a small case:
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum), warp instructions
# (smsp__inst_executed.sum) and duration (gpu__time_duration.sum), with the
# SHA-256 of the kernel's source files at capture time.  A tile pass reads and
# writes the whole state once, so DRAM bytes scale with 2^n.  When the sources
# no longer hash to `sha`, the kernel has changed since the capture and its
# counters are reported as null.
CSRC = os.path.join(ROOT, "paper_1601_07195_gb300", "csrc")
NCU_COUNTERS = {
    "df": {"kernel": "k_tile_df_p<12>", "sources": ["tile_df.cu", "tile_df_ops.cuh", "df.cuh", "device.cuh"],
           "sha": "02ec315fe702a534", "n": 26, "dram_bytes": 1.075091e9 + 1.013137e9, "warp_inst": 2.48020992e9,
           "ms": 2.662048},
    "c64": {"kernel": "k_tile_p<float, 12>", "sources": ["tile.cu", "tile_ops.cuh", "device.cuh"],
            "sha": "7aeefc8007452f30", "n": 27, "dram_bytes": 1.073797e9 + 1.012957e9, "warp_inst": 1.891237888e9,
            "ms": 1.8576},
    "dense": {"kernel": "k_dense6_tc", "sources": ["dense_tc.cu"],
              "sha": "9a74760c8df754dc", "n": 25, "dram_bytes": 268.584960e6 + 206.582528e6, "warp_inst": 37525171.0,
              "ms": 0.091456},
}


def sources_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_counters(kind):
    """The capture's counters for tile kernel `kind`, or None when none is
    recorded or the kernel's sources changed since it was taken."""
    c = NCU_COUNTERS.get(kind)
    if not c or c["sha"] is None or c["sha"] != sources_sha(c["sources"]):
        return None
    return c


def bf16_peak():
    """(TFLOP/s, source) of the dense bf16 tensor peak: the measured cuBLAS burst, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def gate_cost(g, n, s, table=None):
    """(algorithmic bytes, flops) of one gate on a 2^n state of s-byte amplitudes;
    flops per touched amplitude from `table` (FP64 flops of the update by default)."""
    table = _FLOPS if table is None else table
    N = float(1 << n)
    kind = int(g["kind"])
    if kind == G.G_SWAP:
        return N * s, 0.0
    if kind == G.G_U1:
        c = gate_class(g)
        touched = 0.5 if c == "diag1" else 1.0
        return (2.0 if c != "diag1" else 1.0) * N * s, table[c] * N * touched
    if kind == G.G_CU:
        c = gate_class(g)
        touched = 0.25 if c == "diag1" else 0.5
        return (0.5 if c == "diag1" else 1.0) * N * s, table[c] * N * touched
    raise ValueError("rotation kinds are not part of this workload")


_CLASSES = ["general", "real", "diag", "diag1", "antidiag", "perm"]


def issue_summary(kind):
    """Instruction issue of tile kernel `kind` from its ncu capture (None when the
    capture is missing or stale)."""
    c = ncu_counters(kind)
    if c is None or c["warp_inst"] is None:
        return None
    return {"warp_instructions": c["warp_inst"], "launch_ms": c["ms"],
            "frac_of_issue_peak": c["warp_inst"] / (c["ms"] / 1e3) / ISSUE_PEAK_PER_S,
            "source": f"ncu capture of one n={c['n']} launch of {c['kernel']}; "
                      "issue peak 152 SMs x 4 schedulers x 2.07 GHz"}


def kernel_flops(counts, n, table):
    """Flops of the updates a pass's kernel applies (after fusion), from the plan's
    per-pass op counts (rows: single-qubit, controlled, swap; columns: classes)."""
    N = float(1 << n)
    total = 0.0
    for c, name in enumerate(_CLASSES):
        touched_1q = 0.5 if name == "diag1" else 1.0
        touched_cu = 0.25 if name == "diag1" else 0.5
        total += counts[0][c] * table[name] * N * touched_1q + counts[1][c] * table[name] * N * touched_cu
    return total


# ---- clocks ----------------------------------------------------------------------

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # raw samples go to a temporary file (QS_CLOCK_DIR overrides the directory);
        # the JSON line carries their summary
        self.path = os.path.join(os.environ.get("QS_CLOCK_DIR", tempfile.gettempdir()), f"qs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]) if f[3] not in ("[N/A]", "N/A") else 0.0, f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ---- measurement legs ----------------------------------------------------------------

def _oracle_sample(O, n, gates, s_bytes, target_s, parallel):
    """Gates spread evenly over the circuit, applied to the n-qubit host state by the
    oracle until target_s seconds of work: (GB/s in the paper's convention, gates used, s)."""
    psi = O.basis(n, G.random_basis(n, G.SEEDS["qft30"]))
    idx = np.linspace(0, len(gates) - 1, 256).astype(int)
    done_bytes, elapsed, used = 0.0, 0.0, []
    for j in idx:
        t0 = time.perf_counter()
        O.run(psi, gates[j:j + 1], parallel=parallel)
        elapsed += time.perf_counter() - t0
        done_bytes += gate_cost(gates[j], n, s_bytes)[0]
        used.append(int(j))
        if elapsed > target_s:
            break
    return done_bytes / elapsed / 1e9, used, elapsed


def cpu_baseline(n, gates, s_bytes, target_s=10.0):
    """Time the CPU FP64 oracle, as it stands, on a bounded sample of the workload:
    its OpenMP build on every host core, and its single-threaded build."""
    from oracle import oracle as O
    O.build()
    v, used, el = _oracle_sample(O, n, gates, s_bytes, target_s, parallel=True)
    v1, used1, el1 = _oracle_sample(O, n, gates, s_bytes, target_s, parallel=False)
    return {"value": v, "unit": "GB/s", "cores": O.threads(), "kind": "oracle",
            "sample": f"{len(used)} gates spread over the n={n} workload (circuit positions {used[0]}..{used[-1]}), "
                      f"applied by the oracle's OpenMP build (-O3 -fopenmp, {O.threads()} threads) to a 2^{n} "
                      f"complex128 host state; {el:.1f} s of work",
            "cpu_model": _cpu_model(),
            "single_thread": {"value": v1, "unit": "GB/s", "cores": 1,
                              "sample": f"{len(used1)} gates, single-threaded -O2 build; {el1:.1f} s of work"}}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    """--impl reference: the CPU oracle on the same metric, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    s = 16
    x, gates = workload(n)
    from oracle import oracle as O
    O.build()
    psi = O.basis(n, x)
    idx = np.linspace(0, len(gates) - 1, 8 * (args.steps + args.warmup)).astype(int)
    chunks = np.array_split(idx, args.steps + args.warmup)
    times, bts = [], []
    for i, ch in enumerate(chunks):
        t0 = time.perf_counter()
        for j in ch:
            O.run(psi, gates[j:j + 1], parallel=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            bts.append(sum(gate_cost(gates[j], n, s)[0] for j in ch))
    value = sum(bts) / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"QFT({n}) on a random basis state + 1000-gate random circuit, complex128",
                       "n": n, "gates": len(gates)},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": O.threads(), "kind": "oracle",
                             "sample": f"8 gates per step spread over the n={n} workload, the oracle's OpenMP "
                                       f"build on {O.threads()} host threads", "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def partition_instances(costs, world):
    """Instances to ranks for the batched path: longest first, each to the rank
    with the least cost so far (cost = 2^n x gates, the work of one instance).
    Returns one ascending list of instance indices per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads, parts = [0.0] * world, [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(local, world, dist=None):
    """The final gather of the batched path: every rank's {instance: (energy,
    gradients)} merged on all ranks (the only collective besides timing)."""
    if world == 1 or dist is None:
        return dict(local)
    objs = [None] * world
    dist.all_gather_object(objs, local)
    merged = {}
    for o in objs:
        merged.update(o)
    return merged


def shard_value(count, local_s, world, dist=None):
    """Instances per second of a batch split over `world` ranks: all `count`
    instances over the slowest rank's time.  Returns (value, max seconds)."""
    s = local_s
    if world > 1 and dist is not None:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        s = float(t.item())
    return count / s, s


def secondary_gradients(qs, dtype, torch, world=1, rank=0, dist=None):
    """Batched adjoint gradients of the 512-instance variational workload vs
    per-circuit central finite differences on the same GPU (sampled).  With
    `world` ranks the instances are split by cost and each rank runs its share
    as one batch (no collective until the final gather of the results)."""
    all_insts = G.batch_instances(G.SEEDS["batch512"], count=512)
    mine = partition_instances([float(1 << x["n"]) * len(x["gates"]) for x in all_insts], world)[rank]
    insts = [all_insts[i] for i in mine]
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    batch = qs.Batch(insts, dtype)   # plans, buffers
    batch.execute()                  # first execution captures the CUDA graph
    t_setup = time.perf_counter() - t0
    reps = 3
    # the new angle sets are drawn before the timed region (input generation is not the method)
    new_thetas = [[G.angles(len(all_insts[i]["theta"]), 7000 + 1000 * r + i) for i in mine] for r in range(reps)]
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for r in range(reps):            # new angles each time: matrices re-staged, graph replayed
        energies, grads = batch.execute(new_thetas[r])
    t_local = (time.perf_counter() - t0) / reps
    results = gather_results({i: (float(energies[k]), grads[k]) for k, i in enumerate(mine)}, world, dist)
    value, t_adj = shard_value(len(all_insts), t_local, world, dist)
    if len(results) != len(all_insts):
        raise RuntimeError("batched path: the gather lost instances")
    t0 = time.perf_counter()
    for r in range(reps):            # same angles: graph replay only (no host-side matrix staging)
        batch.execute()
    t_replay = (time.perf_counter() - t0) / reps
    bstats = batch.stats()
    batch.close()
    insts = all_insts
    # finite-difference comparator: 2P+1 planned energy evaluations per instance (complex128
    # central differences, h = 1e-6), one instance of every qubit count in the batch, weighted
    # by how many instances of that count the batch holds
    by_n = {}
    for inst in insts:
        by_n.setdefault(inst["n"], []).append(inst)
    fd_s = {}
    for n, group in (sorted(by_n.items()) if rank == 0 else ()):  # the comparator runs on rank 0 only
        inst = group[0]
        th = inst["theta"]
        with qs.State.create(n, dtype, stream=stream) as st:
            def energy(theta):
                st.init_basis(0)
                st.run(inst["gates"], theta)
                return st.expect(inst["terms"])
            energy(th)
            t0 = time.perf_counter()
            energy(th)
            for p in range(len(th)):
                tp, tm = th.copy(), th.copy()
                tp[p] += 1e-6
                tm[p] -= 1e-6
                energy(tp)
                energy(tm)
            fd_s[n] = time.perf_counter() - t0
    fd_total = sum(fd_s[n] * len(g) for n, g in by_n.items()) if fd_s else float("nan")
    # arithmetic the batch applies, for its bound: forward on psi, then the reverse sweep on
    # phi and lambda, every gate once per state; RY (real) and RZ (diagonal) updates at
    # 44 FP32 flops per amplitude in double-float (complex128) or 6 in FP32 (complex64),
    # CNOTs as moves; the gradient products and lambda = H psi are left out (an underestimate)
    per_amp = 44.0 if dtype == 1 else 6.0
    flops = sum(3 * 2 * inst["n"] * 8 * per_amp * float(1 << inst["n"]) for inst in insts)  # L = 8 layers
    tf = flops / t_adj / 1e12
    return {"metric": "batched adjoint-gradient circuits/sec", "value": value, "unit": "circuits/s",
            "instances": len(insts), "dtype": "c128" if dtype == 1 else "c64", "setup_s": t_setup,
            "ranks": world, "scaling": "strong" if world > 1 else None,
            "s_per_execution_new_angles": t_adj, "s_per_execution_same_angles": t_replay,
            "persistent_small_instances": bstats["small"], "structure_groups": bstats["groups"],
            "launches_per_execution": bstats["launches"],
            "timing": "host wall clock per qs_batch_execute (angle staging + graph replay + results), mean of 3; "
                      "the angle sets are drawn before the timed region",
            "fd_circuits_per_s": len(insts) / fd_total,
            "fd_sample": "one instance per qubit count (n = %d..%d), weighted by the batch's counts" % (min(by_n),
                                                                                                    max(by_n)),
            "fd_s_by_n": {str(k): v for k, v in fd_s.items()},
            "speedup_vs_fd": fd_total / t_adj,
            "roofline": {"bound": "alu", "achieved": tf, "unit": "TFLOP/s",
                         "peak": FFMA_MEASURED_TFLOPS, "frac": tf / FFMA_MEASURED_TFLOPS,
                         "peak_source": "measured FFMA rate of this GPU",
                         "what": "estimate: FP32 flops of the rotation updates on psi, phi and lambda "
                                 "(lower bound on the arithmetic), per second of execution"}}


def dense_leg(qs, torch, n, reps):
    """The tensor-core dense block (k_dense6_tc) on an n-qubit complex64 state: a
    complex64 plan of a 32-gate run on qubits 0..5 is one dense pass; CUDA events
    around each execution on the state's stream, after 3 warm-up executions."""
    hbm, hbm_src = hbm_peak()
    gates, _ = _gate_run_low6(32, 72)
    stream = torch.cuda.Stream()
    with qs.State.create(n, qs.QS_C64, stream=stream) as st:
        st.init_basis(0)
        p = st.plan(gates)
        kinds = [ps["kind"] for ps in p.passes()]
        for _ in range(3):
            p.execute()
        ms = []
        for _ in range(reps):
            m, _ = _timed(p.execute, stream, torch)
            ms.append(m)
        p.close()
    t = statistics.median(ms)
    N = float(1 << n)
    bytes_ = 2 * N * 8
    flops = 6 * 2 * 128 * 128 * (N / 64)
    cnt = ncu_counters("dense")
    return {"kernel": "k_dense6_tc (tcgen05.mma kind::f16, TMEM accumulators)", "workload":
            f"32-gate run on qubits 0..5 of an n={n} complex64 state, planned as {kinds.count('dense')} dense pass",
            "ms": t, "reps": reps,
            "roofline": {"bound": "hbm", "achieved": bytes_ / (t / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_ / (t / 1e3) / 1e9 / hbm, "peak_source": hbm_src,
                         "traffic": cnt["dram_bytes"] * 2.0 ** (n - cnt["n"]) if cnt else None},
            "tensor_tflops": flops / (t / 1e3) / 1e12,
            "tensor_frac_of_bf16_peak": flops / (t / 1e3) / 1e12 / bf16_peak()[0],
            "bf16_peak_source": bf16_peak()[1] + " bf16 GEMM burst (MEASURED_PEAKS.json bf16_tflops)"}


def job_value(local_ms, step_bytes, steps, world, dist=None):
    """Whole-job throughput of `world` independent replicas (no collective on the
    data path): each rank did `steps` steps of `step_bytes`; the job took the
    slowest rank's time.  Returns (GB/s over all ranks, max ms per step)."""
    total_ms = local_ms
    if world > 1 and dist is not None:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return world * step_bytes / (ms_per_step / 1e3) / 1e9, ms_per_step


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1601_07195_gb300 import qs
    qs.load()

    n = args.n
    dtype = qs.QS_C128 if args.dtype == "c128" else qs.QS_C64
    s_bytes = 16 if dtype == qs.QS_C128 else 8
    x, gates = workload(n)
    N = float(1 << n)
    gate_bytes = sum(gate_cost(g, n, s_bytes)[0] for g in gates)
    step_bytes = gate_bytes + 2 * N * s_bytes  # init write + one read for the marginals and the norm

    stream = torch.cuda.Stream()
    state = qs.State.create(n, dtype, stream=stream)
    t0 = time.perf_counter()
    plan_flags = qs.PLAN_NO_DENSE if args.no_dense else qs.PLAN_DEFAULT
    plan = state.plan(gates, flags=plan_flags)
    plan_ms = 1e3 * (time.perf_counter() - t0)
    passes = plan.passes()
    device_ops = plan.stats()["device_ops"]
    hbm, hbm_src = hbm_peak()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(pl, steps, warmup):
        """W untimed and K timed steps of pl (init |x>, the plan, FP64 norm and
        marginals), CUDA events on the state's stream, clocks sampled meanwhile."""
        pl.set_timing(steps)

        def step():
            state.init_basis(x)
            pl.execute()
            marg, nrm = state.marginals_and_norm()  # one FP64 read pass for both
            return nrm, marg

        for _ in range(warmup):
            nrm, _ = step()
        if abs(nrm - 1.0) > (1e-9 if dtype == qs.QS_C128 else 1e-4):  # complex64: FP32 rounding drift
            raise RuntimeError(f"norm drifted: {nrm}")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(steps):
                step()
            ev1.record(stream)
            ev1.synchronize()
        barrier()
        times = np.array([pl.pass_times(r) for r in range(steps)])  # steps x passes, events on the same stream
        return ev0.elapsed_time(ev1), times, clk.summary()

    total_ms, times, clocks = timed_steps(plan, args.steps, args.warmup)
    value, ms_per_step = job_value(total_ms, step_bytes, args.steps, world, dist if world > 1 else None)

    tile_idx = [i for i, p in enumerate(passes) if p["kind"] == "tile"]
    dense_idx = [i for i, p in enumerate(passes) if p["kind"] == "dense"]
    tile_ms = times[:, tile_idx].sum(axis=1).mean() if tile_idx else 0.0
    tile_launch_ms = times[:, tile_idx].mean() if tile_idx else float("nan")
    gates_ms = times.sum(axis=1).mean()
    df = dtype == qs.QS_C128
    # FP32 flops of the kernel's own algorithm: double-float updates for complex128, plain FP32 for complex64
    fp32_flops = sum(kernel_flops(plan.op_counts(i), n, _DF_FLOPS if df else _FLOPS) for i in tile_idx)
    if df:  # balanced real and phase-shear-phase updates were counted as real / general ones above
        for i in tile_idx:
            b1, bc = plan.balanced(i)
            fp32_flops -= (_DF_FLOPS["real"] - _DF_FLOPS_BALANCED) * N * (b1 + 0.5 * bc)
            prp, bal_free, prp_nz = plan.scalar_free(i)
            fp32_flops -= (_DF_FLOPS["general"] - _DF_FLOPS_PRP) * N * prp
            fp32_flops -= (_DF_FLOPS_PRP - _DF_FLOPS_PRP_NZ) * N * prp_nz
            fp32_flops -= (_DF_FLOPS["real"] - _DF_FLOPS_BALANCED_FREE) * N * bal_free
    fp32_tf = fp32_flops / (tile_ms / 1e3) / 1e12 if tile_ms else 0.0
    kind = "df" if df else "c64"
    cnt = ncu_counters(kind)
    pass_bytes = 2 * N * s_bytes  # one tile pass reads and writes the whole state once
    achieved = pass_bytes / (tile_launch_ms / 1e3) / 1e9 if tile_idx else 0.0
    roofline = {
        "bound": "hbm", "kernel": ("k_tile_df_p<12> (fused tile pass, double-float)" if df
                                   else "k_tile_p<float, 12> (fused tile pass, FP32)"),
        "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
        "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured"
                       else "fallback 6.8 TB/s (no measured copy bandwidth available)",
        "bytes_per_launch": pass_bytes, "launches_per_step": len(tile_idx), "avg_launch_ms": tile_launch_ms,
        "traffic": cnt["dram_bytes"] * 2.0 ** (n - cnt["n"]) if cnt else None,
        "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one n={cnt['n']} launch, "
                           f"scaled by 2^(n-{cnt['n']})") if cnt else "no ncu capture of the current kernel source",
        "alu": {"what": ("FP32 flops of the double-float updates the kernel applies after fusion, per touched "
                         "amplitude: general 104, general in phase-shear-phase form 74 (52 without its trailing "
                         "phase), real / diagonal / anti-diagonal 44, balanced real 34 (22 without its scalar), "
                         "permutation 0; a phase run counts as one diagonal update") if df else
                        "FP32 flops of the updates the kernel applies after fusion",
                "tflops": fp32_tf, "frac_of_measured_ffma": fp32_tf / FFMA_MEASURED_TFLOPS,
                "frac_of_derived_fp32_peak": fp32_tf / FP32_PEAK_TFLOPS,
                "instruction_issue": issue_summary(kind)},
        "limiter": ("instruction issue of the double-float arithmetic, shared-memory sweeps and index work"
                    if df else "shared-memory bandwidth and instruction issue"),
    }
    launches_per_step = 1 + len(passes) + 2  # init, passes, marginals and norm (2 kernels)

    e2e = None
    if not args.no_e2e:
        # public API with host buffers: the host state (qs_host_alloc: huge pages, page-locked)
        # -> device, qs_run (plans inside), marginals -> host
        hostbuf = qs.HostBuffer(1 << n, np.complex128 if dtype == qs.QS_C128 else np.complex64)
        hostbuf.array[x] = 1.0
        e2e_steps = 5
        state.copy_in_ptr(hostbuf.ptr, 1 << n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        parts = [[], [], []]  # each call below returns after its work is done
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            state.copy_in_ptr(hostbuf.ptr, 1 << n)
            tb = time.perf_counter()
            state.run(gates)
            tc = time.perf_counter()
            state.marginals()
            td = time.perf_counter()
            parts[0].append(tb - ta)
            parts[1].append(tc - tb)
            parts[2].append(td - tc)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_bytes = gate_bytes + 2 * N * s_bytes  # h2d of the state + marginals read (plus gates)
        e2e = {"value": world * e2e_bytes / e2e_s / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": int(N * s_bytes + gates.nbytes), "d2h_bytes_per_step": int(8 * n),
               "ms_per_step": 1e3 * e2e_s, "steps": e2e_steps,
               "breakdown_ms": {"h2d_state": 1e3 * statistics.mean(parts[0]),
                                "h2d_state_each": [round(1e3 * v, 1) for v in parts[0]],
                                "qs_run": 1e3 * statistics.mean(parts[1]),
                                "marginals_to_host": 1e3 * statistics.mean(parts[2])},
               "h2d_GBps": N * s_bytes / statistics.mean(parts[0]) / 1e9,
               "host_buffer": "qs_host_alloc (transparent huge pages, page-locked)",
               "host_huge_page_fraction": hostbuf.huge_page_fraction()}
        hostbuf.close()

    native = None
    if dtype == qs.QS_C128 and not args.no_native:
        # the same step with native FP64 instructions for the gate arithmetic (the paper's
        # precision), under the same protocol; fewer steps, each takes about 4 s
        pn = state.plan(gates, flags=qs.PLAN_ARITH_F64)
        k_native, w_native = min(args.steps, 5), max(3, min(args.warmup, 3))
        n_ms, n_times, n_clocks = timed_steps(pn, k_native, w_native)
        n_value, n_ms_step = job_value(n_ms, step_bytes, k_native, world, dist if world > 1 else None)
        n_tile = n_times[:, tile_idx].mean() if tile_idx else float("nan")
        n_tile_ms = n_times[:, tile_idx].sum(axis=1).mean() if tile_idx else 0.0
        f64_flops = sum(kernel_flops(pn.op_counts(i), n, _FLOPS) for i in tile_idx)
        f64_tf = f64_flops / (n_tile_ms / 1e3) / 1e12 if n_tile_ms else 0.0
        native = {"value": n_value, "unit": "GB/s", "ms_per_step": n_ms_step, "steps": k_native,
                  "warmup": w_native, "dtype": "f64", "clocks": n_clocks,
                  "note": "same step, plan flag QS_PLAN_ARITH_F64 (IEEE double arithmetic on the FP64 pipe)",
                  "roofline": {"bound": "alu", "kernel": "k_tile_p<double, 12> (fused tile pass, FP64)",
                               "achieved": f64_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": f64_tf / FP64_PEAK_TFLOPS,
                               "peak_source": "derived: 152 SMs x 2 DFMA (4 flop) per clock x 2.07 GHz",
                               "what": "FP64 flops of the updates the kernel applies after fusion: 14 per "
                                       "amplitude of a general update, 6 of a real / diagonal / anti-diagonal "
                                       "one, 0 of a permutation",
                               "avg_launch_ms": n_tile,
                               "hbm_frac": pass_bytes / (n_tile / 1e3) / 1e9 / hbm if tile_idx else None}}
        pn.close()

    dense_tc = None
    if not args.no_dense_leg and rank == 0:
        dense_tc = dense_leg(qs, torch, n, max(3, min(args.steps, 10)))

    secondary = None
    if not args.no_secondary:  # every rank runs its share of the instances
        secondary = secondary_gradients(qs, dtype, torch, world, rank, dist if world > 1 else None)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = cpu_baseline(n, gates, s_bytes)

    plan.close()
    state.close()
    if rank == 0:
        kinds = {}
        for p in passes:
            kinds[p["kind"]] = kinds.get(p["kind"], 0) + p["n_gates"]
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2" if dtype == qs.QS_C128 else "f32", "data": "synthetic",
            "config": {"workload": f"QFT({n}) on random basis |x> + 1000-gate random circuit "
                                   f"({'complex128' if dtype == qs.QS_C128 else 'complex64'}, n={n})",
                       "n": n, "gates": len(gates), "state_bytes": int(N * s_bytes),
                       "l2": "state larger than L2 (129 MB): no flush needed", "parallelism": f"replicas x{world}",
                       "arith": ("complex128 state, IEEE double at plan boundaries; gate arithmetic in "
                                 "double-float (FP32 pairs, error-free transforms), parity with the FP64 oracle "
                                 "at 1e-12 on every amplitude of this step; native FP64 in native_f64")
                       if dtype == qs.QS_C128 else "complex64 state, FP32 arithmetic, FP64 reductions"},
            "effective_over_hbm_peak": value / hbm,
            "breakdown": {"plan_ms": plan_ms, "gates_ms": gates_ms, "tile_ms": tile_ms, "passes": len(passes),
                          "dense_passes": len(dense_idx),
                          "dense_ms": float(times[:, dense_idx].sum(axis=1).mean()) if dense_idx else 0.0,
                          "device_ops_after_fusion": device_ops,
                          "tile_passes": len(tile_idx), "gates_in_tile_passes": kinds.get("tile", 0),
                          "gates_in_single_passes": kinds.get("single", 0), "gate_bytes": gate_bytes,
                          "gates_per_s": len(gates) / (gates_ms / 1e3)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "secondary": secondary,
            "native_f64": native,
            "dense_tc": dense_tc,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed(fn, stream, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_random33(args):
    """500-gate random circuits at n=33 complex128 and n=34 complex64 (128 GiB each),
    and the error of both precisions against the FP64 oracle at n=26."""
    import torch
    torch.cuda.set_device(0)
    from paper_1601_07195_gb300 import qs
    from oracle import oracle as O
    seed = G.SEEDS["random33"]
    out = {"workload": "random33", "runs": []}
    for n, dt, s_bytes in ((33, qs.QS_C128, 16), (34, qs.QS_C64, 8)):
        gates, _ = G.random_circuit(n, 500, seed)
        stream = torch.cuda.Stream()
        st = qs.State.create(n, dt, stream=stream)
        plan = st.plan(gates)
        bytes_ = sum(gate_cost(g, n, s_bytes)[0] for g in gates)
        times = []
        for rep in range(1 + max(1, args.steps)):
            st.init_basis(0)
            ms, _ = _timed(plan.execute, stream, torch)
            if rep >= 1:
                times.append(ms)
        nrm = st.norm()
        ms = statistics.mean(times)
        out["runs"].append({"n": n, "dtype": "c128" if dt == qs.QS_C128 else "c64", "gates": len(gates),
                            "passes": plan.stats()["passes"], "ms_per_circuit": ms,
                            "gates_per_s": len(gates) / (ms / 1e3), "GBps": bytes_ / (ms / 1e3) / 1e9,
                            "hbm_frac": bytes_ / (ms / 1e3) / 1e9 / hbm_peak()[0], "norm_minus_1": nrm - 1.0})
        plan.close()
        st.close()
        torch.cuda.empty_cache()
    # error table at n = 26 (same circuit family and seed)
    n = 26
    gates, _ = G.random_circuit(n, 500, seed)
    t0 = time.perf_counter()
    ref = O.simulate(n, gates)
    t_oracle = time.perf_counter() - t0
    z0 = G.terms([(G.P_Z, 0, -1, 1.0)])
    ref_z0 = O.expect(ref, z0)
    for dt, name in ((qs.QS_C128, "c128"), (qs.QS_C64, "c64")):
        with qs.State.create(n, dt) as st:
            st.run(gates)
            amp = st.to_numpy()
            out.setdefault("error_n26", {})[name] = {
                "max_abs_amplitude": float(np.max(np.abs(amp - ref))),
                "norm_minus_1": st.norm() - 1.0, "z0_error": st.expect(z0) - ref_z0}
    out["error_n26"]["oracle_seconds_single_core"] = t_oracle
    print(json.dumps(out), flush=True)


def run_adjoint28(args):
    """Adjoint gradient of the n=28 complex64 Ising workload (L=20, 1120 angles)
    against parameter shift (2 forward simulations per angle) on the same GPU."""
    import torch
    torch.cuda.set_device(0)
    from paper_1601_07195_gb300 import qs
    n, layers = 28, 20
    seed = G.SEEDS["adjoint28"]
    gates, p = G.ansatz(n, layers)
    theta = G.angles(p, seed)
    obs = G.ising_observable(n, seed + 1)
    inst = [{"n": n, "gates": gates, "theta": theta, "terms": obs}]
    res = {"workload": "adjoint28", "n": n, "params": p, "gates": len(gates)}
    for dt, name in ((qs.QS_C64, "c64"), (qs.QS_C128, "c128")):
        b = qs.Batch(inst, dt)
        b.execute()  # plans and captures
        t0 = time.perf_counter()
        reps = max(1, args.steps)
        for _ in range(reps):
            e, g = b.execute()
        res[f"adjoint_s_{name}"] = (time.perf_counter() - t0) / reps
        res[f"energy_{name}"] = float(e[0])
        res[f"grad_{name}"] = g[0]
        b.close()
        torch.cuda.empty_cache()
    res["grad_max_abs_c64_vs_c128"] = float(np.max(np.abs(res["grad_c64"] - res["grad_c128"])))
    res["energy_c64_minus_c128"] = res["energy_c64"] - res["energy_c128"]
    # parameter shift on the same GPU: 2 planned forward simulations + expectation per angle (sampled)
    stream = torch.cuda.Stream()
    with qs.State.create(n, qs.QS_C64, stream=stream) as st:
        def energy(th):
            st.init_basis(0)
            pl = st.plan(gates, th)
            pl.execute()
            e = st.expect(obs)
            pl.close()
            return e
        energy(theta)
        sample = 6
        t0 = time.perf_counter()
        shift = []
        for k in range(sample):
            tp, tm = theta.copy(), theta.copy()
            tp[k] += np.pi / 2
            tm[k] -= np.pi / 2
            shift.append(0.5 * (energy(tp) - energy(tm)))
        t_ps = (time.perf_counter() - t0) / sample
    res["param_shift_s_per_angle"] = t_ps
    res["param_shift_s_all_angles_extrapolated"] = t_ps * p
    res["param_shift_sample"] = sample
    res["param_shift_vs_adjoint_c64_max_abs"] = float(np.max(np.abs(np.array(shift) - res["grad_c64"][:sample])))
    res["speedup_adjoint_c64_vs_param_shift"] = t_ps * p / res["adjoint_s_c64"]
    res["grad_c64"] = None
    res["grad_c128"] = None
    print(json.dumps(res), flush=True)


def _lanes_vs_pairs(st, m, amp_bytes, stream, torch):
    """GB/s of a single-qubit gate, and of a gate controlled by the top qubit, on
    targets 0..4 through each kernel form (the lane exchange and the pair kernel)."""
    from paper_1601_07195_gb300 import qs
    n = st.n
    N = float(1 << n)
    out = {}
    for name, mode in (("lanes", qs.LANES_ON), ("pair_kernel", qs.LANES_OFF)):
        st.set_lanes(mode)
        g1, gc = [], []
        for k in range(5):
            ms, _ = _timed(lambda: [st.apply_1q(k, m) for _ in range(3)], stream, torch)
            g1.append(2 * N * amp_bytes / (ms / 3 / 1e3) / 1e9)
            ms, _ = _timed(lambda: [st.apply_ctrl(n - 1, k, m) for _ in range(3)], stream, torch)
            gc.append(N * amp_bytes / (ms / 3 / 1e3) / 1e9)
        out[name] = {"gate1q_GBps": g1, "ctrl_top_GBps": gc}
    st.set_lanes(qs.LANES_AUTO)
    return out


def run_sweeps(args):
    """Per-target single-gate GB/s at n (default 30) complex128 (strided kernels),
    the controlled-gate (c, t) grid (the Fig. 6 analogue), and IQFT fused vs
    unfused for n = 18..33 (the Fig. 8 analogue; the largest sizes as memory allows)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1601_07195_gb300 import qs
    n = args.n
    hbm, _ = hbm_peak()
    stream = torch.cuda.Stream()
    out = {"workload": "sweeps", "n": n, "dtype": "c128", "hbm_peak_GBps": hbm}
    haar = G.gate_u1(0, G.haar_2x2(G.SplitMix64(9)))[0]["m"]
    N = float(1 << n)
    parts = set(args.parts.split(","))
    with qs.State.create(n, qs.QS_C128, stream=stream) as st:
        st.init_basis(0)
        for name, native in ((("df", False), ("f64", True)) if "gate1q" in parts else ()):
            st.set_arith(native)
            for _ in range(3):
                st.apply_1q(0, haar)
            per_k = []
            for k in range(n):
                ms, _ = _timed(lambda: [st.apply_1q(k, haar) for _ in range(3)], stream, torch)
                per_k.append(2 * N * 16 / (ms / 3 / 1e3) / 1e9)
            out[f"gate1q_GBps_by_target_{name}"] = per_k
            out[f"gate1q_frac_{name}"] = {"min": min(per_k) / hbm, "max": max(per_k) / hbm}
            # targets 0..4: the two kernel forms (the line above uses the default choice)
            out[f"targets0to4_{name}"] = _lanes_vs_pairs(st, haar, 16, stream, torch)
        st.set_arith(False)
        grid = [[None] * n for _ in range(n)]
        for c in (range(n) if "ctrl" in parts else ()):
            for t in range(n):
                if c == t:
                    continue
                ms, _ = _timed(lambda: st.apply_ctrl(c, t, haar), stream, torch)
                grid[c][t] = N * 16 / (ms / 1e3) / 1e9
        flat = [v for row in grid for v in row if v is not None]
    if "gate1q" in parts:
        with qs.State.create(n, qs.QS_C64, stream=stream) as st:
            for _ in range(3):
                st.apply_1q(0, haar)
            per_k = []
            for k in range(n):
                ms, _ = _timed(lambda: [st.apply_1q(k, haar) for _ in range(3)], stream, torch)
                per_k.append(2 * N * 8 / (ms / 3 / 1e3) / 1e9)
            out["gate1q_GBps_by_target_c64"] = per_k
            out["gate1q_frac_c64"] = {"min": min(per_k) / hbm, "max": max(per_k) / hbm}
            out["targets0to4_c64"] = _lanes_vs_pairs(st, haar, 8, stream, torch)
    if flat:
        out["ctrl_GBps_grid"] = grid
        out["ctrl_GBps_summary"] = {"min": min(flat), "max": max(flat), "mean": statistics.mean(flat),
                                   "c0_mean": statistics.mean(v for v in grid[0] if v is not None),
                                   "c_ge_10_mean": statistics.mean(v for c in range(min(10, n - 1), n)
                                                                   for v in grid[c] if v is not None)}
    torch.cuda.empty_cache()
    iqft = []
    free = torch.cuda.mem_get_info()[0]
    for m in (range(18, 34) if "iqft" in parts else ()):
        if (16 << m) > 0.9 * free:
            iqft.append({"n": m, "skipped": "state does not fit device memory"})
            continue
        gates = G.inverse_circuit(G.qft_circuit(m))
        bytes_ = sum(gate_cost(g, m, 16)[0] for g in gates)
        row = {"n": m, "gates": len(gates), "algorithmic_GB": bytes_ / 1e9}
        with qs.State.create(m, qs.QS_C128, stream=stream) as st:
            for name, flags in (("fused", qs.PLAN_DEFAULT), ("unfused", qs.PLAN_NO_FUSION)):
                p = st.plan(gates, flags=flags)
                st.init_basis(1)
                p.execute()
                ms, _ = _timed(p.execute, stream, torch)
                row[f"{name}_ms"] = ms
                row[f"{name}_GBps"] = bytes_ / (ms / 1e3) / 1e9
                row[f"{name}_passes"] = p.stats()["passes"]
                p.close()
        row["fused_over_unfused"] = row["unfused_ms"] / row["fused_ms"]
        iqft.append(row)
        torch.cuda.empty_cache()
    if iqft:
        out["iqft_fused_vs_unfused"] = iqft
    print(json.dumps(out), flush=True)


def _gate_run_low6(depth, seed):
    """`depth` gates on qubits 0..5 (two Haar single-qubit gates, then a controlled
    Haar gate, repeating), and their product as a 64 x 64 matrix (host, FP64)."""
    rng = G.SplitMix64(seed)
    gates = []
    for j in range(depth):
        t = j % 6
        gates.append(G.gate_cu((t + 1 + j % 5) % 6, t, G.haar_2x2(rng)) if j % 3 == 2 else G.gate_u1(t, G.haar_2x2(rng)))
    gates = G.concat(gates)
    U = np.eye(64, dtype=np.complex128)
    eye2 = np.eye(2)
    for g in gates:
        m = g["m"]
        Q = np.array([[m[0] + 1j * m[1], m[2] + 1j * m[3]], [m[4] + 1j * m[5], m[6] + 1j * m[7]]])
        if int(g["kind"]) == G.G_U1:
            op = np.eye(1)
            for k in reversed(range(6)):
                op = np.kron(op, Q if k == g["t"] else eye2)
        else:
            p0, p1 = np.eye(1), np.eye(1)
            for k in reversed(range(6)):
                p0 = np.kron(p0, np.diag([1.0, 0.0]) if k == g["c"] else eye2)
                p1 = np.kron(p1, np.diag([0.0, 1.0]) if k == g["c"] else (Q if k == g["t"] else eye2))
            op = p0 + p1
        U = op @ U
    return gates, U


def run_dense(args):
    """The dense 64 x 64 block on qubits 0..5 of an n = 30 complex64 state on the
    tensor cores (qs_apply_dense), against the same gate runs applied by the
    fused SIMT tile pass (one tile pass of `depth` updates), CUDA events."""
    import torch
    torch.cuda.set_device(0)
    from paper_1601_07195_gb300 import qs
    n = args.n
    N = float(1 << n)
    hbm, hbm_src = hbm_peak()
    stream = torch.cuda.Stream()
    out = {"workload": "dense", "n": n, "dtype": "c64", "runs": []}
    with qs.State.create(n, qs.QS_C64, stream=stream) as st:
        st.init_basis(0)
        for depth in (8, 32, 128):
            gates, U = _gate_run_low6(depth, 40 + depth)
            for _ in range(max(3, args.warmup)):
                st.apply_dense(U)
            ms = []
            for _ in range(max(3, args.steps)):
                m, _ = _timed(lambda: st.apply_dense(U), stream, torch)
                ms.append(m)
            tc_ms = statistics.median(ms)
            p = st.plan(gates, flags=qs.PLAN_NO_DENSE)
            for _ in range(3):
                p.execute()
            sm = []
            for _ in range(max(3, args.steps)):
                m, _ = _timed(p.execute, stream, torch)
                sm.append(m)
            simt_ms = statistics.median(sm)
            stats = p.stats()
            p.close()
            # the same run planned as usual: one tensor-core pass when it is long enough
            pd = st.plan(gates)
            for _ in range(3):
                pd.execute()
            dm = []
            for _ in range(max(3, args.steps)):
                m, _ = _timed(pd.execute, stream, torch)
                dm.append(m)
            planned_ms = statistics.median(dm)
            dense_passes = sum(1 for ps in pd.passes() if ps["kind"] == "dense")
            pd.close()
            bytes_ = 2 * N * 8
            flops = 6 * 2 * 128 * 128 * (N / 64)  # six bf16 piece products per 64-amplitude row
            out["runs"].append({
                "depth": depth, "tensor_ms": tc_ms, "simt_tile_ms": simt_ms,
                "planned_dense_ms": planned_ms, "planned_dense_passes": dense_passes,
                "simt_passes": stats["passes"], "simt_device_ops": stats["device_ops"],
                "speedup_tensor_vs_simt": simt_ms / tc_ms,
                "roofline": {"bound": "hbm", "achieved": bytes_ / (tc_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": bytes_ / (tc_ms / 1e3) / 1e9 / hbm, "peak_source": hbm_src,
                             "traffic": (ncu_counters("dense")["dram_bytes"] * 2.0 ** (n - 25)
                                         if ncu_counters("dense") else None),
                             "tensor_tflops": flops / (tc_ms / 1e3) / 1e12,
                             "tensor_frac_of_bf16_peak": flops / (tc_ms / 1e3) / 1e12 / bf16_peak()[0]}})
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "random33":
        run_random33(args)
    elif args.workload == "adjoint28":
        run_adjoint28(args)
    elif args.workload == "sweeps":
        run_sweeps(args)
    elif args.workload == "dense":
        run_dense(args)
    elif args.workload == "batch512":
        import torch
        torch.cuda.set_device(0)
        from paper_1601_07195_gb300 import qs
        for dt in (qs.QS_C128, qs.QS_C64):
            print(json.dumps(secondary_gradients(qs, dt, torch)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
