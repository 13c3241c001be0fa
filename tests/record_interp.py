"""Host reading of a complex128 double-float plan's tile records (test aid).

Applies the records each tile pass hands its kernel (include/qs_records.h) to
a whole state vector in complex128 numpy arithmetic, with each record double
taken as hi + lo.  Single-gate passes apply their gate through the oracle.
Comparing the result with the oracle applying the circuit checks the
planner's rewrites on the CPU: the products of adjacent gates, the phase-run
tables, the phase-shear-phase and scalar-free forms and the scalars moved
between records.  It does not check the kernels.
"""

import numpy as np

from oracle import oracle as O


def _dbl(c, j):
    return float(c[2 * j]) + float(c[2 * j + 1])


def _cpx(c, j):
    """doubles j, j + 1 as (re, im)"""
    return complex(_dbl(c, j), _dbl(c, j + 1))


def _pair(cls, c, a, b):
    if cls <= 5:
        q11, q12, q21, q22 = _cpx(c, 0), _cpx(c, 2), _cpx(c, 4), _cpx(c, 6)
        return q11 * a + q12 * b, q21 * a + q22 * b
    if cls == 6:
        s1, s3 = float(c[2]), float(c[10])
        return _dbl(c, 0) * (a + s1 * b), _dbl(c, 4) * (a + s3 * b)
    if cls == 9:
        s1, s3, r = float(c[2]), float(c[10]), float(c[8])
        return a + s1 * b, r * (a + s3 * b)
    if cls in (7, 8, 10, 11):
        if cls in (8, 11):
            a, b = b, a
        y, t, z = _cpx(c, 0), _dbl(c, 2), _cpx(c, 4)
        w = y * b
        a2, b2 = a + t * w, w - t * a
        return a2, (z * b2 if cls in (7, 8) else b2)
    raise ValueError(f"unknown record class {cls}")


def apply_records(psi, recs, tile_qubits):
    """Apply one pass's records to psi (complex128, modified in place)."""
    idx = np.arange(psi.size, dtype=np.int64)
    b = len(tile_qubits)
    g = 0
    while g < len(recs):
        r = recs[g]
        kind, cls, c = int(r["kind"]), int(r["cls"]), r["c"]
        if kind == 3:  # phase run: header, tile-bit factors, outside factors
            j, n_out, tile_rec = int(r["tq"]), int(r["cb"]), (b + 3) // 4
            fac = np.full(psi.size, _cpx(c, 0), dtype=np.complex128)
            for k in range(b):
                v = _cpx(recs[g + 1 + k // 4]["c"], 2 * (k % 4))
                fac = np.where((idx >> tile_qubits[k]) & 1, fac * v, fac)
            for i in range(n_out):
                pr = recs[g + 1 + tile_rec + i // 4]
                f = i % 4
                q = int((pr["tb"], pr["tq"], pr["cb"], pr["cq"])[f])
                fac = np.where((idx >> q) & 1, fac * _cpx(pr["c"], 2 * f), fac)
            sel = ((idx >> j) & 1) == 1
            psi[sel] *= fac[sel]
            g += 1 + cls
            continue
        if kind == 2:
            qa, qb = int(r["tq"]), int(r["cq"])
            diff = ((idx >> qa) ^ (idx >> qb)) & 1
            psi[:] = psi[idx ^ (diff * ((1 << qa) | (1 << qb)))]
        elif kind in (0, 1):
            t = int(r["tq"])
            lo = idx[((idx >> t) & 1) == 0]
            if kind == 1:
                lo = lo[((lo >> int(r["cq"])) & 1) == 1]
            hi = lo | (1 << t)
            a2, b2 = _pair(cls, c, psi[lo], psi[hi])
            psi[lo], psi[hi] = a2, b2
        else:
            raise ValueError(f"record kind {kind} outside a phase run")
        g += 1
    return psi


def run_plan(plan, psi, gates, theta=None):
    """psi after every pass of plan (a complex128 double-float plan of gates)."""
    psi = np.array(psi, dtype=np.complex128)
    for i, ps in enumerate(plan.passes()):
        if ps["kind"] == "single":
            psi = O.run(psi, gates[ps["gates"][0]:ps["gates"][0] + 1], theta)
        else:
            recs, tq = plan.records(i)
            apply_records(psi, recs, tq)
    return psi
