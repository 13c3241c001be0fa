"""Host reading of a complex128 double-float plan's tile records (test aid).

Applies the records each tile pass hands its kernel (include/qs_records.h) to
a whole state vector in complex128 numpy arithmetic, with each record double
taken as hi + lo (phase runs and diagonal runs included).  Single-gate passes apply their gate through the oracle; dense passes (complex64
plans) apply the 64 x 64 matrix the planner formed for them.
Comparing the result with the oracle applying the circuit checks the
planner's rewrites on the CPU: the products of adjacent gates, the phase-run
tables, the phase-shear-phase and scalar-free forms and the scalars moved
between records.  It does not check the kernels.
"""

import numpy as np

from oracle import oracle as O


class _Rec:
    """The eight matrix / factor numbers of a record: double j of a
    double-float record is c[2j] + c[2j+1]; a native record holds m[j]."""

    def __init__(self, r, fmt):
        self.c = r["c"] if fmt == 1 else None
        self.v = ([float(r["c"][2 * j]) + float(r["c"][2 * j + 1]) for j in range(8)] if fmt == 1
                  else [float(x) for x in r["m"]])

    def dbl(self, j):
        return self.v[j]

    def cpx(self, j):
        """numbers j, j + 1 as (re, im)"""
        return complex(self.v[j], self.v[j + 1])


def _pair(cls, rec, a, b):
    """(a', b') of one pair update of class cls; classes 6-11 occur in
    double-float records only and read their signs from the raw floats c."""
    if cls <= 5:
        q11, q12, q21, q22 = rec.cpx(0), rec.cpx(2), rec.cpx(4), rec.cpx(6)
        return q11 * a + q12 * b, q21 * a + q22 * b
    c = rec.c
    if cls == 6:
        s1, s3 = float(c[2]), float(c[10])
        return rec.dbl(0) * (a + s1 * b), rec.dbl(4) * (a + s3 * b)
    if cls == 9:
        s1, s3, r = float(c[2]), float(c[10]), float(c[8])
        return a + s1 * b, r * (a + s3 * b)
    if cls in (7, 8, 10, 11):
        if cls in (8, 11):
            a, b = b, a
        y, t, z = rec.cpx(0), rec.dbl(2), rec.cpx(4)
        w = y * b
        a2, b2 = a + t * w, w - t * a
        return a2, (z * b2 if cls in (7, 8) else b2)
    raise ValueError(f"unknown record class {cls}")


def apply_records(psi, recs, tile_qubits, fmt=1):
    """Apply one pass's records (format fmt, include/qs_records.h) to psi
    (complex128, modified in place)."""
    idx = np.arange(psi.size, dtype=np.int64)
    b = len(tile_qubits)
    g = 0
    while g < len(recs):
        r = recs[g]
        kind, cls, rec = int(r["kind"]), int(r["cls"]), _Rec(r, fmt)
        if kind == 3:  # phase run: header, tile-bit factors, outside factors
            j, n_out, tile_rec = int(r["tq"]), int(r["cb"]), (b + 3) // 4
            fac = np.full(psi.size, rec.cpx(0), dtype=np.complex128)
            for k in range(b):
                v = _Rec(recs[g + 1 + k // 4], fmt).cpx(2 * (k % 4))
                fac = np.where((idx >> tile_qubits[k]) & 1, fac * v, fac)
            for i in range(n_out):
                pr = recs[g + 1 + tile_rec + i // 4]
                f = i % 4
                q = int((pr["tb"], pr["tq"], pr["cb"], pr["cq"])[f])
                fac = np.where((idx >> q) & 1, fac * _Rec(pr, fmt).cpx(2 * f), fac)
            sel = ((idx >> j) & 1) == 1
            psi[sel] *= fac[sel]
            g += 1 + cls
            continue
        if kind == 5:  # diagonal run: header, then bit / pair / scalar terms, four per record
            n_terms = int(r["tb"])
            fac = np.ones(psi.size, dtype=np.complex128)
            for i in range(n_terms):
                pr = recs[g + 1 + i // 4]
                f = i % 4
                code = int((pr["tb"], pr["tq"], pr["cb"], pr["cq"])[f])
                typ, x, y = code >> 16, (code >> 8) & 255, code & 255
                if typ == 0:    # tile bit x, outside condition y (255: none)
                    on = (idx >> tile_qubits[x]) & 1
                    if y != 255:
                        on = on & ((idx >> y) & 1)
                elif typ == 1:  # tile bits x and y
                    on = ((idx >> tile_qubits[x]) & 1) & ((idx >> tile_qubits[y]) & 1)
                else:           # outside qubits x and y (255: none)
                    on = (idx >> x) & 1
                    if y != 255:
                        on = on & ((idx >> y) & 1)
                fac = np.where(on == 1, fac * _Rec(pr, fmt).cpx(2 * f), fac)
            psi *= fac
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
            a2, b2 = _pair(cls, rec, psi[lo], psi[hi])
            psi[lo], psi[hi] = a2, b2
        else:
            raise ValueError(f"record kind {kind} outside a phase run")
        g += 1
    return psi


def run_plan(plan, psi, gates, theta=None):
    """psi (complex128) after every pass of plan, a plan of gates."""
    psi = np.array(psi, dtype=np.complex128)
    for i, ps in enumerate(plan.passes()):
        if ps["kind"] == "single":
            psi = O.run(psi, gates[ps["gates"][0]:ps["gates"][0] + 1], theta)
        elif ps["kind"] == "dense":  # the pass's 64 x 64 matrix on qubits 0..5
            psi = (psi.reshape(-1, 64) @ plan.dense_matrix(i).T).reshape(-1)
        else:
            recs, tq, fmt = plan.records(i)
            apply_records(psi, recs, tq, fmt)
    return psi
