/* qs_records.h -- read-only view of the tile-pass records a complex128
 * double-float plan hands its tile kernel (Section 4.4, Fig. 5: the gates of a
 * pass applied block by block).  A test aid: it lets a host program apply a
 * plan's records in its own arithmetic and check the planner's rewrites
 * (products of adjacent gates, phase runs, the scalar-free forms of
 * QS_PLAN_NO_PRP) against a reference, without a GPU.  Nothing here is needed
 * to run a plan.
 *
 * Record layout (96 bytes, native byte order):
 *   int32 kind    0 single-qubit, 1 controlled, 2 swap, 3 phase-run header,
 *                 4 phase-run or diagonal-run payload, 5 diagonal-run header
 *   int32 cls     gate class, see below
 *   int32 tb, tq  target tile bit (-1: outside the tile) and target qubit;
 *                 swap: first qubit
 *   int32 cb, cq  control tile bit (-1: outside the tile or none) and control
 *                 qubit (-1: none); swap: second qubit
 *   int32 pad[2]
 *   float c[16]   eight doubles, each as an unevaluated pair c[2j] + c[2j+1]
 *                 (hi, lo); for classes 0-5 doubles 0..7 are q11, q12, q21,
 *                 q22 as (re, im) pairs in row-major order.
 *
 * Classes (gate update on the amplitude pair (a, b) = (bit t = 0, bit t = 1),
 * for controlled records only where the control bit is 1):
 *   0 general, 1 real, 2 diagonal, 3 diagonal with q11 = 1, 4 anti-diagonal,
 *   5 the exact X matrix: the 2x2 product with the matrix above.  A diagonal
 *     record whose target is outside the tile multiplies every amplitude by
 *     q11 or q22 according to its target bit.
 *   6 balanced real: a' = q11 (a + s1 b), b' = q21 (a + s3 b) with q11 in
 *     double 0, q21 in double 4, s1 = c[2], s3 = c[10] (+-1).
 *   9 balanced real without its scalar: a' = a + s1 b, b' = r (a + s3 b),
 *     s1 = c[2], s3 = c[10], r = c[8] (+-1).
 *   7 phase-shear-phase: w = y b; a' = a + t w; b' = z (w - t a) with
 *     y = doubles (0, 1), t = double 2, z = doubles (4, 5);
 *   8 the same applied to the swapped pair: (a, b) := (b, a) first;
 *  10, 11 classes 7 and 8 without the final product by z.
 *   The scalars left out by classes 7-11 are multiplied into another record
 *   of the same pass, so a pass's records together apply the pass's gates.
 *
 * Phase runs (kind 3 and 4): a header (cls = number of payload records,
 * tb = tile bit jb of pivot qubit j = tq, cb = number of outside factors,
 * cq = unused here) with factor C0 = doubles (0, 1); then ceil(b / 4) payload
 * records whose factor slot f (doubles 2f, 2f+1) of record r is psi for tile
 * bit 4r + f; then ceil(cb / 4) payload records whose slot f holds the factor
 * of the qubit in field tb, tq, cb or cq (f = 0..3).  Every amplitude whose
 * bit j is 1 is multiplied by C0 times psi of each of its set tile bits times
 * the factor of each outside qubit it has set.
 *
 * Diagonal runs (kind 5 and 4): a header (cls = number of payload records,
 * tb = number of terms T, cq = lob, the low-half bit count); then ceil(T / 4)
 * payload records whose slot f holds the factor of term 4r + f and whose int
 * field tb, tq, cb or cq (f = 0..3) holds type << 16 | x << 8 | y:
 *   type 0: tile bit x, times outside qubit y (255: unconditional);
 *   type 1: tile bits x and y (both in one half: both < lob or both >= lob);
 *   type 2: outside qubit x, times outside qubit y (255: none).
 * Every amplitude is multiplied by the factor of each term whose bits are all
 * set in its index.
 */
#ifndef QS_RECORDS_H
#define QS_RECORDS_H

#include "qs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Records of pass i of plan p (zero records for single-gate passes).  *n
 * receives the count; when out is not NULL it receives the records (cap =
 * room in records; QS_EINVAL if too small).  tile_qubits, if not NULL,
 * receives the qubit of each tile bit (up to 14 ints), *b, if not NULL, the
 * number of tile bits, and *format, if not NULL, the record format:
 *   1 double-float (complex128 plans; the 96-byte layout above),
 *   2 float (complex64 plans), 3 double (complex128 with QS_PLAN_ARITH_F64):
 *     the same eight int32 fields followed by eight floats / doubles m[8]
 *     (64 / 96 bytes) that hold the matrix q11, q12, q21, q22 as (re, im)
 *     pairs; classes 0-5 only; a phase-run factor slot f is m[2f], m[2f+1].
 * The plan keeps ownership of its records; this copies them. */
QS_API qs_status qs_plan_pass_records(const qs_plan* p, int i, void* out, int cap, int* n, int* tile_qubits,
                                      int* b, int* format);

#ifdef __cplusplus
}
#endif

#endif /* QS_RECORDS_H */
