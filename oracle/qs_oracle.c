/*
 * qs_oracle.c -- plain, slow, single-threaded CPU FP64 reference for the
 * state-vector gate engine.  TEST INFRASTRUCTURE ONLY: it is used by the
 * tests, by the smoke check and by the CPU-baseline leg of the benchmark,
 * never by the product path.  It shares no code with the CUDA library.
 *
 * Source of each routine (qHiPSTER, Smelyanskiy, Sawaya, Aspuru-Guzik,
 * arXiv:1601.07195):
 *   - state of n qubits = 2^n complex doubles, qubit k = bit k of the index
 *     (Section 2; "2^(n+4) bytes" in the introduction, stride 2^k in Section 2);
 *   - single-qubit gate = Eq. 2, evaluated as the two-level loop of Fig. 3
 *     (outer loop over groups of 2^(k+1), inner loop over the 2^k pairs);
 *   - controlled-Q gate = Eq. 3: the same update restricted to indices whose
 *     control bit c is 1 (Section 3.1);
 *   - SWAP, rotation gates, reductions and gradients are not in the paper;
 *     each is written from its textbook definition, stated at the routine.
 *
 * Compiled with -ffp-contract=off: every product and sum is a separately
 * rounded IEEE double operation.  Reductions use Neumaier's compensated sum
 * (A. Neumaier, ZAMM 54, 1974) so the reference is tighter than the kernels.
 *
 * The same file is also compiled a second way, -O3 -fopenmp, for timing on
 * all host cores and for reference states too large for one core: the
 * "#pragma omp" lines below split the pair loops of the gate routines (and
 * the closed-form QFT fill) across threads, the threading of Section 4.2.
 * Every pair is still updated by the same separately rounded operations, so
 * both builds give bit-identical states.  Reductions stay serial.  Without
 * -fopenmp the pragmas are ignored.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t kind, t, c, param; double m[8]; } or_gate;    /* 80 bytes */
typedef struct { int32_t kind, q0, q1, pad; double coef; } or_term;    /* 24 bytes */

enum { OR_U1 = 0, OR_CU = 1, OR_SWAP = 2, OR_RX = 3, OR_RY = 4, OR_RZ = 5 };
enum { OR_Z = 0, OR_ZZ = 1, OR_X = 2 };

/* ---- complex helpers on (re, im) pairs, no fused operations ---------------- */
typedef struct { double re, im; } cplx;

static cplx cmul(cplx a, cplx b) {
    cplx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}
static cplx cadd(cplx a, cplx b) { cplx r; r.re = a.re + b.re; r.im = a.im + b.im; return r; }
static cplx entry(const double m[8], int j) { cplx r; r.re = m[2 * j]; r.im = m[2 * j + 1]; return r; }

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum* a) { return a->s + a->c; }

/* ---- state preparation ----------------------------------------------------- */
void or_init_basis(double* psi, int n, uint64_t x) {
    uint64_t N = (uint64_t)1 << n;
    memset(psi, 0, (size_t)N * 2 * sizeof(double));
    psi[2 * x] = 1.0;
}

/* ---- Eq. 2 via the loop nest of Fig. 3 ------------------------------------- */
/* alpha'_{..0_k..} = q11 alpha_{..0_k..} + q12 alpha_{..1_k..}
   alpha'_{..1_k..} = q21 alpha_{..0_k..} + q22 alpha_{..1_k..}
   m = (q11, q12, q21, q22) as (re, im) pairs; the pair is (i, i + s). */
static void pair_update(double* psi, uint64_t i, uint64_t s, const double m[8]) {
    cplx q11 = entry(m, 0), q12 = entry(m, 1), q21 = entry(m, 2), q22 = entry(m, 3);
    cplx a, b;
    a.re = psi[2 * i]; a.im = psi[2 * i + 1];
    b.re = psi[2 * (i + s)]; b.im = psi[2 * (i + s) + 1];
    cplx a2 = cadd(cmul(q11, a), cmul(q12, b));
    cplx b2 = cadd(cmul(q21, a), cmul(q22, b));
    psi[2 * i] = a2.re; psi[2 * i + 1] = a2.im;
    psi[2 * (i + s)] = b2.re; psi[2 * (i + s) + 1] = b2.im;
}

/* Outer loop over the groups of 2^(k+1) amplitudes, inner loop over the 2^k
 * pairs of a group.  The OpenMP build splits the outer loop across threads when
 * there are many groups, else the inner loop of each group. */
void or_apply_1q(double* psi, int n, int k, const double m[8]) {
    uint64_t N = (uint64_t)1 << n, s = (uint64_t)1 << k;
    if (N / (2 * s) >= 64) {
#pragma omp parallel for schedule(static)
        for (uint64_t g = 0; g < N; g += 2 * s)
            for (uint64_t i = g; i < g + s; ++i) pair_update(psi, i, s, m);
    } else {
        for (uint64_t g = 0; g < N; g += 2 * s) {
#pragma omp parallel for schedule(static) if (s >= 4096)
            for (uint64_t i = g; i < g + s; ++i) pair_update(psi, i, s, m);
        }
    }
}

/* ---- Eq. 3: Q on target t only where control bit c is 1 --------------------- */
void or_apply_ctrl(double* psi, int n, int c, int t, const double m[8]) {
    uint64_t N = (uint64_t)1 << n, s = (uint64_t)1 << t;
    if (N / (2 * s) >= 64) {
#pragma omp parallel for schedule(static)
        for (uint64_t g = 0; g < N; g += 2 * s)
            for (uint64_t i = g; i < g + s; ++i)
                if ((i >> c) & 1u) pair_update(psi, i, s, m);  /* control in |0>: unchanged */
    } else {
        for (uint64_t g = 0; g < N; g += 2 * s) {
#pragma omp parallel for schedule(static) if (s >= 4096)
            for (uint64_t i = g; i < g + s; ++i)
                if ((i >> c) & 1u) pair_update(psi, i, s, m);
        }
    }
}

/* ---- a dense 2^q x 2^q matrix on qubits 0..q-1 -------------------------------
 * Not in the paper: the product of a run of gates on the q lowest qubits as one
 * matrix U (row-major, U[r][c] at U[2 (r 2^q + c)], (re, im)), applied to every
 * group of 2^q consecutive amplitudes x (fixed higher bits): y_r = sum_c U[r][c] x_c,
 * summed in column order.  1 <= q <= 10. */
void or_apply_dense(double* psi, int n, int q, const double* U) {
    uint64_t N = (uint64_t)1 << n, G = (uint64_t)1 << q;
#pragma omp parallel for schedule(static) if (N / G >= 64)
    for (uint64_t g = 0; g < N; g += G) {
        double y[2 * 1024];
        for (uint64_t r = 0; r < G; ++r) {
            cplx acc = {0.0, 0.0};
            for (uint64_t c = 0; c < G; ++c) {
                cplx u, x;
                u.re = U[2 * (r * G + c)]; u.im = U[2 * (r * G + c) + 1];
                x.re = psi[2 * (g + c)]; x.im = psi[2 * (g + c) + 1];
                acc = cadd(acc, cmul(u, x));
            }
            y[2 * r] = acc.re; y[2 * r + 1] = acc.im;
        }
        for (uint64_t r = 0; r < G; ++r) { psi[2 * (g + r)] = y[2 * r]; psi[2 * (g + r) + 1] = y[2 * r + 1]; }
    }
}

/* ---- SWAP(a, b): |.. x_a .. x_b ..> -> |.. x_b .. x_a ..> (index permutation) */
void or_apply_swap(double* psi, int n, int a, int b) {
    uint64_t N = (uint64_t)1 << n;
    /* iteration i touches only i and its partner j, which no other iteration swaps */
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (uint64_t i = 0; i < N; ++i) {
        if (((i >> a) & 1u) == 0 && ((i >> b) & 1u) == 1) {
            uint64_t j = i ^ ((uint64_t)1 << a) ^ ((uint64_t)1 << b);
            double r = psi[2 * i], m = psi[2 * i + 1];
            psi[2 * i] = psi[2 * j]; psi[2 * i + 1] = psi[2 * j + 1];
            psi[2 * j] = r; psi[2 * j + 1] = m;
        }
    }
}

/* ---- closed form of the quantum Fourier transform of a basis state ---------
 * QFT |x> = 2^(-n/2) sum_y exp(2 pi i x y / 2^n) |y>  (the transform the QFT
 * workload of Section 5.3 applies; textbook form, Nielsen & Chuang 5.1).  The
 * phase x y mod 2^n is taken in exact integer arithmetic (n <= 32, so x y
 * fits 64 bits) before the double-precision cosine and sine. */
void or_qft_basis(double* psi, int n, uint64_t x) {
    uint64_t N = (uint64_t)1 << n, mask = N - 1;
    double scale = pow(2.0, -0.5 * n), w = 2.0 * 3.14159265358979323846 / (double)N;
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (uint64_t y = 0; y < N; ++y) {
        double ph = w * (double)((x * y) & mask);
        psi[2 * y] = scale * cos(ph);
        psi[2 * y + 1] = scale * sin(ph);
    }
}

/* ---- rotation gates U(theta) = exp(-i theta G / 2), G in {X, Y, Z} ---------- */
static void set(double m[8], int j, double re, double im) { m[2 * j] = re; m[2 * j + 1] = im; }

/* U(theta); for deriv != 0 the entrywise derivative dU/dtheta = (-i/2) G U(theta). */
static void rotation_matrix(int kind, double theta, int deriv, double m[8]) {
    double c = cos(0.5 * theta), s = sin(0.5 * theta);
    memset(m, 0, 8 * sizeof(double));
    if (!deriv) {
        if (kind == OR_RX) { set(m, 0, c, 0); set(m, 1, 0, -s); set(m, 2, 0, -s); set(m, 3, c, 0); }
        if (kind == OR_RY) { set(m, 0, c, 0); set(m, 1, -s, 0); set(m, 2, s, 0); set(m, 3, c, 0); }
        if (kind == OR_RZ) { set(m, 0, c, -s); set(m, 3, c, s); }
    } else {
        if (kind == OR_RX) { set(m, 0, -0.5 * s, 0); set(m, 1, 0, -0.5 * c); set(m, 2, 0, -0.5 * c); set(m, 3, -0.5 * s, 0); }
        if (kind == OR_RY) { set(m, 0, -0.5 * s, 0); set(m, 1, -0.5 * c, 0); set(m, 2, 0.5 * c, 0); set(m, 3, -0.5 * s, 0); }
        if (kind == OR_RZ) { set(m, 0, -0.5 * s, -0.5 * c); set(m, 3, -0.5 * s, 0.5 * c); }
    }
}

void or_gate_matrix(const or_gate* g, const double* theta, double m[8]) {
    if (g->kind == OR_RX || g->kind == OR_RY || g->kind == OR_RZ) rotation_matrix(g->kind, theta[g->param], 0, m);
    else memcpy(m, g->m, 8 * sizeof(double));
}

static int check_gate(const or_gate* g, int n) {
    if (g->t < 0 || g->t >= n) return -1;
    if (g->kind == OR_CU || g->kind == OR_SWAP) {
        if (g->c < 0 || g->c >= n || g->c == g->t) return -1;
    } else if (g->kind == OR_U1) {
        return 0;
    } else if (g->kind == OR_RX || g->kind == OR_RY || g->kind == OR_RZ) {
        if (g->param < 0) return -1;
    } else {
        return -1;
    }
    return 0;
}

/* Apply one gate; deriv != 0 applies dU/dtheta instead of U for a rotation. */
static void apply_gate(double* psi, int n, const or_gate* g, const double* theta, int deriv) {
    double m[8];
    switch (g->kind) {
    case OR_U1: or_apply_1q(psi, n, g->t, g->m); break;
    case OR_CU: or_apply_ctrl(psi, n, g->c, g->t, g->m); break;
    case OR_SWAP: or_apply_swap(psi, n, g->t, g->c); break;
    default:
        rotation_matrix(g->kind, theta[g->param], deriv, m);
        or_apply_1q(psi, n, g->t, m);
        break;
    }
}

/* The circuit U_P ... U_1 applied in order to psi.  Returns -1 on a bad record. */
int or_run(double* psi, int n, const or_gate* g, int ng, const double* theta, int n_params) {
    for (int j = 0; j < ng; ++j) {
        if (check_gate(&g[j], n)) return -1;
        if (g[j].param >= n_params || (g[j].param >= 0 && theta == NULL)) return -1;
    }
    for (int j = 0; j < ng; ++j) apply_gate(psi, n, &g[j], theta, 0);
    return 0;
}

/* ---- reductions ------------------------------------------------------------ */
/* sum_i |alpha_i|^2 (squared 2-norm, the total probability) */
double or_norm2(const double* psi, int n) {
    uint64_t N = (uint64_t)1 << n;
    nsum a = {0, 0};
    for (uint64_t i = 0; i < N; ++i) nadd(&a, psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1]);
    return nval(&a);
}

/* p1[k] = sum over indices with bit k = 1 of |alpha_i|^2, for every k < n */
void or_marginals(const double* psi, int n, double* p1) {
    uint64_t N = (uint64_t)1 << n;
    for (int k = 0; k < n; ++k) {
        nsum a = {0, 0};
        for (uint64_t i = 0; i < N; ++i)
            if ((i >> k) & 1u) nadd(&a, psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1]);
        p1[k] = nval(&a);
    }
}

/* out[i] = |alpha_i|^2 */
void or_probs(const double* psi, int n, double* out) {
    uint64_t N = (uint64_t)1 << n;
    for (uint64_t i = 0; i < N; ++i) out[i] = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
}

/* <psi| P |psi> for one Pauli term without its coefficient:
   Z_q: eigenvalue 1 - 2 b_q(i);  Z_q Z_r: product of the two signs;
   X_q: sum_i Re(conj(alpha_i) alpha_{i xor 2^q}). */
static double term_value(const double* psi, int n, const or_term* t) {
    uint64_t N = (uint64_t)1 << n;
    nsum a = {0, 0};
    for (uint64_t i = 0; i < N; ++i) {
        double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        if (t->kind == OR_Z) {
            nadd(&a, ((i >> t->q0) & 1u) ? -p : p);
        } else if (t->kind == OR_ZZ) {
            int par = (int)(((i >> t->q0) ^ (i >> t->q1)) & 1u);
            nadd(&a, par ? -p : p);
        } else {
            uint64_t j = i ^ ((uint64_t)1 << t->q0);
            nadd(&a, psi[2 * i] * psi[2 * j] + psi[2 * i + 1] * psi[2 * j + 1]);
        }
    }
    return nval(&a);
}

static int check_terms(const or_term* t, int nt, int n) {
    for (int j = 0; j < nt; ++j) {
        if (t[j].q0 < 0 || t[j].q0 >= n) return -1;
        if (t[j].kind == OR_ZZ && (t[j].q1 < 0 || t[j].q1 >= n || t[j].q1 == t[j].q0)) return -1;
        if (t[j].kind != OR_Z && t[j].kind != OR_ZZ && t[j].kind != OR_X) return -1;
    }
    return 0;
}

/* <psi|H|psi> = sum_j coef_j <psi|P_j|psi>.  Returns NAN on a bad term. */
double or_expect(const double* psi, int n, const or_term* t, int nt) {
    if (check_terms(t, nt, n)) return NAN;
    nsum a = {0, 0};
    for (int j = 0; j < nt; ++j) nadd(&a, t[j].coef * term_value(psi, n, &t[j]));
    return nval(&a);
}

/* out = H psi (out must not alias psi).  Terms are added to each amplitude in
 * term order; the OpenMP build splits the amplitude loop, which keeps that order. */
static void apply_hamiltonian(const double* psi, int n, const or_term* t, int nt, double* out) {
    uint64_t N = (uint64_t)1 << n;
    memset(out, 0, (size_t)N * 2 * sizeof(double));
    for (int j = 0; j < nt; ++j) {
#pragma omp parallel for schedule(static) if (N >= 65536)
        for (uint64_t i = 0; i < N; ++i) {
            if (t[j].kind == OR_X) {
                uint64_t k = i ^ ((uint64_t)1 << t[j].q0);
                out[2 * i] += t[j].coef * psi[2 * k];
                out[2 * i + 1] += t[j].coef * psi[2 * k + 1];
            } else {
                int neg = (t[j].kind == OR_Z) ? (int)((i >> t[j].q0) & 1u)
                                              : (int)(((i >> t[j].q0) ^ (i >> t[j].q1)) & 1u);
                double s = neg ? -t[j].coef : t[j].coef;
                out[2 * i] += s * psi[2 * i];
                out[2 * i + 1] += s * psi[2 * i + 1];
            }
        }
    }
}

/* out = H psi for a checked Pauli sum.  Returns -1 on a bad term. */
int or_apply_hamiltonian(const double* psi, int n, const or_term* t, int nt, double* out) {
    if (check_terms(t, nt, n)) return -1;
    apply_hamiltonian(psi, n, t, nt, out);
    return 0;
}

/* Re <a|b> = sum_i Re(conj(a_i) b_i), compensated. */
double or_dot_re(const double* a, const double* b, int n) {
    uint64_t N = (uint64_t)1 << n;
    nsum s = {0, 0};
    for (uint64_t i = 0; i < N; ++i) nadd(&s, a[2 * i] * b[2 * i] + a[2 * i + 1] * b[2 * i + 1]);
    return nval(&s);
}

/* One checked gate record applied to psi; deriv != 0 applies dU/dtheta of a
 * rotation instead of U (the factor the derivative of the circuit puts in gate
 * j's place).  Returns -1 on a bad record. */
int or_apply_gate(double* psi, int n, const or_gate* g, const double* theta, int n_params, int deriv) {
    if (check_gate(g, n) || g->param >= n_params || (g->param >= 0 && theta == NULL)) return -1;
    if (deriv && g->kind != OR_RX && g->kind != OR_RY && g->kind != OR_RZ) return -1;
    apply_gate(psi, n, g, theta, deriv);
    return 0;
}

/* Energy and gradient of E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U_P..U_1 |0..0>.
 * Definition of the derivative, written out: for every rotation gate j with
 * parameter p, d psi / d theta_p gets the term U_P..U_{j+1} (dU_j/dtheta) U_{j-1}..U_1 |0>,
 * and dE/dtheta_p = 2 Re <H psi | d psi/d theta_p>  (H Hermitian).
 * One full forward simulation per rotation gate: slow, and obviously the definition.
 * grads has n_params entries and is overwritten.  Returns -1 on bad input. */
int or_grad(int n, const or_gate* g, int ng, const double* theta, int n_params,
            const or_term* t, int nt, double* energy, double* grads) {
    uint64_t N = (uint64_t)1 << n;
    for (int j = 0; j < ng; ++j) {
        if (check_gate(&g[j], n)) return -1;
        if (g[j].param >= n_params) return -1;
    }
    if (check_terms(t, nt, n)) return -1;
    double* psi = (double*)malloc((size_t)N * 2 * sizeof(double));
    double* hpsi = (double*)malloc((size_t)N * 2 * sizeof(double));
    double* d = (double*)malloc((size_t)N * 2 * sizeof(double));
    if (!psi || !hpsi || !d) { free(psi); free(hpsi); free(d); return -2; }
    or_init_basis(psi, n, 0);
    for (int j = 0; j < ng; ++j) apply_gate(psi, n, &g[j], theta, 0);
    apply_hamiltonian(psi, n, t, nt, hpsi);
    nsum e = {0, 0};
    for (uint64_t i = 0; i < N; ++i) nadd(&e, psi[2 * i] * hpsi[2 * i] + psi[2 * i + 1] * hpsi[2 * i + 1]);
    *energy = nval(&e);
    for (int p = 0; p < n_params; ++p) grads[p] = 0.0;
    for (int j = 0; j < ng; ++j) {
        if (g[j].param < 0 || (g[j].kind != OR_RX && g[j].kind != OR_RY && g[j].kind != OR_RZ)) continue;
        or_init_basis(d, n, 0);
        for (int i = 0; i < ng; ++i) apply_gate(d, n, &g[i], theta, i == j);
        nsum a = {0, 0};
        for (uint64_t i = 0; i < N; ++i) nadd(&a, hpsi[2 * i] * d[2 * i] + hpsi[2 * i + 1] * d[2 * i + 1]);
        grads[g[j].param] += 2.0 * nval(&a);
    }
    free(psi); free(hpsi); free(d);
    return 0;
}
