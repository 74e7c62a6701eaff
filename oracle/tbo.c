/*
 * CPU oracle for exact amplitudes psi(x) = <x|U|0^n> of open-boundary 1D
 * brickwork circuits (Sec. 2.1 and Sec. 2.2, the amplitude definition).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link or call
 * this file; it exists so that tests, the package smoke check and the
 * benchmark's CPU-baseline leg can check the CUDA path against an
 * independent, slow, obviously correct computation in FP64.
 *
 * It shares no code with the CUDA path. All arithmetic is plain FP64 complex
 * (C99 double _Complex).
 *
 * Conventions (shared with the seeded input generator, not with the kernels):
 *   - qubits q = 0..n-1, CZ layers l = 0..d-1; layer l acts on (i, i+1) for
 *     every i = l (mod 2), i+1 < n;
 *   - one-qubit slots t = 0..d: slot t < d before CZ layer t, slot d after the
 *     last layer;
 *   - gate array u: (d+1)*n gates, gate (t, q) at index t*n + q, each a
 *     row-major 2x2 complex matrix stored as 8 doubles (re, im);
 *   - bitstring x: x[q] in {0,1}; state-vector basis index bit q = x_q.
 *
 * Contents:
 *   tbo_sv_state      dense state vector (the definition written out); its
 *                     entangler may also be a controlled phase diag(1,1,1,
 *                     e^(i phi)) per gate (phi = pi is CZ; Sec. 2.1 allows any
 *                     two-qubit gate of operator Schmidt rank 2)
 *   tbo_nb_amplitude  naive boundary contraction over qubit rows, every row
 *                     in forward time with an explicit wire index (the
 *                     network of Sec. 2.2 contracted row by row; no slot
 *                     reuse, no snake order, no fusion, no rescaling)
 *   tbo_feynman       brute-force sum over every CZ-layer wire value
 *   tbo_tableau_prob  |psi(x)|^2 for Clifford-only circuits from an
 *                     Aaronson-Gottesman stabilizer tableau
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static inline cplx gate(const double* u, int n, int t, int q, int r, int c) {
    const double* g = u + ((size_t)(t * n + q) * 4 + (size_t)(r * 2 + c)) * 2;
    return g[0] + I * g[1];
}

int tbo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the OpenMP thread count of later calls (t >= 1); returns the count. */
int tbo_set_num_threads(int t) {
#ifdef _OPENMP
    if (t >= 1) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Dense state vector. out: 2*2^n doubles (re, im), index bit q = qubit q.   */
/* ph: NULL (every entangler is CZ) or d*(n-1) phases, ph[l*(n-1) + i] the   */
/* angle of the controlled-phase gate on (i, i+1) in layer l.                */
/* ------------------------------------------------------------------------ */
int tbo_sv_state(int n, int d, const double* u, const double* ph, double* out) {
    if (n < 1 || n > 30 || d < 0) return -1;
    const int64_t N = (int64_t)1 << n;
    cplx* psi = (cplx*)calloc((size_t)N, sizeof(cplx));
    if (!psi) return -2;
    psi[0] = 1.0;
    for (int t = 0; t <= d; ++t) {
        for (int q = 0; q < n; ++q) {
            const cplx g00 = gate(u, n, t, q, 0, 0), g01 = gate(u, n, t, q, 0, 1);
            const cplx g10 = gate(u, n, t, q, 1, 0), g11 = gate(u, n, t, q, 1, 1);
            const int64_t m = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                if (i & m) continue;
                const cplx a = psi[i], b = psi[i | m];
                psi[i] = g00 * a + g01 * b;
                psi[i | m] = g10 * a + g11 * b;
            }
        }
        if (t == d) break;
        /* entangling layer t: phase -1 (CZ) or e^(i phi) when both qubits of a
           coupled pair are 1. */
        for (int i0 = t % 2; i0 + 1 < n; i0 += 2) {
            const int64_t m = ((int64_t)1 << i0) | ((int64_t)1 << (i0 + 1));
            const cplx w = ph ? cexp(I * ph[(size_t)t * (n - 1) + i0]) : -1.0;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i)
                if ((i & m) == m) psi[i] = ph ? w * psi[i] : -psi[i];
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        out[2 * i] = creal(psi[i]);
        out[2 * i + 1] = cimag(psi[i]);
    }
    free(psi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Naive boundary contraction.                                              */
/*                                                                          */
/* A dense tensor whose index bits carry labels: label l >= 0 is the value  */
/* s_{q,l} of a qubit during CZ layer l that still waits for its partner    */
/* row; label WIRE is the running time value of the row being absorbed.     */
/* ------------------------------------------------------------------------ */
#define WIRE (-1)
#define MAXB 40

typedef struct {
    cplx* a;
    int nbits;
    int label[MAXB];
} tens;

static int find_label(const tens* T, int lab) {
    for (int j = 0; j < T->nbits; ++j)
        if (T->label[j] == lab) return j;
    return -1;
}

/* Insert bit value v at position j of index i' (bits >= j move up). */
static inline int64_t ins_bit(int64_t ip, int j, int v) {
    const int64_t lo = ip & (((int64_t)1 << j) - 1);
    const int64_t hi = ip >> j;
    return lo | ((int64_t)v << j) | (hi << (j + 1));
}

/* New top index (the wire) with weight v[w]. */
static int add_wire(tens* T, const cplx v[2]) {
    const int64_t N = (int64_t)1 << T->nbits;
    cplx* b = (cplx*)malloc((size_t)(2 * N) * sizeof(cplx));
    if (!b) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        b[i] = T->a[i] * v[0];
        b[i + N] = T->a[i] * v[1];
    }
    free(T->a);
    T->a = b;
    T->label[T->nbits++] = WIRE;
    return 0;
}

/* CZ between the stored bit with label lab and the wire, then sum the
 * stored bit out: b[i'] = sum_s a[i'(s)] * (-1)^(s * wire). */
static int consume(tens* T, int lab) {
    const int j = find_label(T, lab);
    if (j < 0) return -3;
    const int64_t No = (int64_t)1 << (T->nbits - 1);
    cplx* b = (cplx*)malloc((size_t)No * sizeof(cplx));
    if (!b) return -2;
    const int w = find_label(T, WIRE);
#pragma omp parallel for schedule(static)
    for (int64_t ip = 0; ip < No; ++ip) {
        const int64_t i0 = ins_bit(ip, j, 0), i1 = ins_bit(ip, j, 1);
        const int wire = (int)((i1 >> w) & 1);
        b[ip] = T->a[i0] + (wire ? -T->a[i1] : T->a[i1]);
    }
    free(T->a);
    T->a = b;
    for (int k = j; k + 1 < T->nbits; ++k) T->label[k] = T->label[k + 1];
    T->nbits--;
    return 0;
}

/* Copy the wire into a new stored index labelled lab (the CZ half on the
 * creating side is the projector |a><a|). */
static int create(tens* T, int lab) {
    const int64_t N = (int64_t)1 << T->nbits;
    cplx* b = (cplx*)malloc((size_t)(2 * N) * sizeof(cplx));
    if (!b) return -2;
    const int w = find_label(T, WIRE);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const int wire = (int)((i >> w) & 1);
        b[i] = wire ? 0.0 : T->a[i];
        b[i + N] = wire ? T->a[i] : 0.0;
    }
    free(T->a);
    T->a = b;
    T->label[T->nbits++] = lab;
    return 0;
}

/* Apply a one-qubit gate to the wire: b[.., w'] = sum_w g[w'][w] a[.., w]. */
static void apply_wire(tens* T, cplx g00, cplx g01, cplx g10, cplx g11) {
    const int w = find_label(T, WIRE);
    const int64_t m = (int64_t)1 << w;
    const int64_t N = (int64_t)1 << T->nbits;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if (i & m) continue;
        const cplx a0 = T->a[i], a1 = T->a[i | m];
        T->a[i] = g00 * a0 + g01 * a1;
        T->a[i | m] = g10 * a0 + g11 * a1;
    }
}

/* Close the wire with the output projector <x_q|. */
static int project_wire(tens* T, int xq) {
    const int w = find_label(T, WIRE);
    const int64_t No = (int64_t)1 << (T->nbits - 1);
    cplx* b = (cplx*)malloc((size_t)No * sizeof(cplx));
    if (!b) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t ip = 0; ip < No; ++ip) b[ip] = T->a[ins_bit(ip, w, xq)];
    free(T->a);
    T->a = b;
    for (int k = w; k + 1 < T->nbits; ++k) T->label[k] = T->label[k + 1];
    T->nbits--;
    return 0;
}

/* Qubit q takes part in a CZ of layer l with qubit q+1 iff q = l (mod 2). */
static inline int couples_up(int q, int l, int n) { return q + 1 < n && (q % 2) == (l % 2); }

int tbo_nb_amplitude(int n, int d, const double* u, const uint8_t* x, double* out,
                     int* max_bits) {
    if (n < 1 || d < 0) return -1;
    tens T;
    T.a = (cplx*)malloc(sizeof(cplx));
    if (!T.a) return -2;
    T.a[0] = 1.0;
    T.nbits = 0;
    int peak = 0;
    int rc = 0;
    for (int q = 0; q < n && rc == 0; ++q) {
        /* |0> through slot 0. */
        const cplx v[2] = {gate(u, n, 0, q, 0, 0), gate(u, n, 0, q, 1, 0)};
        if ((rc = add_wire(&T, v))) break;
        for (int l = 0; l < d && rc == 0; ++l) {
            if (q > 0 && couples_up(q - 1, l, n)) rc = consume(&T, l);
            if (rc) break;
            if (couples_up(q, l, n)) rc = create(&T, l);
            if (rc) break;
            if (T.nbits > peak) peak = T.nbits;
            if (T.nbits >= MAXB - 1) { rc = -4; break; }
            apply_wire(&T, gate(u, n, l + 1, q, 0, 0), gate(u, n, l + 1, q, 0, 1),
                       gate(u, n, l + 1, q, 1, 0), gate(u, n, l + 1, q, 1, 1));
        }
        if (rc) break;
        if (d == 0) { /* no layer: the wire only sees slot 0 */ }
        rc = project_wire(&T, x[q]);
    }
    if (rc == 0 && T.nbits != 0) rc = -5;
    if (rc == 0) {
        out[0] = creal(T.a[0]);
        out[1] = cimag(T.a[0]);
        if (max_bits) *max_bits = peak;
    }
    free(T.a);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Brute force: sum over all s_{q,l} (q < n, l < d) of the product of gate  */
/* entries along each qubit's time line times the CZ signs.                 */
/* ------------------------------------------------------------------------ */
int tbo_feynman(int n, int d, const double* u, const uint8_t* x, double* out) {
    const int nv = n * d;
    if (n < 1 || d < 0 || nv > 26) return -1;
    const int64_t NS = (int64_t)1 << nv;
    double sre = 0.0, sim = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sre, sim)
    for (int64_t s = 0; s < NS; ++s) {
        /* s_{q,l} = bit (q*d + l) of s */
        cplx amp = 1.0;
        for (int q = 0; q < n; ++q) {
            int prev = 0; /* input |0> */
            for (int t = 0; t < d; ++t) {
                const int cur = (int)((s >> (q * d + t)) & 1);
                amp *= gate(u, n, t, q, cur, prev);
                prev = cur;
            }
            amp *= gate(u, n, d, q, x[q], prev);
        }
        int sign = 0;
        for (int l = 0; l < d; ++l)
            for (int i0 = l % 2; i0 + 1 < n; i0 += 2)
                sign ^= (int)(((s >> (i0 * d + l)) & 1) & ((s >> ((i0 + 1) * d + l)) & 1));
        if (sign) amp = -amp;
        sre += creal(amp);
        sim += cimag(amp);
    }
    out[0] = sre;
    out[1] = sim;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Stabilizer tableau (Aaronson & Gottesman 2004): rows 0..n-1 destabilizers, */
/* n..2n-1 stabilizers, row 2n scratch. Clifford-only circuits.              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    uint8_t* x; /* (2n+1) * n */
    uint8_t* z;
    uint8_t* r; /* 2n+1 */
} tableau;

#define TX(T, i, j) ((T)->x[(size_t)(i) * (T)->n + (j)])
#define TZ(T, i, j) ((T)->z[(size_t)(i) * (T)->n + (j)])

static void tab_h(tableau* T, int a) {
    for (int i = 0; i < 2 * T->n; ++i) {
        T->r[i] ^= TX(T, i, a) & TZ(T, i, a);
        const uint8_t t = TX(T, i, a);
        TX(T, i, a) = TZ(T, i, a);
        TZ(T, i, a) = t;
    }
}

static void tab_s(tableau* T, int a) {
    for (int i = 0; i < 2 * T->n; ++i) {
        T->r[i] ^= TX(T, i, a) & TZ(T, i, a);
        TZ(T, i, a) ^= TX(T, i, a);
    }
}

static void tab_cnot(tableau* T, int a, int b) {
    for (int i = 0; i < 2 * T->n; ++i) {
        T->r[i] ^= TX(T, i, a) & TZ(T, i, b) & (TX(T, i, b) ^ TZ(T, i, a) ^ 1);
        TX(T, i, b) ^= TX(T, i, a);
        TZ(T, i, a) ^= TZ(T, i, b);
    }
}

/* Exponent of i picked up when Pauli (x1,z1) multiplies (x2,z2). */
static int g_exp(int x1, int z1, int x2, int z2) {
    if (!x1 && !z1) return 0;
    if (x1 && z1) return z2 - x2;
    if (x1 && !z1) return z2 * (2 * x2 - 1);
    return x2 * (1 - 2 * z2);
}

/* row h <- row i * row h */
static void rowsum(tableau* T, int h, int i) {
    int e = 2 * T->r[h] + 2 * T->r[i];
    for (int j = 0; j < T->n; ++j) e += g_exp(TX(T, i, j), TZ(T, i, j), TX(T, h, j), TZ(T, h, j));
    e = ((e % 4) + 4) % 4;
    T->r[h] = (uint8_t)(e == 2);
    for (int j = 0; j < T->n; ++j) {
        TX(T, h, j) ^= TX(T, i, j);
        TZ(T, h, j) ^= TZ(T, i, j);
    }
}

/* Z measurement of qubit a forced to outcome o; returns its probability. */
static double tab_measure(tableau* T, int a, int o) {
    const int n = T->n;
    int p = -1;
    for (int i = n; i < 2 * n; ++i)
        if (TX(T, i, a)) { p = i; break; }
    if (p >= 0) {
        for (int i = 0; i < 2 * n; ++i)
            if (i != p && TX(T, i, a)) rowsum(T, i, p);
        memcpy(&TX(T, p - n, 0), &TX(T, p, 0), (size_t)n);
        memcpy(&TZ(T, p - n, 0), &TZ(T, p, 0), (size_t)n);
        T->r[p - n] = T->r[p];
        memset(&TX(T, p, 0), 0, (size_t)n);
        memset(&TZ(T, p, 0), 0, (size_t)n);
        TZ(T, p, a) = 1;
        T->r[p] = (uint8_t)o;
        return 0.5;
    }
    const int s = 2 * n;
    memset(&TX(T, s, 0), 0, (size_t)n);
    memset(&TZ(T, s, 0), 0, (size_t)n);
    T->r[s] = 0;
    for (int i = 0; i < n; ++i)
        if (TX(T, i, a)) rowsum(T, s, i + n);
    return (T->r[s] == o) ? 1.0 : 0.0;
}

/* The Clifford C_k = P_(k mod 4) . R_(k div 4) as a time-ordered list of H
 * (code 0) and S (code 1), up to a global phase. R in (I, H, S, S.H, H.S,
 * H.S.H), P in (I, X, Y, Z) with X = H S S H, Z = S S and Y ~ X.Z. */
static int clifford_seq(int k, int* seq) {
    static const int R[6][3] = {{-1}, {0, -1}, {1, -1}, {0, 1, -1}, {1, 0, -1}, {0, 1, 0}};
    static const int Rlen[6] = {0, 1, 1, 2, 2, 3};
    static const int P[4][6] = {{-1}, {0, 1, 1, 0}, {1, 1, 0, 1, 1, 0}, {1, 1}};
    static const int Plen[4] = {0, 4, 6, 2};
    int len = 0;
    const int r = k / 4, p = k % 4;
    for (int i = 0; i < Rlen[r]; ++i) seq[len++] = R[r][i];
    for (int i = 0; i < Plen[p]; ++i) seq[len++] = P[p][i];
    return len;
}

/* |<x|U|0^n>|^2 for a circuit whose slots hold only Cliffords cliff[t*n+q]
 * (0..23) and whose CZ layers follow the brickwork rule. */
int tbo_tableau_prob(int n, int d, const uint8_t* cliff, const uint8_t* x, double* prob) {
    if (n < 1 || d < 0) return -1;
    tableau T;
    T.n = n;
    T.x = (uint8_t*)calloc((size_t)(2 * n + 1) * n, 1);
    T.z = (uint8_t*)calloc((size_t)(2 * n + 1) * n, 1);
    T.r = (uint8_t*)calloc((size_t)(2 * n + 1), 1);
    if (!T.x || !T.z || !T.r) return -2;
    for (int i = 0; i < n; ++i) {
        TX(&T, i, i) = 1;
        TZ(&T, i + n, i) = 1;
    }
    int seq[16];
    for (int t = 0; t <= d; ++t) {
        for (int q = 0; q < n; ++q) {
            const int k = cliff[(size_t)t * n + q];
            if (k > 23) { free(T.x); free(T.z); free(T.r); return -1; }
            const int len = clifford_seq(k, seq);
            for (int i = 0; i < len; ++i) {
                if (seq[i] == 0) tab_h(&T, q);
                else tab_s(&T, q);
            }
        }
        if (t == d) break;
        for (int i0 = t % 2; i0 + 1 < n; i0 += 2) { /* CZ = H_b CNOT_ab H_b */
            tab_h(&T, i0 + 1);
            tab_cnot(&T, i0, i0 + 1);
            tab_h(&T, i0 + 1);
        }
    }
    double p = 1.0;
    for (int q = 0; q < n && p > 0.0; ++q) p *= tab_measure(&T, q, x[q]);
    *prob = p;
    free(T.x);
    free(T.z);
    free(T.r);
    return 0;
}
