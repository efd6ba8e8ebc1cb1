/*
 * Oracle: full state-vector simulation in complex128.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the independent CPU oracle
 * that checks the CUDA path.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does.
 *
 * What it computes (Sec. II, the state-vector picture): the circuit's output
 * state is obtained by storing the 2^n amplitudes of the initial state |0...0>
 * and applying each gate's unitary in circuit order; an amplitude <x|C|0> is
 * then read from that vector.  The tensor-network contraction of the same
 * circuit with the outputs closed by <x_q| reaches exactly this value (up to
 * rounding order), which is why it is the reference result.
 *
 * Conventions: qubit 0 is the most significant bit of the state index; a
 * two-qubit gate matrix is row-major in the basis |q0 q1> (row = 2*b(q0)+b(q1)).
 *
 * Parity pins: GHZ and product-state closed forms, unitarity of the evolved
 * state, agreement with the independent plan einsum (tests/test_oracle.py).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nq;
    int32_t q[2];
    int32_t pad;
    double re[16];
    double im[16];
} qxo_gate;

static double complex entry(const qxo_gate* g, int r, int c, int dim) {
    return g->re[r * dim + c] + I * g->im[r * dim + c];
}

/* Apply one gate in place.  p0/p1 are bit positions (n-1-q). */
static void apply_gate(int n, const qxo_gate* g, double complex* psi) {
    const int64_t N = (int64_t)1 << n;
    if (g->nq == 1) {
        const int64_t m = (int64_t)1 << (n - 1 - g->q[0]);
        const double complex u00 = entry(g, 0, 0, 2), u01 = entry(g, 0, 1, 2);
        const double complex u10 = entry(g, 1, 0, 2), u11 = entry(g, 1, 1, 2);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (i & m) continue;
            const double complex a0 = psi[i], a1 = psi[i | m];
            psi[i] = u00 * a0 + u01 * a1;
            psi[i | m] = u10 * a0 + u11 * a1;
        }
    } else {
        const int64_t m0 = (int64_t)1 << (n - 1 - g->q[0]);
        const int64_t m1 = (int64_t)1 << (n - 1 - g->q[1]);
        double complex u[4][4];
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) u[r][c] = entry(g, r, c, 4);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (i & (m0 | m1)) continue;
            const int64_t idx[4] = {i, i | m1, i | m0, i | m0 | m1}; /* |00>,|01>,|10>,|11> */
            double complex a[4], b[4];
            for (int c = 0; c < 4; ++c) a[c] = psi[idx[c]];
            for (int r = 0; r < 4; ++r) {
                b[r] = 0;
                for (int c = 0; c < 4; ++c) b[r] += u[r][c] * a[c];
            }
            for (int r = 0; r < 4; ++r) psi[idx[r]] = b[r];
        }
    }
}

/* Evolve |0...0> through the gates.  psi must hold 2^n complex128 values
 * (interleaved re, im).  Returns 0, or -1 on a malformed gate. */
int qxo_sv_evolve(int n, const qxo_gate* gates, int64_t n_gates, double* psi_out) {
    if (n < 1 || n > 34) return -1;
    for (int64_t k = 0; k < n_gates; ++k) {
        const qxo_gate* g = &gates[k];
        if (g->nq != 1 && g->nq != 2) return -1;
        for (int j = 0; j < g->nq; ++j)
            if (g->q[j] < 0 || g->q[j] >= n) return -1;
        if (g->nq == 2 && g->q[0] == g->q[1]) return -1;
    }
    double complex* psi = (double complex*)psi_out;
    const int64_t N = (int64_t)1 << n;
    memset(psi, 0, sizeof(double complex) * (size_t)N);
    psi[0] = 1.0;
    for (int64_t k = 0; k < n_gates; ++k) apply_gate(n, &gates[k], psi);
    return 0;
}

/* Read amplitudes from an evolved state.  For each bitstring b (n bytes of 0/1)
 * and each assignment o of the open qubits (open_mask[q] = 1; first open qubit is
 * the most significant bit of o), out[b][o] = psi[index].  out holds
 * n_bits * 2^n_open complex128 values. */
int qxo_sv_read(int n, const double* psi_in, const uint8_t* open_mask, const uint8_t* bits,
                int64_t n_bits, double* out) {
    const double complex* psi = (const double complex*)psi_in;
    double complex* amps = (double complex*)out;
    int open_q[64];
    int n_open = 0;
    for (int q = 0; q < n; ++q)
        if (open_mask && open_mask[q]) open_q[n_open++] = q;
    const int64_t n_o = (int64_t)1 << n_open;
    for (int64_t b = 0; b < n_bits; ++b) {
        int64_t base = 0;
        for (int q = 0; q < n; ++q) {
            const uint8_t v = bits[b * n + q];
            if (v > 1) return -1;
            if (!(open_mask && open_mask[q]) && v) base |= (int64_t)1 << (n - 1 - q);
        }
        for (int64_t o = 0; o < n_o; ++o) {
            int64_t idx = base;
            for (int j = 0; j < n_open; ++j)
                if ((o >> (n_open - 1 - j)) & 1) idx |= (int64_t)1 << (n - 1 - open_q[j]);
            amps[b * n_o + o] = psi[idx];
        }
    }
    return 0;
}
