/*
 * qsim_oracle.c -- plain, slow, FP64 CPU oracle for the state-vector simulator.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the bench's CPU-baseline
 * leg may load this library. It shares no code with the CUDA path.
 *
 * Every routine is the paper's definition written out as plain loops over the
 * full index range, in double-precision complex arithmetic:
 *
 *  - oracle_apply_matrix: the basic-gate update of Sec. 4.3.2, Eq. (update_mat):
 *    for every x0 in B(0) (all target bits zero) gather the 2^m amplitudes
 *    psi[x0 + s(w)], multiply by the gate matrix K~ (row z = output, column w =
 *    input; bit j of the local index <-> targets[j]), scatter back. Controlled
 *    gates (Sec. 4.3.2, "controlled quantum gates") skip every x0 whose control
 *    bits differ from the control value, i.e. L_{x,x} = I off the control block.
 *  - oracle_apply_diagonal: the diagonal-matrix gate, psi_x <- d_{r(x)} psi_x.
 *  - oracle_apply_pauli: P|y> for a Pauli string (Pauli matrices of Sec. 4.3.2).
 *  - oracle_pauli_expectation: sum_y conj(psi_y) (P psi)_y for each term of an
 *    observable O = sum_P alpha_P P (Sec. 4.5), weighted sum returned.
 *  - oracle_inner / oracle_norm2: <a|b> and <psi|psi> (Sec. 4.2.2).
 *
 * The only parallelism is an optional OpenMP loop over x0 (the paper's own
 * scheme, Sec. 5.3), used when the oracle is timed as a CPU baseline; the
 * result does not depend on the thread count.
 *
 * Return value of the apply routines: 0 on success, -1 on invalid arguments.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_MAX_M 10

static int bad_qubits(int n, int m, const int* targets, int mc, const int* controls) {
    uint64_t seen = 0;
    if (n < 1 || n > 40 || m < 0 || mc < 0) return 1;
    for (int j = 0; j < m; j++) {
        if (targets[j] < 0 || targets[j] >= n || (seen >> targets[j]) & 1) return 1;
        seen |= 1ULL << targets[j];
    }
    for (int j = 0; j < mc; j++) {
        if (controls[j] < 0 || controls[j] >= n || (seen >> controls[j]) & 1) return 1;
        seen |= 1ULL << controls[j];
    }
    return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
    return t;
#else
    return 1;
#endif
}

/* psi <- K psi, K acting on `targets` (m of them), only where controls[j] == cvals[j]. */
int oracle_apply_matrix(cplx* psi, int n, int m, const int* targets, const cplx* K,
                        int mc, const int* controls, const int* cvals) {
    if (m < 1 || m > ORACLE_MAX_M || bad_qubits(n, m, targets, mc, controls)) return -1;
    const uint64_t dim = 1ULL << m;
    uint64_t tmask = 0, cmask = 0, cval = 0;
    uint64_t s[1 << ORACLE_MAX_M];            /* s(w): local index -> bit string of B(1) */
    for (int j = 0; j < m; j++) tmask |= 1ULL << targets[j];
    for (int j = 0; j < mc; j++) {
        cmask |= 1ULL << controls[j];
        if (cvals[j]) cval |= 1ULL << controls[j];
    }
    for (uint64_t w = 0; w < dim; w++) {
        uint64_t b = 0;
        for (int j = 0; j < m; j++)
            if ((w >> j) & 1) b |= 1ULL << targets[j];
        s[w] = b;
    }
    const uint64_t N = 1ULL << n;
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; x++) {
        if (x & tmask) continue;                 /* x must lie in B(0) */
        if ((x & cmask) != cval) continue;       /* controlled: act only on block c */
        cplx in[1 << ORACLE_MAX_M];
        cplx out[1 << ORACLE_MAX_M];
        for (uint64_t w = 0; w < dim; w++) in[w] = psi[x + s[w]];
        for (uint64_t z = 0; z < dim; z++) {
            cplx acc = 0.0;
            for (uint64_t w = 0; w < dim; w++) acc += K[z * dim + w] * in[w];
            out[z] = acc;
        }
        for (uint64_t z = 0; z < dim; z++) psi[x + s[z]] = out[z];
    }
    return 0;
}

/* psi_x <- d[r(x)] psi_x where r(x) collects the target bits (bit j <- targets[j]). */
int oracle_apply_diagonal(cplx* psi, int n, int m, const int* targets, const cplx* d,
                          int mc, const int* controls, const int* cvals) {
    if (m < 1 || m > ORACLE_MAX_M || bad_qubits(n, m, targets, mc, controls)) return -1;
    uint64_t cmask = 0, cval = 0;
    for (int j = 0; j < mc; j++) {
        cmask |= 1ULL << controls[j];
        if (cvals[j]) cval |= 1ULL << controls[j];
    }
    const uint64_t N = 1ULL << n;
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < N; x++) {
        if ((x & cmask) != cval) continue;
        uint64_t r = 0;
        for (int j = 0; j < m; j++)
            if ((x >> targets[j]) & 1) r |= 1ULL << j;
        psi[x] *= d[r];
    }
    return 0;
}

static int popcount64(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; c++; }
    return c;
}

/* i^k for integer k */
static cplx ipow(int k) {
    switch (k & 3) {
        case 0: return 1.0;
        case 1: return I;
        case 2: return -1.0;
        default: return -I;
    }
}

/* P|y> = i^{#Y} (-1)^{popcount(y & z)} |y xor x> with x = X-or-Y positions,
 * z = Z-or-Y positions (Y = i X Z on one qubit, from the Pauli matrices).
 * out must not alias psi. */
void oracle_apply_pauli(const cplx* psi, cplx* out, int n, uint64_t xmask, uint64_t zmask) {
    const uint64_t N = 1ULL << n;
    const cplx ph = ipow(popcount64(xmask & zmask));
    for (uint64_t y = 0; y < N; y++) {
        double sgn = (popcount64(y & zmask) & 1) ? -1.0 : 1.0;
        out[y ^ xmask] = ph * sgn * psi[y];
    }
}

/* <psi|P|psi> for one Pauli string (complex; its imaginary part is zero for a Hermitian P). */
cplx oracle_pauli_term(const cplx* psi, int n, uint64_t xmask, uint64_t zmask) {
    const uint64_t N = 1ULL << n;
    const cplx ph = ipow(popcount64(xmask & zmask));
    cplx acc = 0.0;
    for (uint64_t y = 0; y < N; y++) {
        double sgn = (popcount64(y & zmask) & 1) ? -1.0 : 1.0;
        /* (P psi)_{y xor x} = ph * sgn(y) * psi_y  ->  conj(psi_{y^x}) * that */
        acc += conj(psi[y ^ xmask]) * ph * sgn * psi[y];
    }
    return acc;
}

/* sum_k coef[k] <psi|P_k|psi>; real part returned, imaginary part in *imag_out (may be NULL). */
double oracle_pauli_expectation(const cplx* psi, int n, int nterms, const double* coef,
                                const uint64_t* xmask, const uint64_t* zmask, double* imag_out) {
    cplx e = 0.0;
    for (int k = 0; k < nterms; k++) e += coef[k] * oracle_pauli_term(psi, n, xmask[k], zmask[k]);
    if (imag_out) *imag_out = cimag(e);
    return creal(e);
}

/* <a|b> = sum_x conj(a_x) b_x, written to out[0] (re), out[1] (im). */
void oracle_inner(const cplx* a, const cplx* b, int n, double* out) {
    const uint64_t N = 1ULL << n;
    cplx acc = 0.0;
    for (uint64_t x = 0; x < N; x++) acc += conj(a[x]) * b[x];
    out[0] = creal(acc);
    out[1] = cimag(acc);
}

double oracle_norm2(const cplx* psi, int n) {
    const uint64_t N = 1ULL << n;
    double acc = 0.0;
    for (uint64_t x = 0; x < N; x++) acc += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    return acc;
}
