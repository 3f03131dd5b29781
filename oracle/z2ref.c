/*
 * z2ref.c -- FP64 CPU reference ("oracle") for the digital adiabatic
 * simulation of quantum Z2 lattice gauge theory (Cui, Shi, Yang,
 * arXiv:1910.08020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source, header, table or helper with
 * the CUDA path.
 *
 * The state vector is 2^n complex amplitudes stored as interleaved doubles
 * (re, im).  Qubit l is bit l of the amplitude index (bit 0 least
 * significant); sigma^z|0> = |0>, sigma^z|1> = -|1> (Sec. 2.1).
 *
 * Everything is written as the plain definition, one operator at a time, with
 * no fusion: the only concession to speed is an OpenMP loop over amplitudes.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static int parity64(uint64_t x) { return __builtin_popcountll(x) & 1; }

/* sum_p u_p(i), with u_p(i) = prod_{l in p} sigma^z_l evaluated on basis
 * state |i> = (-1)^{popcount(i & m_p)}  (U_p = -Z_box, Sec. 2.1). */
static double plaquette_sum(uint64_t i, int n_plaq, const uint64_t *masks) {
    double s = 0.0;
    for (int p = 0; p < n_plaq; ++p) s += parity64(i & masks[p]) ? -1.0 : 1.0;
    return s;
}

/* |+>^n: every amplitude 2^{-n/2} (Sec. 2.3, the "ground state of X" start). */
void z2ref_init_plus(int n, double *psi_) {
    cplx *psi = (cplx *)psi_;
    const uint64_t dim = 1ull << n;
    const double a = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; ++i) psi[i] = a;
}

/* D(theta) = exp(i theta sum_p U_p): the diagonal plaquette layer.  For the
 * Hamiltonian H(s) = -sum_l sigma^x_l - s*lambda*sum_p U_p the plaquette part of
 * exp(-i H dt) is D(s*lambda*dt).  Per plaquette this is the phase produced by
 * the ancilla circuit of Eq. (ara) (Sec. 2.2). */
void z2ref_apply_D(int n, double *psi_, int n_plaq, const uint64_t *masks, double theta) {
    cplx *psi = (cplx *)psi_;
    const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; ++i) {
        double ph = theta * plaquette_sum((uint64_t)i, n_plaq, masks);
        psi[i] *= cexp(I * ph);
    }
}

/* One single-qubit gate exp(+i dt sigma^x) on qubit l:
 *   (a, b) -> (cos dt a + i sin dt b, i sin dt a + cos dt b)
 * for each pair (i, i | 2^l) with bit l of i clear.  This is the transverse
 * field factor exp(-i dt (-sigma^x_l)) = R_x(-2 dt) (Sec. 2.2). */
void z2ref_apply_rx_qubit(int n, double *psi_, int l, double dt) {
    cplx *psi = (cplx *)psi_;
    const uint64_t dim = 1ull << n, bit = 1ull << l;
    const double c = cos(dt), s = sin(dt);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; ++i) {
        if ((uint64_t)i & bit) continue;
        cplx a = psi[i], b = psi[(uint64_t)i | bit];
        psi[i] = c * a + I * s * b;
        psi[(uint64_t)i | bit] = I * s * a + c * b;
    }
}

/* R(dt) = prod_l exp(i dt sigma^x_l): the whole transverse-field layer. */
void z2ref_apply_R(int n, double *psi, double dt) {
    for (int l = 0; l < n; ++l) z2ref_apply_rx_qubit(n, psi, l, dt);
}

/* Hadamard on every qubit (used to measure sigma^x-type quantities as
 * H sigma^z H, Sec. 2.4). */
void z2ref_apply_hadamard_all(int n, double *psi_) {
    cplx *psi = (cplx *)psi_;
    const uint64_t dim = 1ull << n;
    const double r = 1.0 / sqrt(2.0);
    for (int l = 0; l < n; ++l) {
        const uint64_t bit = 1ull << l;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)dim; ++i) {
            if ((uint64_t)i & bit) continue;
            cplx a = psi[i], b = psi[(uint64_t)i | bit];
            psi[i] = r * (a + b);
            psi[(uint64_t)i | bit] = r * (a - b);
        }
    }
}

/* Schedule: dt = T/M and s_j = j/M on the grid j = 0..M (H(s) ramps s from 0
 * to 1).  decomp 0 = first order, 1 = symmetric.  sampling 0 = standard,
 * 1 = the paper's literal right-endpoint rule for both symmetric halves.
 *
 *   first order, step j:   psi <- R(dt) D(lambda s_j dt) psi
 *       (the varying-coefficient factor acts first and is sampled at the
 *        right end of the step, mirroring Eq. (a) with g_{k,m} of Sec. 2.2)
 *   symmetric, step j:     psi <- D(lambda s_j dt/2) R(dt) D(lambda s_{j-1} dt/2) psi
 *       (trapezoid split of Eq. (s); with sampling = 1 both halves use s_j)
 *
 * Steps j0+1 .. j1 are applied (j0 = 0, j1 = M for a whole run), so a run can
 * be cut into segments.  Returns 0, or -1 on bad arguments. */
int z2ref_evolve(int n, double *psi, int n_plaq, const uint64_t *masks, double lambda,
                 double T, int M, int decomp, int sampling, int j0, int j1) {
    if (M <= 0 || j0 < 0 || j1 > M || j0 > j1) return -1;
    if (decomp != 0 && decomp != 1) return -1;
    const double dt = T / (double)M;
    for (int j = j0 + 1; j <= j1; ++j) {
        const double s_j = (double)j / (double)M;
        const double s_jm1 = (double)(j - 1) / (double)M;
        if (decomp == 0) {
            z2ref_apply_D(n, psi, n_plaq, masks, lambda * s_j * dt);
            z2ref_apply_R(n, psi, dt);
        } else {
            const double s_first = sampling ? s_j : s_jm1;
            z2ref_apply_D(n, psi, n_plaq, masks, lambda * s_first * dt / 2.0);
            z2ref_apply_R(n, psi, dt);
            z2ref_apply_D(n, psi, n_plaq, masks, lambda * s_j * dt / 2.0);
        }
    }
    return 0;
}

/* out[k] = sum_i |psi_i|^2 (-1)^{popcount(i & masks[k])}
 *        = <prod_{l in mask} sigma^z_l>  (Wilson loops, plaquettes, sigma^z_l;
 *          a zero mask gives the norm).  Sec. 2.4. */
void z2ref_zsums(int n, const double *psi_, int n_masks, const uint64_t *masks, double *out) {
    const cplx *psi = (const cplx *)psi_;
    const uint64_t dim = 1ull << n;
    for (int k = 0; k < n_masks; ++k) {
        double acc = 0.0;
        const uint64_t m = masks[k];
#pragma omp parallel for reduction(+ : acc) schedule(static)
        for (int64_t i = 0; i < (int64_t)dim; ++i) {
            double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            acc += parity64((uint64_t)i & m) ? -p : p;
        }
        out[k] = acc;
    }
}

/* out[2k], out[2k+1] = Re, Im of <psi| prod_{l in mask} sigma^x_l |psi>
 *   = sum_i conj(psi_{i ^ mask}) psi_i   (sigma^x flips bit l).
 * Gauss-law stars G_i, 't Hooft loops V_mu and sigma^x_l.  Sec. 2.1, 2.4. */
void z2ref_xsums(int n, const double *psi_, int n_masks, const uint64_t *masks, double *out) {
    const cplx *psi = (const cplx *)psi_;
    const uint64_t dim = 1ull << n;
    for (int k = 0; k < n_masks; ++k) {
        double re = 0.0, im = 0.0;
        const uint64_t m = masks[k];
#pragma omp parallel for reduction(+ : re, im) schedule(static)
        for (int64_t i = 0; i < (int64_t)dim; ++i) {
            cplx t = conj(psi[(uint64_t)i ^ m]) * psi[i];
            re += creal(t);
            im += cimag(t);
        }
        out[2 * k] = re;
        out[2 * k + 1] = im;
    }
}

/* Z density of states: out[k] = sum of |psi_i|^2 over basis states with
 * exactly k plaquettes of odd parity (U_p = -1), k = 0..n_plaq.  Sec. 3.3. */
void z2ref_zdos(int n, const double *psi_, int n_plaq, const uint64_t *masks, double *out) {
    const cplx *psi = (const cplx *)psi_;
    const uint64_t dim = 1ull << n;
    for (int k = 0; k <= n_plaq; ++k) out[k] = 0.0;
    for (uint64_t i = 0; i < dim; ++i) {
        int odd = 0;
        for (int p = 0; p < n_plaq; ++p) odd += parity64(i & masks[p]);
        out[odd] += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    }
}

/* <a|b> = sum_i conj(a_i) b_i, written to out[0] (re), out[1] (im). */
void z2ref_overlap(int n, const double *a_, const double *b_, double *out) {
    const cplx *a = (const cplx *)a_, *b = (const cplx *)b_;
    const uint64_t dim = 1ull << n;
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; ++i) {
        cplx t = conj(a[i]) * b[i];
        re += creal(t);
        im += cimag(t);
    }
    out[0] = re;
    out[1] = im;
}

/* y = H(s) x with H(s) = -sum_l sigma^x_l - s*lambda*sum_p U_p, the form of the
 * Hamiltonian ramped here (the "X + K Z" start of Sec. 2.3 with K = s*lambda).
 * Used by the Lanczos ground-state solver. */
void z2ref_hamiltonian_apply(int n, const double *x_, double *y_, int n_plaq, const uint64_t *masks,
                             double s_lambda) {
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; ++i) {
        cplx acc = -s_lambda * plaquette_sum((uint64_t)i, n_plaq, masks) * x[i];
        for (int l = 0; l < n; ++l) acc -= x[(uint64_t)i ^ (1ull << l)];
        y[i] = acc;
    }
}
