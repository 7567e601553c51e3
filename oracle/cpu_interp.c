/*
 * cpu_interp.c -- TEST INFRASTRUCTURE ONLY (a timed CPU comparison).
 *
 * The CPU scheme the paper's radiation-transfer code runs in production
 * (Section 6, and the "CPU (interpolation)" column of Table 1): the
 * temperature comes from a per-grain table of 2000 temperatures between 3 K
 * and 1500 K, interpolated linearly, instead of from a root solve; the
 * heating power before it (Eq. 6) and the emission SED after it (Eqs. 8-10)
 * are computed in full.  It is not the parity oracle (dust_oracle.c is):
 * the benchmark times it on the host cores beside the GPU path, and the
 * tests bound its error against the oracle.  It shares no code with the
 * oracle or with the CUDA library; only the tests and the benchmark's CPU
 * leg load it.
 *
 * Readings where the paper is silent:
 *   - the table's temperatures are spaced uniformly in ln T (T_j = T_lo
 *     (T_hi / T_lo)^(j / (NT - 1))), so its relative resolution is the same
 *     at 3 K as at 1500 K;
 *   - "linear interpolation" is linear in (P, T) between the two nodes whose
 *     emitted powers bracket the absorbed power A (P_g(T) rises with T, so a
 *     binary search finds them);
 *   - A below the first node's power gives T_lo (flag 1), above the last
 *     node's T_hi (flag 2), A = 0 flag 1, a negative or non-finite A NaN
 *     (flag 4): the oracle's flag convention;
 *   - FP64 throughout, one OpenMP thread per cell in turn.
 *
 * Build: part of libdust_oracle.so (see build.py).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CI_H 6.62607015e-34   /* Planck constant [J s]       */
#define CI_C 299792458.0      /* speed of light [m s^-1]     */
#define CI_K 1.380649e-23     /* Boltzmann constant [J K^-1] */
#define CI_PI 3.14159265358979323846

/* Per-wavelength constants of B(lambda, T) = b_k / (exp(x_k / T) - 1) with
 * b_k = 2 h c^2 lambda_k^-5 and x_k = h c / (k lambda_k)  (Eq. 1). */
static void planck_consts(int K, const double *lambda, double *b, double *x)
{
    for (int k = 0; k < K; ++k) {
        const double l = lambda[k];
        b[k] = 2.0 * CI_H * CI_C * CI_C / (l * l * l * l * l);
        x[k] = CI_H * CI_C / (CI_K * l);
    }
}

static double planck_k(double b, double x, double T)
{
    return b / expm1(x / T);
}

/* The table: T_nodes [NT] and P [G][NT], P[g][j] = sum_k w_k C[g,k]
 * B(lambda_k, T_j)  (Eq. 7 at the nodes).  Returns 0, or -1 on bad sizes. */
int dust_interp_table(int K, const double *lambda, const double *w, int G, const double *C,
                      double T_lo, double T_hi, int NT, double *T_nodes, double *P)
{
    if (K < 1 || G < 1 || NT < 2 || !(T_lo > 0.0) || !(T_hi > T_lo)) return -1;
    double *b = malloc(sizeof(double) * (size_t)K), *x = malloc(sizeof(double) * (size_t)K);
    if (!b || !x) { free(b); free(x); return -1; }
    planck_consts(K, lambda, b, x);
    const double r = log(T_hi / T_lo) / (double)(NT - 1);
    for (int j = 0; j < NT; ++j)
        T_nodes[j] = (j == NT - 1) ? T_hi : T_lo * exp(r * (double)j);
#pragma omp parallel for schedule(static)
    for (int g = 0; g < G; ++g) {
        const double *Cg = C + (size_t)g * K;
        for (int j = 0; j < NT; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k)
                s += w[k] * Cg[k] * planck_k(b[k], x[k], T_nodes[j]);
            P[(size_t)g * NT + j] = s;
        }
    }
    free(b);
    free(x);
    return 0;
}

/* Temperature of one grain for absorbed power A from its table row Pg;
 * returns the flag. */
static int interp_T(int NT, const double *T_nodes, const double *Pg, double A, double *T)
{
    if (!(A >= 0.0) || isinf(A)) { *T = NAN; return 4; }
    if (A < Pg[0] || A == 0.0) { *T = T_nodes[0]; return 1; }
    if (A > Pg[NT - 1]) { *T = T_nodes[NT - 1]; return 2; }
    int lo = 0, hi = NT - 1;  /* Pg[lo] <= A <= Pg[hi] */
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Pg[mid] <= A) lo = mid; else hi = mid;
    }
    const double f = (A - Pg[lo]) / (Pg[hi] - Pg[lo]);
    *T = T_nodes[lo] + f * (T_nodes[hi] - T_nodes[lo]);
    return 0;
}

/* The scheme over n_cells cells: J [n_cells][K], n [n_cells][G] row-major
 * FP64; the table from dust_interp_table.  Per cell: A_g = sum_k w_k C[g,k]
 * J_k (Eq. 6), T_g from the table, L_k = 4 pi sum_g n_g C[g,k]
 * B(lambda_k, T_g) (Eqs. 8-10).  Outputs T [n_cells][G], L [n_cells][K]
 * (or NULL) and flags [n_cells][G] (or NULL).  n_threads <= 0 uses the
 * OpenMP default.  Returns 0, or -1 when scratch cannot be allocated. */
int dust_interp_run(int64_t n_cells, int K, int G, const double *lambda, const double *w,
                    const double *C, const double *J, const double *n, int NT,
                    const double *T_nodes, const double *P, double *T_out, double *L_out,
                    uint8_t *flags_out, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    double *b = malloc(sizeof(double) * (size_t)K), *x = malloc(sizeof(double) * (size_t)K);
    double *W = malloc(sizeof(double) * (size_t)G * K);
    if (!b || !x || !W) { free(b); free(x); free(W); return -1; }
    planck_consts(K, lambda, b, x);
    for (int g = 0; g < G; ++g)
        for (int k = 0; k < K; ++k)
            W[(size_t)g * K + k] = w[k] * C[(size_t)g * K + k];
#pragma omp parallel for schedule(dynamic, 32)
    for (int64_t c = 0; c < n_cells; ++c) {
        const double *Jc = J + c * (int64_t)K;
        const double *nc = n + c * (int64_t)G;
        double *Tc = T_out + c * (int64_t)G;
        for (int g = 0; g < G; ++g) {
            const double *Wg = W + (size_t)g * K;
            double A = 0.0;
            for (int k = 0; k < K; ++k)
                A += Wg[k] * Jc[k];
            const int fl = interp_T(NT, T_nodes, P + (size_t)g * NT, A, &Tc[g]);
            if (flags_out) flags_out[c * (int64_t)G + g] = (uint8_t)fl;
        }
        if (L_out) {
            double *Lc = L_out + c * (int64_t)K;
            for (int k = 0; k < K; ++k) Lc[k] = 0.0;
            for (int g = 0; g < G; ++g) {
                const double *Cg = C + (size_t)g * K;
                const double ng = nc[g], Tg = Tc[g];
                for (int k = 0; k < K; ++k)
                    Lc[k] += ng * Cg[k] * planck_k(b[k], x[k], Tg);
            }
            for (int k = 0; k < K; ++k) Lc[k] *= 4.0 * CI_PI;
        }
    }
    free(b);
    free(x);
    free(W);
    return 0;
}
