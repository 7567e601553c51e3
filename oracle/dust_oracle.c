/*
 * dust_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the dust equilibrium-temperature
 * and emission path of Jonsson & Primack, "Accelerating Dust Temperature
 * Calculations with Graphics Processing Units" (Eqs. 1-10).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline / reference leg may
 * load it.  The product path (the CUDA library) shares no code with it and
 * never calls it.
 *
 * It computes the plain definition of the discrete problem:
 *   A[c,g]  = sum_k w_k C[g,k] J[c,k]                              (Eq. 6)
 *   P_g(T)  = sum_k w_k C[g,k] B(lambda_k, T)                      (Eq. 7)
 *   T[c,g]  = the root of ln P_g(T) = ln A[c,g] in [T_min, T_max]   (Eqs. 1, 7)
 *   L[c,k]  = 4 pi sum_g n[c,g] C[g,k] B(lambda_k, T[c,g])         (Eqs. 8-10)
 *   r_c     = sum_k w_k L[c,k] / (4 pi sum_g n[c,g] Pe[c,g]) - 1
 * with Pe = A for grains solved inside the bracket and Pe = P_g(T_clamp) for
 * clamped grains (every grain emits the power of its temperature).
 *
 * The root is found with Brent's method (Brent 1973, "Algorithms for
 * Minimization without Derivatives", ch. 4) on F(u) = ln P_g(e^u) - ln A, to
 * an absolute tolerance of 1e-13 in u = ln T, with P_g evaluated by direct
 * quadrature at every step (no table).  The paper's own GPU kernel used
 * Newton-Raphson stopped at 0.1% energy non-conservation (Section 4.3); the
 * oracle needs the converged root of the same equation, not the iteration.
 *
 * Clamp flags: 0 solved; 1 clamped to T_min (A < P_g(T_min), including
 * A = 0); 2 clamped to T_max (A > P_g(T_max)); 4 invalid A (negative or not
 * finite; T = NaN).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <float.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* SI 2019 exact defining constants. */
#define ORC_H 6.62607015e-34   /* Planck constant [J s]      */
#define ORC_C 299792458.0      /* speed of light [m s^-1]    */
#define ORC_K 1.380649e-23     /* Boltzmann constant [J K^-1] */
#define ORC_PI 3.14159265358979323846

/* Planck function per unit wavelength, B(lambda, T) = 2 h c^2 lambda^-5 /
 * (exp(h c / (k lambda T)) - 1)  [W m^-2 m^-1 sr^-1]  (Eq. 1).
 * Written as e^-x / (1 - e^-x) with 1 - e^-x = -expm1(-x): exact in the
 * Rayleigh-Jeans limit and free of overflow in the Wien limit. */
double dust_oracle_planck(double lambda, double T)
{
    double x = ORC_H * ORC_C / (ORC_K * lambda * T);
    double l2 = lambda * lambda;
    double pref = 2.0 * ORC_H * ORC_C * ORC_C / (l2 * l2 * lambda);
    return pref * exp(-x) / (-expm1(-x));
}

/* Heating power of grain g in cell c: A = sum_k w_k C_k J_k, k ascending
 * (Eq. 6; the paper's I_c,l sigma_s,l Delta lambda_l). */
double dust_oracle_absorbed(int K, const double *w, const double *C_g, const double *J_c)
{
    double s = 0.0;
    for (int k = 0; k < K; ++k)
        s += w[k] * C_g[k] * J_c[k];
    return s;
}

/* Emitted power of grain g at temperature T: P = sum_k w_k C_k B(lambda_k, T)
 * (right-hand side of Eq. 7). */
double dust_oracle_power(int K, const double *lambda, const double *w, const double *C_g, double T)
{
    double s = 0.0;
    for (int k = 0; k < K; ++k)
        s += w[k] * C_g[k] * dust_oracle_planck(lambda[k], T);
    return s;
}

typedef struct {
    int K;
    const double *lambda, *w, *C_g;
    double lnA;
    int evals;
} root_fn;

/* F(u) = ln P_g(e^u) - ln A; strictly increasing in u when some C_k > 0. */
static double F_of_u(root_fn *f, double u)
{
    f->evals++;
    return log(dust_oracle_power(f->K, f->lambda, f->w, f->C_g, exp(u))) - f->lnA;
}

/* Brent's method on [lo, hi] with F(lo) < 0 < F(hi).
 * Keeps b (best estimate), a (previous b) and c (the point that brackets the
 * root with b).  Each step tries inverse quadratic interpolation through a, b,
 * c (or the secant through a, b when only two distinct points exist) and falls
 * back to bisection whenever the interpolated step leaves the bracket or does
 * not shrink faster than the step before last. */
static double brent(root_fn *f, double lo, double hi, double flo, double fhi, double tol, int maxit)
{
    double a = lo, b = hi, c = lo;
    double fa = flo, fb = fhi, fc = flo;
    double d = b - a, e = d;
    for (int it = 0; it < maxit; ++it) {
        if ((fb > 0.0 && fc > 0.0) || (fb < 0.0 && fc < 0.0)) {
            /* the root lies between a and b: make c the bracketing end */
            c = a; fc = fa; d = b - a; e = d;
        }
        if (fabs(fc) < fabs(fb)) {
            /* b must be the end with the smaller residual */
            a = b; fa = fb;
            b = c; fb = fc;
            c = a; fc = fa;
        }
        double tol1 = 2.0 * DBL_EPSILON * fabs(b) + 0.5 * tol;
        double half = 0.5 * (c - b);
        if (fabs(half) <= tol1 || fb == 0.0)
            return b;
        if (fabs(e) >= tol1 && fabs(fa) > fabs(fb)) {
            double p, q;
            double s = fb / fa;
            if (a == c) {
                /* secant through (a, fa) and (b, fb) */
                p = 2.0 * half * s;
                q = 1.0 - s;
            } else {
                /* inverse quadratic through (a, fa), (b, fb), (c, fc) */
                double qa = fa / fc, rb = fb / fc;
                p = s * (2.0 * half * qa * (qa - rb) - (b - a) * (rb - 1.0));
                q = (qa - 1.0) * (rb - 1.0) * (s - 1.0);
            }
            if (p > 0.0) q = -q; else p = -p;
            double lim1 = 3.0 * half * q - fabs(tol1 * q);
            double lim2 = fabs(e * q);
            if (2.0 * p < (lim1 < lim2 ? lim1 : lim2)) {
                e = d;          /* accept the interpolated step */
                d = p / q;
            } else {
                d = half;       /* bisect */
                e = d;
            }
        } else {
            d = half;
            e = d;
        }
        a = b; fa = fb;
        b += (fabs(d) > tol1) ? d : (half > 0.0 ? tol1 : -tol1);
        fb = F_of_u(f, b);
    }
    return b;
}

/* Equilibrium temperature of one grain in one cell: the root of Eq. 7 for the
 * heating power A of Eq. 6.  Returns the clamp flag; *T receives the
 * temperature and *evals the number of quadratures used. */
int dust_oracle_temperature(int K, const double *lambda, const double *w, const double *C_g,
                            double A, double T_min, double T_max, double tol_u,
                            double *T, int *evals)
{
    root_fn f = {K, lambda, w, C_g, 0.0, 0};
    if (!(A >= 0.0) || isinf(A)) { *T = NAN; if (evals) *evals = 0; return 4; }
    if (A == 0.0) { *T = T_min; if (evals) *evals = 0; return 1; }
    f.lnA = log(A);
    double lo = log(T_min), hi = log(T_max);
    double flo = F_of_u(&f, lo), fhi = F_of_u(&f, hi);
    int flag = 0;
    if (flo > 0.0) { *T = T_min; flag = 1; }
    else if (fhi < 0.0) { *T = T_max; flag = 2; }
    else if (flo == 0.0) *T = T_min;
    else if (fhi == 0.0) *T = T_max;
    else *T = exp(brent(&f, lo, hi, flo, fhi, tol_u, 400));
    if (evals) *evals = f.evals;
    return flag;
}

/* The same root by plain bisection on u (a cross-check for Brent). */
double dust_oracle_temperature_bisect(int K, const double *lambda, const double *w,
                                      const double *C_g, double A, double T_min, double T_max,
                                      int steps)
{
    root_fn f = {K, lambda, w, C_g, log(A), 0};
    double lo = log(T_min), hi = log(T_max);
    for (int i = 0; i < steps; ++i) {
        double mid = 0.5 * (lo + hi);
        if (F_of_u(&f, mid) < 0.0) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

/* Emission SED of one cell: L_k = 4 pi sum_g n_g C[g,k] B(lambda_k, T_g)
 * (Eqs. 8-10; the paper's n_s m_d;c is the general n[c,g] here, and the 4 pi
 * turns the per-steradian quantities into luminosities). */
void dust_oracle_emission(int K, int G, const double *lambda, const double *C, const double *n_c,
                          const double *T_c, double *L_c)
{
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int g = 0; g < G; ++g)
            s += n_c[g] * C[(size_t)g * K + k] * dust_oracle_planck(lambda[k], T_c[g]);
        L_c[k] = 4.0 * ORC_PI * s;
    }
}

/* The whole path over n_cells cells.  J is [n_cells, K] and n is [n_cells, G],
 * both row-major FP64.  Outputs (any may be NULL except T): A [n_cells, G],
 * T [n_cells, G], L [n_cells, K], flags [n_cells, G], resid [n_cells].
 * n_threads <= 0 uses the OpenMP default.  Returns the number of quadratures
 * spent in root solves. */
int64_t dust_oracle_run(int64_t n_cells, int K, int G, const double *lambda, const double *w,
                        const double *C, const double *J, const double *n, double T_min,
                        double T_max, double tol_u, double *A_out, double *T_out, double *L_out,
                        uint8_t *flags_out, double *resid_out, int n_threads)
{
    int64_t total_evals = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total_evals)
    for (int64_t c = 0; c < n_cells; ++c) {
        const double *Jc = J + c * (int64_t)K;
        const double *nc = n + c * (int64_t)G;
        double *Tc = T_out + c * (int64_t)G;
        double absorbed = 0.0;
        for (int g = 0; g < G; ++g) {
            const double *Cg = C + (size_t)g * K;
            double A = dust_oracle_absorbed(K, w, Cg, Jc);
            int ev = 0;
            int fl = dust_oracle_temperature(K, lambda, w, Cg, A, T_min, T_max, tol_u, &Tc[g], &ev);
            total_evals += ev;
            double pe = (fl == 0) ? A : dust_oracle_power(K, lambda, w, Cg, Tc[g]);
            absorbed += nc[g] * pe;
            if (A_out) A_out[c * (int64_t)G + g] = A;
            if (flags_out) flags_out[c * (int64_t)G + g] = (uint8_t)fl;
        }
        if (L_out || resid_out) {
            double *Lc = L_out ? L_out + c * (int64_t)K : (double *)malloc(sizeof(double) * (size_t)K);
            dust_oracle_emission(K, G, lambda, C, nc, Tc, Lc);
            if (resid_out) {
                double emitted = 0.0;
                for (int k = 0; k < K; ++k)
                    emitted += w[k] * Lc[k];
                resid_out[c] = emitted / (4.0 * ORC_PI * absorbed) - 1.0;
            }
            if (!L_out) free(Lc);
        }
    }
    return total_evals;
}

/* Number of threads an OpenMP region would use (the core count reported next
 * to CPU timings). */
int dust_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
