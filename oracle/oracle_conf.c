/*
 * oracle_conf.c - FP64 CPU reference for the confinement energy (TEST
 * INFRASTRUCTURE ONLY; loaded by the tests and the benchmark's CPU legs,
 * shares no code with the CUDA library).
 *
 * Eq. (TPConf), Sec. 2.2 (Confinement): the tangent-point kernel between the
 * evolving surface S and a fixed confining surface S_conf,
 *
 *   Phi_conf = c * sum_{T in S} sum_{K in S_conf} w_T a_K |<nu_T, x_T - y_K>|^q / |x_T - y_K|^p
 *
 * with one centroid point per flat triangle on both surfaces: x_T, nu_T,
 * w_T the centroid, unit normal and area of T on S; y_K, a_K the centroid
 * and area of K on S_conf.  Only the normal of the evolving surface enters
 * (the paper notes the confinement may be non-smooth because its normal is
 * never evaluated), and only S moves, so the derivatives are taken with
 * respect to S alone.  c stands for rho_conf/alpha; q = alpha, p = 2 alpha.
 * The two surfaces share no vertices, so no pair is left out.
 */
#include <math.h>

#include "oracle.h"

static double cf_powabs(double n, double q) { return pow(fabs(n), q); }

/* d/dn |n|^q = q |n|^(q-1) sgn(n) */
static double cf_dpowabs(double n, double q) {
    if (n == 0.0) return 0.0;
    return q * pow(fabs(n), q - 1.0) * (n > 0.0 ? 1.0 : -1.0);
}

double or_conf_energy(const double* x, const double* nu, const double* w, int64_t nt, const double* y,
                      const double* a, int64_t nk, double q, double p, double c, int nthreads) {
    double E = 0.0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(+ : E)
    for (int64_t T = 0; T < nt; ++T) {
        double s = 0.0;
        for (int64_t K = 0; K < nk; ++K) {
            double d[3], r2 = 0.0, n = 0.0;
            for (int i = 0; i < 3; ++i) {
                d[i] = x[3 * T + i] - y[3 * K + i];
                r2 += d[i] * d[i];
                n += nu[3 * T + i] * d[i];
            }
            s += a[K] * cf_powabs(n, q) / pow(r2, 0.5 * p);
        }
        E += w[T] * s;
    }
    return c * E;
}

/* Per triangle T of S (without c):
 *   dPhi/dw_T  = sum_K a_K |n|^q / r^p
 *   dPhi/dnu_T = sum_K w_T a_K (d/dn |n|^q) d / r^p
 *   dPhi/dx_T  = sum_K w_T a_K [ (d/dn |n|^q) nu_T / r^p - p |n|^q d / r^(p+2) ]
 * with d = x_T - y_K, n = nu_T . d, r = |d|. */
void or_conf_accum(const double* x, const double* nu, const double* w, int64_t nt, const double* y, const double* a,
                   int64_t nk, double q, double p, double* gw, double* gnu, double* gx, int nthreads) {
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t T = 0; T < nt; ++T) {
        double sw = 0.0, sn[3] = {0, 0, 0}, sx[3] = {0, 0, 0};
        for (int64_t K = 0; K < nk; ++K) {
            double d[3], r2 = 0.0, n = 0.0;
            for (int i = 0; i < 3; ++i) {
                d[i] = x[3 * T + i] - y[3 * K + i];
                r2 += d[i] * d[i];
                n += nu[3 * T + i] * d[i];
            }
            const double rp = pow(r2, 0.5 * p);
            const double f = cf_powabs(n, q), df = cf_dpowabs(n, q);
            sw += a[K] * f / rp;
            for (int i = 0; i < 3; ++i) {
                sn[i] += w[T] * a[K] * df * d[i] / rp;
                sx[i] += w[T] * a[K] * (df * nu[3 * T + i] / rp - p * f * d[i] / (rp * r2));
            }
        }
        gw[T] = sw;
        for (int i = 0; i < 3; ++i) {
            gnu[3 * T + i] = sn[i];
            gx[3 * T + i] = sx[i];
        }
    }
}
