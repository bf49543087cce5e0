/*
 * oracle_quad.c - FP64 CPU reference for the multi-point quadrature form of
 * the tangent-point energy (TEST INFRASTRUCTURE ONLY; shares no code with the
 * CUDA library).
 *
 * Sec. 3.1 and Sec. 3.2 integrate both integrals of Eq. (TP) with a
 * quadrature rule per element instead of one centroid point.  On a flat
 * triangle T with a rule of k points (barycentric coordinates l_q and
 * weights om_q summing to 1) the points are x_q = l_q0 v0 + l_q1 v1 + l_q2 v2
 * with the normal nu_T and the weight om_q w_T.  The double sum then runs
 * over ordered pairs of points whose triangles are admitted (different and
 * sharing no vertex), which is the one-point sum of oracle.c over the
 * expanded point set with every point carrying its triangle's vertices.
 * Both integrals use the same rule here.
 */
#include <math.h>

#include "oracle.h"

void or_quad_points(const double* V, const int32_t* F, int64_t nt, int k, const double* bary, const double* om,
                    double* x, double* nu, double* w, int32_t* Fq) {
    for (int64_t T = 0; T < nt; ++T) {
        const double* a = V + 3 * (int64_t)F[3 * T + 0];
        const double* b = V + 3 * (int64_t)F[3 * T + 1];
        const double* c = V + 3 * (int64_t)F[3 * T + 2];
        double e1[3], e2[3], N[3];
        for (int i = 0; i < 3; ++i) {
            e1[i] = b[i] - a[i];
            e2[i] = c[i] - a[i];
        }
        N[0] = e1[1] * e2[2] - e1[2] * e2[1];
        N[1] = e1[2] * e2[0] - e1[0] * e2[2];
        N[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double len = sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
        for (int q = 0; q < k; ++q) {
            const int64_t P = T * k + q;
            const double* l = bary + 3 * q;
            for (int i = 0; i < 3; ++i) {
                x[3 * P + i] = (l[0] * a[i] + l[1] * b[i]) + l[2] * c[i];
                nu[3 * P + i] = N[i] / len;
                Fq[3 * P + i] = F[3 * T + i];
            }
            w[P] = om[q] * (0.5 * len);
        }
    }
}

/* c times the pull-back of per-point (dPhi/dw_q, dPhi/dnu_q, dPhi/dx_q) to the
 * vertices, added into grad[nv][3].  With N = e1 x e2, w_q = om_q |N| / 2,
 * nu_q = N / |N| and x_q = sum_i l_qi v_i:
 *   dPhi/dN = sum_q [ om_q gw_q nu / 2 + (I - nu nu^T) gnu_q / |N| ],
 *   dPhi/dv1 += e2 x dPhi/dN, dPhi/dv2 += dPhi/dN x e1, dPhi/dv0 -= both,
 *   dPhi/dv_i += sum_q l_qi gx_q. */
void or_quad_adjoint(const double* V, const int32_t* F, int64_t nt, int k, const double* bary, const double* om,
                     const double* gw, const double* gnu, const double* gx, double c, double* grad) {
    for (int64_t T = 0; T < nt; ++T) {
        const int64_t i0 = F[3 * T + 0], i1 = F[3 * T + 1], i2 = F[3 * T + 2];
        const double *a = V + 3 * i0, *b = V + 3 * i1, *cc = V + 3 * i2;
        double e1[3], e2[3], N[3];
        for (int i = 0; i < 3; ++i) {
            e1[i] = b[i] - a[i];
            e2[i] = cc[i] - a[i];
        }
        N[0] = e1[1] * e2[2] - e1[2] * e2[1];
        N[1] = e1[2] * e2[0] - e1[0] * e2[2];
        N[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const double nu[3] = {N[0] / len, N[1] / len, N[2] / len};
        double G[3] = {0, 0, 0}, px[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int q = 0; q < k; ++q) {
            const int64_t P = T * k + q;
            const double* gn = gnu + 3 * P;
            const double ndg = nu[0] * gn[0] + nu[1] * gn[1] + nu[2] * gn[2];
            for (int i = 0; i < 3; ++i) {
                G[i] += om[q] * gw[P] * nu[i] * 0.5 + (gn[i] - nu[i] * ndg) / len;
                for (int j = 0; j < 3; ++j) px[j][i] += bary[3 * q + j] * gx[3 * P + i];
            }
        }
        const double g1[3] = {e2[1] * G[2] - e2[2] * G[1], e2[2] * G[0] - e2[0] * G[2], e2[0] * G[1] - e2[1] * G[0]};
        const double g2[3] = {G[1] * e1[2] - G[2] * e1[1], G[2] * e1[0] - G[0] * e1[2], G[0] * e1[1] - G[1] * e1[0]};
        for (int i = 0; i < 3; ++i) {
            grad[3 * i0 + i] += c * (px[0][i] - g1[i] - g2[i]);
            grad[3 * i1 + i] += c * (px[1][i] + g1[i]);
            grad[3 * i2 + i] += c * (px[2][i] + g2[i]);
        }
    }
}
