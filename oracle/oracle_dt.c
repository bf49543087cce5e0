/*
 * oracle_dt.c - FP64 reference of the cluster-cluster (dual-tree) Barnes-Hut
 * form (TEST INFRASTRUCTURE ONLY; nothing outside tests/, the smoke check and
 * the CPU-baseline leg of the benchmark loads it).
 *
 * Sec. 3.2 clusters only the inner integral; its comparison method clusters
 * both integrals.  This file is that second scheme, written out on the same
 * cluster tree (or_lbvh) and moments (or_moments):
 *
 *  - Every unordered pair of triangles {T, S} is assigned to exactly one
 *    unordered pair of tree nodes {A, B} by the recursion from (root, root):
 *      A == B: a node of at most leaf_size members (or a primitive) is a near
 *              self pair; otherwise recurse on (l, l), (r, r), (l, r);
 *      A != B: admissible -> far pair; both nodes of at most leaf_size
 *              members -> near pair; otherwise split the node with more
 *              members (a node of at most leaf_size members is never split).
 *  - Admissibility of {A, B} (the symmetric reading of the separation test):
 *    the vertex boxes are strictly disjoint along some axis (no pair sharing
 *    a vertex is approximated) and max(diag_A, diag_B) < theta |X_A - X_B|,
 *    X the area-weighted centroid; FP64, separately rounded, fixed order.
 *  - A far pair contributes both orderings of the cluster monopole,
 *      E_AB = A_A A_B (|nubar_A.(X_A - X_B)|^q + |nubar_B.(X_B - X_A)|^q) / |X_A - X_B|^p,
 *    nubar = sum(w nu)/A (not renormalised); a near pair contributes its
 *    admitted member pairs exactly (both orderings).
 *  - The gradient is the exact derivative of this approximate energy: the
 *    far terms depend on the triangles through the moments A = sum w,
 *    X = sum w x / A, nubar = sum w nu / A, so a far pair's derivatives with
 *    respect to (A, X, nubar) of each node are collected per node and passed
 *    down to the member triangles:
 *      dE/dx_T  += w_T dE/dX_N / A_N,   dE/dnu_T += w_T dE/dnubar_N / A_N,
 *      dE/dw_T  += dE/dA_N + (dE/dX_N.(x_T - X_N) + dE/dnubar_N.(nu_T - nubar_N)) / A_N
 *    for every node N holding T.
 *
 * Outputs are the per-triangle derivatives (gw, gnu, gx) without the
 * prefactor c, in the layout of or_tri_accum, and the energy without c.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static double dt_powabs(double n, double q) { return pow(fabs(n), q); }

static double dt_dpowabs(double n, double q) {
    if (n == 0.0) return 0.0;
    return q * pow(fabs(n), q - 1.0) * (n > 0.0 ? 1.0 : -1.0);
}

static int dt_excluded(const int32_t* F, int64_t T, int64_t S, int adj) {
    if (T == S) return 1;
    int k = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (F[3 * T + i] == F[3 * S + j]) ++k;
    return adj == 0 ? (k >= 1) : (k >= 2);
}

/* both orderings of the admitted pair (T, S): energy, and the derivatives of
 * e_TS + e_ST with respect to T's and S's own (w, nu, x) */
static double dt_near_pair(const double* x, const double* nu, const double* w, int64_t T, int64_t S, double q,
                           double p, double* gw, double* gnu, double* gx) {
    double d[3], r2 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = x[3 * T + k] - x[3 * S + k];
        r2 += d[k] * d[k];
    }
    for (int k = 0; k < 3; ++k) {
        n1 += nu[3 * T + k] * d[k];    /* nu_T.(x_T - x_S) */
        n2 += nu[3 * S + k] * (-d[k]); /* nu_S.(x_S - x_T) */
    }
    const double rp = pow(r2, -0.5 * p), rp2 = rp / r2;
    const double a1 = dt_powabs(n1, q), b1 = dt_dpowabs(n1, q);
    const double a2 = dt_powabs(n2, q), b2 = dt_dpowabs(n2, q);
    const double wT = w[T], wS = w[S];
    gw[T] += wS * (a1 + a2) * rp;
    gw[S] += wT * (a1 + a2) * rp;
    for (int k = 0; k < 3; ++k) {
        gnu[3 * T + k] += wT * wS * b1 * rp * d[k];
        gnu[3 * S + k] += wT * wS * b2 * rp * (-d[k]);
        /* d/dd of the pair energy; x_T enters as +d, x_S as -d */
        const double g = wT * wS * (b1 * rp * nu[3 * T + k] - b2 * rp * nu[3 * S + k] - p * (a1 + a2) * rp2 * d[k]);
        gx[3 * T + k] += g;
        gx[3 * S + k] -= g;
    }
    return wT * wS * (a1 + a2) * rp;
}

static double dt_diag2(const double* b) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = b[3 + a] - b[a];
        s = s + e * e;
    }
    return s;
}

int or_dt_admissible(const double* bA, const double* mA, const double* bB, const double* mB, double theta) {
    int disjoint = 0;
    for (int a = 0; a < 3; ++a)
        if (bA[3 + a] < bB[a] || bB[3 + a] < bA[a]) disjoint = 1;
    if (!disjoint) return 0;
    const double dA2 = dt_diag2(bA), dB2 = dt_diag2(bB);
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double t = mA[1 + a] / mA[0] - mB[1 + a] / mB[0];
        r2 = r2 + t * t;
    }
    const double diag = sqrt(dA2 > dB2 ? dA2 : dB2);
    return diag < theta * sqrt(r2);
}

/* far pair: energy, and dE/d(A, X[3], nubar[3]) of both nodes into G (7 per node) */
static double dt_far_pair(const double* mA, const double* mB, double q, double p, double* GA, double* GB) {
    const double AA = mA[0], AB = mB[0];
    double XA[3], XB[3], nA[3], nB[3], d[3], r2 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        XA[a] = mA[1 + a] / AA;
        XB[a] = mB[1 + a] / AB;
        nA[a] = mA[4 + a] / AA;
        nB[a] = mB[4 + a] / AB;
        d[a] = XA[a] - XB[a];
        r2 += d[a] * d[a];
    }
    for (int a = 0; a < 3; ++a) {
        n1 += nA[a] * d[a];    /* nubar_A.(X_A - X_B) */
        n2 += nB[a] * (-d[a]); /* nubar_B.(X_B - X_A) */
    }
    const double rp = pow(r2, -0.5 * p), rp2 = rp / r2;
    const double a1 = dt_powabs(n1, q), b1 = dt_dpowabs(n1, q);
    const double a2 = dt_powabs(n2, q), b2 = dt_dpowabs(n2, q);
    const double E = AA * AB * (a1 + a2) * rp;
    GA[0] += AB * (a1 + a2) * rp;
    GB[0] += AA * (a1 + a2) * rp;
    for (int k = 0; k < 3; ++k) {
        const double gX = AA * AB * (b1 * rp * nA[k] - b2 * rp * nB[k] - p * (a1 + a2) * rp2 * d[k]);
        GA[1 + k] += gX;
        GB[1 + k] -= gX;
        GA[4 + k] += AA * AB * b1 * rp * d[k];
        GB[4 + k] += AA * AB * b2 * rp * (-d[k]);
    }
    return E;
}

double or_dt_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t n,
                   const int32_t* perm, const int32_t* left, const int32_t* right, const int32_t* parent,
                   const int32_t* first, const int32_t* last, const double* mom, const double* box, double theta,
                   int leaf_size, double q, double p, int adj, double* gw, double* gnu, double* gx,
                   int64_t* n_near_pairs, int64_t* n_far_pairs, int64_t* n_far_represented) {
    memset(gw, 0, sizeof(double) * (size_t)n);
    memset(gnu, 0, sizeof(double) * 3 * (size_t)n);
    memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    int64_t near_pairs = 0, far_pairs = 0, far_rep = 0;
    double E = 0.0;
    if (n < 1) return 0.0;
    const int64_t nn = 2 * n - 1;
    double* G = (double*)calloc((size_t)nn * 7, sizeof(double));
    /* explicit stack of node pairs */
    int64_t cap = 1024, sp = 0;
    int64_t* st = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)cap);
    st[0] = 0;
    st[1] = 0;
    sp = 1;
    while (sp > 0) {
        --sp;
        const int64_t A = st[2 * sp], B = st[2 * sp + 1];
        const int64_t cA = (int64_t)last[A] - first[A] + 1, cB = (int64_t)last[B] - first[B] + 1;
        const int smallA = cA <= leaf_size || A >= n - 1, smallB = cB <= leaf_size || B >= n - 1;
        int64_t push[3][2];
        int npush = 0;
        if (A == B) {
            if (smallA) {
                for (int64_t i = first[A]; i <= last[A]; ++i)
                    for (int64_t j = i + 1; j <= last[A]; ++j) {
                        const int64_t T = perm[i], S = perm[j];
                        if (dt_excluded(F, T, S, adj)) continue;
                        E += dt_near_pair(x, nu, w, T, S, q, p, gw, gnu, gx);
                        near_pairs += 2;
                    }
            } else {
                push[0][0] = left[A], push[0][1] = left[A];
                push[1][0] = right[A], push[1][1] = right[A];
                push[2][0] = left[A], push[2][1] = right[A];
                npush = 3;
            }
        } else if (or_dt_admissible(box + 6 * A, mom + 13 * A, box + 6 * B, mom + 13 * B, theta)) {
            E += dt_far_pair(mom + 13 * A, mom + 13 * B, q, p, G + 7 * A, G + 7 * B);
            far_pairs += 1;
            far_rep += 2 * cA * cB;
        } else if (smallA && smallB) {
            for (int64_t i = first[A]; i <= last[A]; ++i)
                for (int64_t j = first[B]; j <= last[B]; ++j) {
                    const int64_t T = perm[i], S = perm[j];
                    if (dt_excluded(F, T, S, adj)) continue;
                    E += dt_near_pair(x, nu, w, T, S, q, p, gw, gnu, gx);
                    near_pairs += 2;
                }
        } else if (!smallA && (cA >= cB || smallB)) {
            push[0][0] = left[A], push[0][1] = B;
            push[1][0] = right[A], push[1][1] = B;
            npush = 2;
        } else {
            push[0][0] = A, push[0][1] = left[B];
            push[1][0] = A, push[1][1] = right[B];
            npush = 2;
        }
        if (sp + npush > cap) {
            cap *= 2;
            st = (int64_t*)realloc(st, sizeof(int64_t) * 2 * (size_t)cap);
        }
        for (int k = npush - 1; k >= 0; --k) {
            st[2 * sp] = push[k][0];
            st[2 * sp + 1] = push[k][1];
            ++sp;
        }
    }
    free(st);
    /* pass the node derivatives down to the member triangles */
    for (int64_t k = 0; k < n; ++k) {
        const int64_t T = perm[k];
        for (int64_t N = (n > 1 ? n - 1 + k : 0); N >= 0; N = (N == 0 ? -1 : parent[N])) {
            const double* g = G + 7 * N;
            const double* m = mom + 13 * N;
            const double AN = m[0];
            double dw = g[0];
            for (int a = 0; a < 3; ++a) {
                gx[3 * T + a] += w[T] * g[1 + a] / AN;
                gnu[3 * T + a] += w[T] * g[4 + a] / AN;
                dw += (g[1 + a] * (x[3 * T + a] - m[1 + a] / AN) + g[4 + a] * (nu[3 * T + a] - m[4 + a] / AN)) / AN;
            }
            gw[T] += dw;
            if (N == 0) break;
        }
    }
    free(G);
    if (n_near_pairs) *n_near_pairs = near_pairs;
    if (n_far_pairs) *n_far_pairs = far_pairs;
    if (n_far_represented) *n_far_represented = far_rep;
    return E;
}
