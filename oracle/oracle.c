/*
 * oracle.c - plain FP64 CPU reference for the tangent-point energy and its
 * vertex gradient on a flat triangle mesh (TEST INFRASTRUCTURE ONLY).
 *
 * Nothing outside tests/, the smoke check and the CPU-baseline leg of the
 * benchmark loads this file.  It shares no code with the CUDA library.  It is
 * compiled with -O2 -ffp-contract=off so that every product and sum is
 * rounded separately (IEEE round-to-nearest), which the bit-exact parts
 * (centroids, Morton codes, tree, moments) rely on.
 *
 * Sources followed:
 *  - Eq. (TP), Sec. 2.2.2: Phi = rho/alpha * double integral of
 *    |nu(x).(x-y)|^alpha / |x-y|^(2 alpha); alpha = 6 (Sec. 2.2.2).  Here the
 *    surface is a flat triangle mesh with one quadrature point (the centroid)
 *    per triangle, q = alpha, p = 2 alpha, and c = rho/alpha is the caller's
 *    prefactor.  Pairs of triangles sharing a vertex are left out (the
 *    integrand is singular on the diagonal x = y).
 *  - Eq. (dTP) and Eq. (dTP_reordered), Sec. 3.2: the variation is assembled
 *    per outer point from inner sums of both orderings K(x,y) and K(y,x);
 *    here that is the exact chain rule of the discrete sum, gathered per
 *    triangle into dPhi/dx_T, dPhi/dnu_T, dPhi/dw_T, then pulled back to the
 *    vertices through x_T = (v0+v1+v2)/3, N = (v1-v0)x(v2-v0), w = |N|/2,
 *    nu = N/|N|.
 *  - Sec. 3.2 (clustering of the inner integral only, "precomputed averages
 *    over a patch", admissibility after Yu et al., separation parameter
 *    theta): or_bh_accum.  The cluster tree is a linear BVH over Morton codes
 *    (the paper does not name its tree type).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- helpers */

static int shared_vertices(const int32_t* F, int64_t T, int64_t S) {
    int k = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (F[3 * T + i] == F[3 * S + j]) ++k;
    return k;
}

/* T and S are excluded from the double sum when T == S or they touch. */
static int excluded(const int32_t* F, int64_t T, int64_t S, int adj) {
    if (T == S) return 1;
    int k = shared_vertices(F, T, S);
    return adj == 0 ? (k >= 1) : (k >= 2);
}

static double powabs(double n, double q) { return pow(fabs(n), q); }

/* d/dn |n|^q = q |n|^(q-1) sgn(n) */
static double dpowabs(double n, double q) {
    if (n == 0.0) return 0.0;
    double s = n > 0.0 ? 1.0 : -1.0;
    return q * pow(fabs(n), q - 1.0) * s;
}

/* ------------------------------------------------------------ tri data */

void or_tri_data(const double* V, const int32_t* F, int64_t nt, double* x, double* nu, double* w) {
    for (int64_t T = 0; T < nt; ++T) {
        const double* a = V + 3 * (int64_t)F[3 * T + 0];
        const double* b = V + 3 * (int64_t)F[3 * T + 1];
        const double* c = V + 3 * (int64_t)F[3 * T + 2];
        double e1[3], e2[3], N[3];
        for (int k = 0; k < 3; ++k) {
            x[3 * T + k] = ((a[k] + b[k]) + c[k]) / 3.0;
            e1[k] = b[k] - a[k];
            e2[k] = c[k] - a[k];
        }
        N[0] = e1[1] * e2[2] - e1[2] * e2[1];
        N[1] = e1[2] * e2[0] - e1[0] * e2[2];
        N[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double len = sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
        w[T] = 0.5 * len;
        for (int k = 0; k < 3; ++k) nu[3 * T + k] = N[k] / len;
    }
}

/* ------------------------------------------------------------ energy */

/* one ordered pair: w_T w_S |nu_T.(x_T-x_S)|^q / |x_T-x_S|^p  (Eq. TP) */
static double pair_energy(const double* x, const double* nu, const double* w, int64_t T, int64_t S,
                          double q, double p) {
    double d[3], r2 = 0.0, n = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = x[3 * T + k] - x[3 * S + k];
        r2 += d[k] * d[k];
        n += nu[3 * T + k] * d[k];
    }
    return w[T] * w[S] * powabs(n, q) / pow(r2, 0.5 * p);
}

double or_energy(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                 double q, double p, double c, int adj, int nthreads) {
    double* part = (double*)calloc((size_t)(nt > 0 ? nt : 1), sizeof(double));
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t T = 0; T < nt; ++T) {
        double s = 0.0;
        for (int64_t S = 0; S < nt; ++S) {
            if (excluded(F, T, S, adj)) continue;
            s += pair_energy(x, nu, w, T, S, q, p);
        }
        part[T] = s;
    }
    double E = 0.0;
    for (int64_t T = 0; T < nt; ++T) E += part[T];
    free(part);
    return c * E;
}

/* Number of ordered pairs (T, S) the double sum of or_energy runs over: every
 * T != S that the exclusion rule (adj) keeps.  Brute force over all nt^2
 * ordered pairs with the same test as the energy. */
int64_t or_admitted_pairs(const int32_t* F, int64_t nt, int adj, int nthreads) {
    int64_t total = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads) reduction(+ : total)
    for (int64_t T = 0; T < nt; ++T) {
        int64_t k = 0;
        for (int64_t S = 0; S < nt; ++S) k += excluded(F, T, S, adj) ? 0 : 1;
        total += k;
    }
    return total;
}

/* Energy of the ordered pairs (T,S) with T or S in the set: the part of Phi
 * that changes when only vertices of triangles in the set move. */
double or_energy_touching(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                          const uint8_t* in_set, double q, double p, double c, int adj, int nthreads) {
    int64_t m = 0;
    for (int64_t T = 0; T < nt; ++T) m += in_set[T] ? 1 : 0;
    int64_t* mem = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    m = 0;
    for (int64_t T = 0; T < nt; ++T)
        if (in_set[T]) mem[m++] = T;
    double* part = (double*)calloc((size_t)(nt > 0 ? nt : 1), sizeof(double));
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int64_t T = 0; T < nt; ++T) {
        double s = 0.0;
        if (in_set[T]) {
            for (int64_t S = 0; S < nt; ++S)
                if (!excluded(F, T, S, adj)) s += pair_energy(x, nu, w, T, S, q, p);
        } else {
            for (int64_t k = 0; k < m; ++k)
                if (!excluded(F, T, mem[k], adj)) s += pair_energy(x, nu, w, T, mem[k], q, p);
        }
        part[T] = s;
    }
    double E = 0.0;
    for (int64_t T = 0; T < nt; ++T) E += part[T];
    free(part);
    free(mem);
    return c * E;
}

/* ------------------------------------------------------------ gradient */

/* Add to (gw, gnu, gx) of triangle T the derivatives of e_TS + e_ST with
 * respect to w_T, nu_T and x_T (the chain rule of both orderings; the
 * prefactor c is applied in or_adjoint).  */
static void pair_grad_gather(const double* x, const double* nu, const double* w, int64_t T, int64_t S,
                             double q, double p, double* gw, double* gnu, double* gx) {
    double d[3], r2 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = x[3 * T + k] - x[3 * S + k];
        r2 += d[k] * d[k];
    }
    for (int k = 0; k < 3; ++k) {
        n1 += nu[3 * T + k] * d[k];    /* nu_T . (x_T - x_S) */
        n2 += nu[3 * S + k] * (-d[k]); /* nu_S . (x_S - x_T) */
    }
    double rp = pow(r2, -0.5 * p);  /* |d|^-p     */
    double rp2 = rp / r2;           /* |d|^-(p+2) */
    double a1 = powabs(n1, q), b1 = dpowabs(n1, q);
    double a2 = powabs(n2, q), b2 = dpowabs(n2, q);
    double wT = w[T], wS = w[S];
    /* d(e_TS + e_ST)/dw_T */
    *gw += wS * (a1 + a2) * rp;
    for (int k = 0; k < 3; ++k) {
        /* d e_TS / d nu_T = w_T w_S q|n1|^(q-1) sgn(n1) |d|^-p d */
        gnu[k] += wT * wS * b1 * rp * d[k];
        /* d e_TS / d x_T: n1 depends on x_T through d (+nu_T), |d| through d */
        double g = wT * wS * (b1 * rp * nu[3 * T + k] - p * a1 * rp2 * d[k]);
        /* d e_ST / d x_T: n2 = nu_S.(x_S - x_T) gives -nu_S, |d|^-p gives -p|d|^-(p+2) d */
        g += wT * wS * (-b2 * rp * nu[3 * S + k] - p * a2 * rp2 * d[k]);
        gx[k] += g;
    }
}

void or_tri_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                  const int64_t* list, int64_t nlist, double q, double p, int adj,
                  double* gw, double* gnu, double* gx, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t m = list ? nlist : nt;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t i = 0; i < m; ++i) {
        int64_t T = list ? list[i] : i;
        double a = 0.0, bn[3] = {0, 0, 0}, bx[3] = {0, 0, 0};
        for (int64_t S = 0; S < nt; ++S) {
            if (excluded(F, T, S, adj)) continue;
            pair_grad_gather(x, nu, w, T, S, q, p, &a, bn, bx);
        }
        gw[i] = a;
        for (int k = 0; k < 3; ++k) {
            gnu[3 * i + k] = bn[k];
            gx[3 * i + k] = bx[k];
        }
    }
}

/* Pull (dPhi/dw_T, dPhi/dnu_T, dPhi/dx_T) back to the vertices of T and add
 * c times the result into grad[nv][3].  With N = e1 x e2, |N| = 2 w:
 *   dPhi/dN = gw nu / 2 + (I - nu nu^T) gnu / |N|
 *   dPhi/de1 = e2 x dPhi/dN,   dPhi/de2 = dPhi/dN x e1
 *   v1 += dPhi/de1, v2 += dPhi/de2, v0 -= both, and gx/3 to each vertex. */
void or_adjoint(const double* V, const int32_t* F, const int64_t* list, int64_t nlist,
                const double* gw, const double* gnu, const double* gx, double c, double* grad) {
    for (int64_t i = 0; i < nlist; ++i) {
        int64_t T = list ? list[i] : i;
        int64_t i0 = F[3 * T + 0], i1 = F[3 * T + 1], i2 = F[3 * T + 2];
        const double *a = V + 3 * i0, *b = V + 3 * i1, *cc = V + 3 * i2;
        double e1[3], e2[3], N[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = b[k] - a[k];
            e2[k] = cc[k] - a[k];
        }
        N[0] = e1[1] * e2[2] - e1[2] * e2[1];
        N[1] = e1[2] * e2[0] - e1[0] * e2[2];
        N[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        double nu[3] = {N[0] / len, N[1] / len, N[2] / len};
        const double* gn = gnu + 3 * i;
        double ndg = nu[0] * gn[0] + nu[1] * gn[1] + nu[2] * gn[2];
        double G[3];
        for (int k = 0; k < 3; ++k) G[k] = gw[i] * nu[k] * 0.5 + (gn[k] - nu[k] * ndg) / len;
        double g1[3] = {e2[1] * G[2] - e2[2] * G[1], e2[2] * G[0] - e2[0] * G[2], e2[0] * G[1] - e2[1] * G[0]};
        double g2[3] = {G[1] * e1[2] - G[2] * e1[1], G[2] * e1[0] - G[0] * e1[2], G[0] * e1[1] - G[1] * e1[0]};
        for (int k = 0; k < 3; ++k) {
            double gc = gx[3 * i + k] / 3.0;
            grad[3 * i0 + k] += c * (gc - g1[k] - g2[k]);
            grad[3 * i1 + k] += c * (gc + g1[k]);
            grad[3 * i2 + k] += c * (gc + g2[k]);
        }
    }
}

/* ------------------------------------------------------------ LBVH */

typedef struct {
    uint64_t key;
} okey;

static int cmp_key(const void* a, const void* b) {
    uint64_t x = ((const okey*)a)->key, y = ((const okey*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static uint32_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz, int bits) {
    uint32_t code = 0;
    for (int i = bits - 1; i >= 0; --i) {
        code = (code << 1) | ((qx >> i) & 1u);
        code = (code << 1) | ((qy >> i) & 1u);
        code = (code << 1) | ((qz >> i) & 1u);
    }
    return code;
}

/*
 * Morton codes, sorted order and the binary radix tree of the sorted keys.
 *
 * Quantisation (all FP64, round to nearest): lo/hi are the exact per-axis
 * extremes of the centroids, s_a = 2^b / (hi_a - lo_a) (0 for a flat axis),
 * q_a = min(2^b - 1, floor((x_a - lo_a) * s_a)); code interleaves the bits
 * with x most significant in each triplet; key = code << 32 | T.
 *
 * The tree is the radix tree (Patricia trie) of the distinct sorted keys:
 * the node covering sorted positions [i, j] splits after the last position
 * whose key has a 0 at the highest bit where key_i and key_j differ.
 * Node ids: internal nodes 0..n-2, the one covering [i, j] being numbered
 * by the endpoint it shares with its parent's split (the root is 0), i.e.
 * a left child [i, g] is node g and a right child [g+1, j] is node g+1;
 * sorted position k is node (n-1)+k.  Cluster leaves are the nodes with at
 * most leaf_size primitives whose parent has more.
 */
int or_lbvh(const double* x, int64_t n, int morton_bits, int leaf_size,
            uint32_t* codes, int32_t* perm, int32_t* left, int32_t* right, int32_t* parent,
            int32_t* first, int32_t* last, int32_t* leaves, int64_t* nleaves) {
    if (n < 1 || morton_bits < 3 || morton_bits > 30 || morton_bits % 3 != 0) return 1;
    int b = morton_bits / 3;
    uint32_t Q = 1u << b;
    double lo[3], hi[3], s[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = x[a];
        hi[a] = x[a];
    }
    for (int64_t T = 0; T < n; ++T)
        for (int a = 0; a < 3; ++a) {
            if (x[3 * T + a] < lo[a]) lo[a] = x[3 * T + a];
            if (x[3 * T + a] > hi[a]) hi[a] = x[3 * T + a];
        }
    for (int a = 0; a < 3; ++a) s[a] = hi[a] > lo[a] ? (double)Q / (hi[a] - lo[a]) : 0.0;
    okey* keys = (okey*)malloc((size_t)n * sizeof(okey));
    for (int64_t T = 0; T < n; ++T) {
        uint32_t qa[3];
        for (int a = 0; a < 3; ++a) {
            double t = (x[3 * T + a] - lo[a]) * s[a];
            double f = floor(t);
            qa[a] = f >= (double)(Q - 1) ? Q - 1 : (uint32_t)f;
        }
        codes[T] = interleave3(qa[0], qa[1], qa[2], b);
        keys[T].key = ((uint64_t)codes[T] << 32) | (uint64_t)T;
    }
    qsort(keys, (size_t)n, sizeof(okey), cmp_key);
    for (int64_t k = 0; k < n; ++k) perm[k] = (int32_t)(keys[k].key & 0xffffffffu);

    int64_t nn = 2 * n - 1;
    for (int64_t v = 0; v < nn; ++v) {
        parent[v] = -1;
        if (v < n - 1) left[v] = right[v] = -1;
    }
    for (int64_t k = 0; k < n; ++k) first[n - 1 + k] = last[n - 1 + k] = (int32_t)k;
    if (n > 1) {
        /* explicit stack of (node, i, j) */
        int64_t* st = (int64_t*)malloc((size_t)(3 * (n + 1)) * sizeof(int64_t));
        int64_t sp = 0;
        st[sp++] = 0;
        st[sp++] = 0;
        st[sp++] = n - 1;
        while (sp > 0) {
            int64_t j = st[--sp], i = st[--sp], node = st[--sp];
            first[node] = (int32_t)i;
            last[node] = (int32_t)j;
            uint64_t diff = keys[i].key ^ keys[j].key;
            int hb = 63;
            while (!((diff >> hb) & 1ull)) --hb;
            int64_t g = i;
            while (g + 1 <= j - 1 && !((keys[g + 1].key >> hb) & 1ull)) ++g;
            int64_t lc = (g == i) ? (n - 1 + g) : g;
            int64_t rc = (g + 1 == j) ? (n - 1 + j) : (g + 1);
            left[node] = (int32_t)lc;
            right[node] = (int32_t)rc;
            parent[lc] = (int32_t)node;
            parent[rc] = (int32_t)node;
            if (g != i) {
                st[sp++] = lc;
                st[sp++] = i;
                st[sp++] = g;
            }
            if (g + 1 != j) {
                st[sp++] = rc;
                st[sp++] = g + 1;
                st[sp++] = j;
            }
        }
        free(st);
    }
    /* cluster leaves in ascending order of their first sorted position */
    int64_t m = 0;
    int64_t k = 0;
    while (k < n) {
        /* climb from primitive k to the highest ancestor with <= leaf_size members */
        int64_t v = n - 1 + k;
        while (parent[v] >= 0) {
            int64_t pv = parent[v];
            if ((int64_t)last[pv] - first[pv] + 1 > leaf_size) break;
            v = pv;
        }
        leaves[m++] = (int32_t)v;
        k = (int64_t)last[v] + 1;
    }
    *nleaves = m;
    free(keys);
    return 0;
}

/* Cluster moments per node, bottom-up: a primitive holds its own area w,
 * w*x (3), w*nu (3), (w*nu_a)*nu_b (xx xy xz yy yz zz) and the bounding box
 * of its three vertices; an internal node holds left + right (left first). */
static void mom_node(int64_t v, int64_t n, const double* V, const int32_t* F, const double* x,
                     const double* nu, const double* w, const int32_t* perm, const int32_t* left,
                     const int32_t* right, double* mom, double* box) {
    double* m = mom + 13 * v;
    double* bx = box + 6 * v;
    if (v >= n - 1) {
        int64_t T = perm[v - (n - 1)];
        double wt = w[T];
        m[0] = wt;
        for (int a = 0; a < 3; ++a) m[1 + a] = wt * x[3 * T + a];
        for (int a = 0; a < 3; ++a) m[4 + a] = wt * nu[3 * T + a];
        int o = 7;
        for (int a = 0; a < 3; ++a)
            for (int c = a; c < 3; ++c) m[o++] = (wt * nu[3 * T + a]) * nu[3 * T + c];
        for (int a = 0; a < 3; ++a) {
            double lo = V[3 * (int64_t)F[3 * T] + a], hi = lo;
            for (int k = 1; k < 3; ++k) {
                double t = V[3 * (int64_t)F[3 * T + k] + a];
                if (t < lo) lo = t;
                if (t > hi) hi = t;
            }
            bx[a] = lo;
            bx[3 + a] = hi;
        }
        return;
    }
    int64_t l = left[v], r = right[v];
    mom_node(l, n, V, F, x, nu, w, perm, left, right, mom, box);
    mom_node(r, n, V, F, x, nu, w, perm, left, right, mom, box);
    const double *ml = mom + 13 * l, *mr = mom + 13 * r;
    const double *bl = box + 6 * l, *br = box + 6 * r;
    for (int k = 0; k < 13; ++k) m[k] = ml[k] + mr[k];
    for (int a = 0; a < 3; ++a) {
        bx[a] = bl[a] < br[a] ? bl[a] : br[a];
        bx[3 + a] = bl[3 + a] > br[3 + a] ? bl[3 + a] : br[3 + a];
    }
}

void or_moments(const double* V, const int32_t* F, const double* x, const double* nu, const double* w,
                int64_t n, const int32_t* perm, const int32_t* left, const int32_t* right,
                double* mom, double* box) {
    int64_t root = (n == 1) ? 0 : 0;
    mom_node(root, n, V, F, x, nu, w, perm, left, right, mom, box);
}

/* ------------------------------------------------------------ Barnes-Hut */

/*
 * Admissibility of cluster C for target leaf L (a reading of "as in Yu et
 * al.", Sec. 3.2): the vertex boxes are strictly disjoint along some axis
 * (so no pair sharing a vertex is ever approximated) and
 *     diag(C) < theta * (|X_C - c_L| - diag(L)/2),
 * c_L the centre of L's box, X_C the area-weighted centroid of C.  Every
 * quantity is FP64 with separately rounded operations.
 */
static int admissible(const double* bl, const double* bc, const double* mc, double theta) {
    int disjoint = 0;
    for (int a = 0; a < 3; ++a)
        if (bl[3 + a] < bc[a] || bc[3 + a] < bl[a]) disjoint = 1;
    if (!disjoint) return 0;
    double dl2 = 0.0, dc2 = 0.0, r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double el = bl[3 + a] - bl[a];
        double ec = bc[3 + a] - bc[a];
        double cl = (bl[a] + bl[3 + a]) * 0.5;
        double X = mc[1 + a] / mc[0];
        double t = X - cl;
        dl2 = dl2 + el * el;
        dc2 = dc2 + ec * ec;
        r2 = r2 + t * t;
    }
    double diag_l = sqrt(dl2), diag_c = sqrt(dc2), dist = sqrt(r2);
    double rhs = theta * (dist - 0.5 * diag_l);
    return diag_c < rhs;
}

/* Far-field term of target T against cluster C (monopole with the
 * area-averaged normal, not renormalised): both orderings
 *   e_TC = w_T A |nu_T.(x_T - X)|^q / |x_T - X|^p
 *   e_CT = w_T A |nubar.(X - x_T)|^q / |x_T - X|^p,  nubar = sum(w nu)/A
 * differentiated with respect to T's own w, nu, x (the cluster moments are
 * constants: only the inner integral is clustered, Sec. 3.2). */
static void far_term(const double* x, const double* nu, const double* w, int64_t T, const double* mc,
                     double q, double p, double* gw, double* gnu, double* gx) {
    double A = mc[0];
    double X[3], nb[3], d[3], r2 = 0.0, n1 = 0.0, n2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        X[a] = mc[1 + a] / A;
        nb[a] = mc[4 + a] / A;
        d[a] = x[3 * T + a] - X[a];
        r2 += d[a] * d[a];
    }
    for (int a = 0; a < 3; ++a) {
        n1 += nu[3 * T + a] * d[a];
        n2 += nb[a] * (-d[a]);
    }
    double rp = pow(r2, -0.5 * p), rp2 = rp / r2;
    double a1 = powabs(n1, q), b1 = dpowabs(n1, q);
    double a2 = powabs(n2, q), b2 = dpowabs(n2, q);
    double wT = w[T];
    *gw += A * (a1 + a2) * rp;
    for (int k = 0; k < 3; ++k) {
        gnu[k] += wT * A * b1 * rp * d[k];
        gx[k] += wT * A * (b1 * rp * nu[3 * T + k] - p * a1 * rp2 * d[k]);
        gx[k] += wT * A * (-b2 * rp * nb[k] - p * a2 * rp2 * d[k]);
    }
}

void or_bh_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t n,
                 const int32_t* perm, const int32_t* left, const int32_t* right,
                 const int32_t* first, const int32_t* last, const int32_t* leaves, int64_t nleaves,
                 const double* mom, const double* box, double theta, int leaf_size,
                 double q, double p, int adj, double* gw, double* gnu, double* gx,
                 int64_t* n_near_pairs, int64_t* n_far_terms, int nthreads) {
    int64_t near_tot = 0, far_tot = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads) reduction(+ : near_tot, far_tot)
    for (int64_t li = 0; li < nleaves; ++li) {
        int64_t L = leaves[li];
        const double* bl = box + 6 * L;
        int64_t stack[256];
        int sp = 0;
        stack[sp++] = 0; /* the root (node 0, or the only primitive when n == 1) */
        while (sp > 0) {
            int64_t C = stack[--sp];
            int64_t cnt = (int64_t)last[C] - first[C] + 1;
            if (admissible(bl, box + 6 * C, mom + 13 * C, theta)) {
                for (int64_t k = first[L]; k <= last[L]; ++k) {
                    int64_t T = perm[k];
                    far_term(x, nu, w, T, mom + 13 * C, q, p, gw + T, gnu + 3 * T, gx + 3 * T);
                    ++far_tot;
                }
            } else if (cnt <= leaf_size) {
                for (int64_t k = first[L]; k <= last[L]; ++k) {
                    int64_t T = perm[k];
                    for (int64_t m = first[C]; m <= last[C]; ++m) {
                        int64_t S = perm[m];
                        if (excluded(F, T, S, adj)) continue;
                        pair_grad_gather(x, nu, w, T, S, q, p, gw + T, gnu + 3 * T, gx + 3 * T);
                        ++near_tot;
                    }
                }
            } else {
                /* right first so the left child is visited first */
                stack[sp++] = right[C];
                stack[sp++] = left[C];
            }
        }
    }
    if (n_near_pairs) *n_near_pairs = near_tot;
    if (n_far_terms) *n_far_terms = far_tot;
}
