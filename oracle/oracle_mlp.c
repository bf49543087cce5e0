/*
 * oracle_mlp.c - FP64 reference of the learned far-field correction
 * (TEST INFRASTRUCTURE ONLY; loaded only by tests, the smoke check and the
 * CPU-baseline leg of the benchmark).
 *
 * The paper has no learned component; this is the reference for the
 * network that corrects the Barnes-Hut monopole far terms (Sec. 3.2 far
 * field: the inner integral over an admissible cluster replaced by averages
 * over the patch).  Everything is the plain definition:
 *
 *   network   24 -> 64 -> 64 -> 64 -> 7, y = W4 g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4,
 *             g(z) = z (1 + tanh(c (z + 0.044715 z^3))) / 2, c = sqrt(2/pi)
 *             (the tanh form of GELU, Hendrycks and Gimpel 2016)
 *   loss      L = sum_i sum_c m_ic (y_ic - t_ic)^2 / sum_i sum_c m_ic
 *   AdamW     m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *             w -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps) + lr wd w
 *   features  24 rotation-invariant numbers of a (target leaf L, cluster C)
 *             pair built from their moments (see or_far_features)
 *   labels    log of exact/monopole for 7 channels of the far term, summed
 *             over the targets of L and the members of C (see or_far_labels)
 *
 * Parameter layout (packed, row-major): W1[64][24] b1[64] W2[64][64] b2[64]
 * W3[64][64] b3[64] W4[7][64] b4[7]  (10,375 numbers).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NI 24
#define NH 64
#define NO 7
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NH * NH)
#define OFF_W4 (OFF_B3 + NH)
#define OFF_B4 (OFF_W4 + NO * NH)
#define NPARAM (OFF_B4 + NO)

#define GELU_C 0.79788456080286535588 /* sqrt(2/pi) */
#define GELU_A 0.044715
static double gelu(double z) { return 0.5 * z * (1.0 + tanh(GELU_C * (z + GELU_A * z * z * z))); }
/* d/dz of the above: (1 + t)/2 + z (1 - t^2) c (1 + 3 a z^2) / 2 */
static double dgelu(double z) {
    const double t = tanh(GELU_C * (z + GELU_A * z * z * z));
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z);
}

int64_t or_mlp_nparam(void) { return NPARAM; }

static void layer(const double* W, const double* b, int nout, int nin, const double* x, double* z) {
    for (int o = 0; o < nout; ++o) {
        double s = b[o];
        for (int i = 0; i < nin; ++i) s += W[o * nin + i] * x[i];
        z[o] = s;
    }
}

/* Y[n][7] = network(X[n][24]) */
void or_mlp_forward(const double* P, int64_t n, const double* X, double* Y) {
    for (int64_t s = 0; s < n; ++s) {
        double z1[NH], h1[NH], z2[NH], h2[NH], z3[NH], h3[NH];
        layer(P + OFF_W1, P + OFF_B1, NH, NI, X + NI * s, z1);
        for (int j = 0; j < NH; ++j) h1[j] = gelu(z1[j]);
        layer(P + OFF_W2, P + OFF_B2, NH, NH, h1, z2);
        for (int j = 0; j < NH; ++j) h2[j] = gelu(z2[j]);
        layer(P + OFF_W3, P + OFF_B3, NH, NH, h2, z3);
        for (int j = 0; j < NH; ++j) h3[j] = gelu(z3[j]);
        layer(P + OFF_W4, P + OFF_B4, NO, NH, h3, Y + NO * s);
    }
}

/* dP += sum over samples of dL/dP given dY[n][7] = dL/dY (back-propagation) */
void or_mlp_backward(const double* P, int64_t n, const double* X, const double* dY, double* dP) {
    for (int64_t s = 0; s < n; ++s) {
        const double* x = X + NI * s;
        double z1[NH], h1[NH], z2[NH], h2[NH], z3[NH], h3[NH];
        layer(P + OFF_W1, P + OFF_B1, NH, NI, x, z1);
        for (int j = 0; j < NH; ++j) h1[j] = gelu(z1[j]);
        layer(P + OFF_W2, P + OFF_B2, NH, NH, h1, z2);
        for (int j = 0; j < NH; ++j) h2[j] = gelu(z2[j]);
        layer(P + OFF_W3, P + OFF_B3, NH, NH, h2, z3);
        for (int j = 0; j < NH; ++j) h3[j] = gelu(z3[j]);
        const double* dy = dY + NO * s;
        double dh3[NH], dz3[NH], dh2[NH], dz2[NH], dh1[NH], dz1[NH];
        /* output layer */
        for (int o = 0; o < NO; ++o) {
            dP[OFF_B4 + o] += dy[o];
            for (int j = 0; j < NH; ++j) dP[OFF_W4 + o * NH + j] += dy[o] * h3[j];
        }
        for (int j = 0; j < NH; ++j) {
            double t = 0.0;
            for (int o = 0; o < NO; ++o) t += P[OFF_W4 + o * NH + j] * dy[o];
            dh3[j] = t;
            dz3[j] = t * dgelu(z3[j]);
        }
        /* layer 3 */
        for (int o = 0; o < NH; ++o) {
            dP[OFF_B3 + o] += dz3[o];
            for (int j = 0; j < NH; ++j) dP[OFF_W3 + o * NH + j] += dz3[o] * h2[j];
        }
        for (int j = 0; j < NH; ++j) {
            double t = 0.0;
            for (int o = 0; o < NH; ++o) t += P[OFF_W3 + o * NH + j] * dz3[o];
            dh2[j] = t;
            dz2[j] = t * dgelu(z2[j]);
        }
        /* layer 2 */
        for (int o = 0; o < NH; ++o) {
            dP[OFF_B2 + o] += dz2[o];
            for (int j = 0; j < NH; ++j) dP[OFF_W2 + o * NH + j] += dz2[o] * h1[j];
        }
        for (int j = 0; j < NH; ++j) {
            double t = 0.0;
            for (int o = 0; o < NH; ++o) t += P[OFF_W2 + o * NH + j] * dz2[o];
            dh1[j] = t;
            dz1[j] = t * dgelu(z1[j]);
        }
        /* layer 1 */
        for (int o = 0; o < NH; ++o) {
            dP[OFF_B1 + o] += dz1[o];
            for (int i = 0; i < NI; ++i) dP[OFF_W1 + o * NI + i] += dz1[o] * x[i];
        }
        (void)dh1;
        (void)dh2;
        (void)dh3;
    }
}

/* weighted mean-square loss and its gradient with respect to Y */
double or_mlp_loss(int64_t n, const double* Y, const double* T, const double* M, double* dY) {
    double msum = 0.0, L = 0.0;
    for (int64_t k = 0; k < n * NO; ++k) msum += M[k];
    if (msum <= 0.0) msum = 1.0;
    for (int64_t k = 0; k < n * NO; ++k) {
        const double r = Y[k] - T[k];
        L += M[k] * r * r;
        if (dY) dY[k] = 2.0 * M[k] * r / msum;
    }
    return L / msum;
}

/* one decoupled-weight-decay Adam step (t = step number, from 1) */
void or_adamw_step(double* w, double* m, double* v, const double* g, int64_t n, double lr, double b1, double b2,
                   double eps, double wd, int t) {
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        w[i] = w[i] - lr * (mh / (sqrt(vh) + eps)) - lr * wd * w[i];
    }
}

/* ------------------------------------------------------------------ */
/* features and labels of (target leaf, cluster) pairs                */

/* Frame of a pair: e1 along D = X_C - X_L, e2 along the part of nubar_C
 * orthogonal to e1 (or, when that vanishes, of the coordinate axis least
 * aligned with e1), e3 = e1 x e2. */
static void pair_frame(const double* D, const double* nbc, double e[3][3]) {
    double r = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    for (int a = 0; a < 3; ++a) e[0][a] = D[a] / r;
    double u[3] = {nbc[0], nbc[1], nbc[2]};
    double p = u[0] * e[0][0] + u[1] * e[0][1] + u[2] * e[0][2];
    for (int a = 0; a < 3; ++a) u[a] -= p * e[0][a];
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (un < 1e-12) {
        int k = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(e[0][a]) < fabs(e[0][k])) k = a;
        for (int a = 0; a < 3; ++a) u[a] = (a == k ? 1.0 : 0.0);
        p = e[0][k];
        for (int a = 0; a < 3; ++a) u[a] -= p * e[0][a];
        un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    for (int a = 0; a < 3; ++a) e[1][a] = u[a] / un;
    e[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    e[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    e[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
}

/* second moment sum(w nu nu^T)/A (packed xx xy xz yy yz zz) in the frame */
static void moment_in_frame(const double* m6, double A, double e[3][3], double* out6) {
    double M[3][3] = {{m6[0], m6[1], m6[2]}, {m6[1], m6[3], m6[4]}, {m6[2], m6[4], m6[5]}};
    int o = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s += e[i][a] * M[a][b] * e[j][b];
            out6[o++] = s / A;
        }
}

/*
 * 24 features of the pair (leaf L, cluster C) from their moments
 * mom = [A, sum w x (3), sum w nu (3), sum w nu nu^T (6)] and boxes:
 *   0 log(r / sqrt(A_C)), 1 log(r / sqrt(A_L)), 2 diag_C / r, 3 diag_L / r,
 *   4-6 nubar_L in the frame, 7-8 nubar_C . e1, nubar_C . e2,
 *   9-14 second normal moment of C / A_C in the frame,
 *   15-20 second normal moment of L / A_L in the frame,
 *   21 |nubar_L|, 22 |nubar_C|, 23 log(A_C / A_L),
 * with r = |X_C - X_L|, X the area-weighted centroids, nubar = sum(w nu)/A.
 */
void or_far_features(const double* momL, const double* boxL, const double* momC, const double* boxC, double* f) {
    double XL[3], XC[3], D[3], nbl[3], nbc[3], e[3][3];
    for (int a = 0; a < 3; ++a) {
        XL[a] = momL[1 + a] / momL[0];
        XC[a] = momC[1 + a] / momC[0];
        D[a] = XC[a] - XL[a];
        nbl[a] = momL[4 + a] / momL[0];
        nbc[a] = momC[4 + a] / momC[0];
    }
    const double r = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    pair_frame(D, nbc, e);
    double dl2 = 0.0, dc2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        dl2 += (boxL[3 + a] - boxL[a]) * (boxL[3 + a] - boxL[a]);
        dc2 += (boxC[3 + a] - boxC[a]) * (boxC[3 + a] - boxC[a]);
    }
    f[0] = log(r / sqrt(momC[0]));
    f[1] = log(r / sqrt(momL[0]));
    f[2] = sqrt(dc2) / r;
    f[3] = sqrt(dl2) / r;
    for (int i = 0; i < 3; ++i) f[4 + i] = nbl[0] * e[i][0] + nbl[1] * e[i][1] + nbl[2] * e[i][2];
    for (int i = 0; i < 2; ++i) f[7 + i] = nbc[0] * e[i][0] + nbc[1] * e[i][1] + nbc[2] * e[i][2];
    moment_in_frame(momC + 7, momC[0], e, f + 9);
    moment_in_frame(momL + 7, momL[0], e, f + 15);
    f[21] = sqrt(nbl[0] * nbl[0] + nbl[1] * nbl[1] + nbl[2] * nbl[2]);
    f[22] = sqrt(nbc[0] * nbc[0] + nbc[1] * nbc[1] + nbc[2] * nbc[2]);
    f[23] = log(momC[0] / momL[0]);
}

/*
 * Channel sums of one (leaf L, cluster C) pair, q = 6 / p = 12 style with
 * lambda = p/q, over the targets T of L (indices tl[nl]) and the members S of
 * C (indices sc[ns]); x, nu, w per triangle (AoS).  With d = x_T - y,
 * al = nu_T.d/|d|^2, be = n.d/|d|^2 (y, n, a the source position, normal,
 * area), wts = lambda w_T a, inv = 1/|d|^2:
 *   ch0 E_TC = wts al^q,   ch1 E_CT = wts be^q,   ch2 U = wts inv al^(q-1),
 *   ch3 Gn = wts inv al^(q-1) d,    ch4 Gx_nu = wts inv be^(q-1) n,
 *   ch5 k_TC = lambda wts inv al^q d,   ch6 k_CT = lambda wts inv be^q d.
 * mono[7]: the monopole (y = X_C, n = nubar_C, a = A_C) summed over T, the
 * vector channels projected on the monopole's own direction (|d| for 3, 5,
 * 6 and |nubar_C| for 4);  exact[7]: the member sums, vector channels
 * projected on the monopole unit directions (d_TC/|d_TC|, nubar_C/|nubar_C|).
 */
void or_far_channels(const double* x, const double* nu, const double* w, const int64_t* tl, int64_t nl,
                     const int64_t* sc, int64_t ns, const double* momC, double q, double p, double* mono,
                     double* exact) {
    const double lam = p / q;
    double XC[3], nbc[3];
    for (int a = 0; a < 3; ++a) {
        XC[a] = momC[1 + a] / momC[0];
        nbc[a] = momC[4 + a] / momC[0];
    }
    const double nbn = sqrt(nbc[0] * nbc[0] + nbc[1] * nbc[1] + nbc[2] * nbc[2]);
    for (int c = 0; c < 7; ++c) mono[c] = exact[c] = 0.0;
    for (int64_t i = 0; i < nl; ++i) {
        const int64_t T = tl[i];
        double d[3], r2 = 0.0, a = 0.0, b = 0.0;
        for (int k = 0; k < 3; ++k) {
            d[k] = x[3 * T + k] - XC[k];
            r2 += d[k] * d[k];
        }
        for (int k = 0; k < 3; ++k) {
            a += nu[3 * T + k] * d[k];
            b += nbc[k] * d[k];
        }
        const double inv = 1.0 / r2, al = a * inv, be = b * inv, rn = sqrt(r2);
        const double wts = lam * w[T] * momC[0];
        double dhat[3] = {d[0] / rn, d[1] / rn, d[2] / rn};
        mono[0] += wts * pow(al, q);
        mono[1] += wts * pow(be, q);
        mono[2] += wts * inv * pow(al, q - 1.0);
        mono[3] += wts * inv * pow(al, q - 1.0) * rn;
        mono[4] += wts * inv * pow(be, q - 1.0) * nbn;
        mono[5] += lam * wts * inv * pow(al, q) * rn;
        mono[6] += lam * wts * inv * pow(be, q) * rn;
        double e3 = 0.0, e4 = 0.0, e5 = 0.0, e6 = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            const int64_t S = sc[j];
            double ds[3], s2 = 0.0, as = 0.0, bs = 0.0;
            for (int k = 0; k < 3; ++k) {
                ds[k] = x[3 * T + k] - x[3 * S + k];
                s2 += ds[k] * ds[k];
            }
            for (int k = 0; k < 3; ++k) {
                as += nu[3 * T + k] * ds[k];
                bs += nu[3 * S + k] * ds[k];
            }
            const double iv = 1.0 / s2, als = as * iv, bes = bs * iv;
            const double wt = lam * w[T] * w[S];
            exact[0] += wt * pow(als, q);
            exact[1] += wt * pow(bes, q);
            exact[2] += wt * iv * pow(als, q - 1.0);
            double pd = ds[0] * dhat[0] + ds[1] * dhat[1] + ds[2] * dhat[2];
            double pn = (nu[3 * S] * nbc[0] + nu[3 * S + 1] * nbc[1] + nu[3 * S + 2] * nbc[2]) / nbn;
            e3 += wt * iv * pow(als, q - 1.0) * pd;
            e4 += wt * iv * pow(bes, q - 1.0) * pn;
            e5 += lam * wt * iv * pow(als, q) * pd;
            e6 += lam * wt * iv * pow(bes, q) * pd;
        }
        exact[3] += e3;
        exact[4] += e4;
        exact[5] += e5;
        exact[6] += e6;
    }
}
