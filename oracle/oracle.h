/*
 * FP64 CPU oracle for the discrete tangent-point energy (TEST INFRASTRUCTURE).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header or table with
 * the CUDA library; it is the plain definition written out:
 *
 *   Phi = c * sum_{(T,S) ordered, T != S, T and S share no vertex}
 *               w_T w_S |<nu_T, x_T - x_S>|^q / |x_T - x_S|^p
 *
 * with x_T the centroid, nu_T the unit normal and w_T the area of the flat
 * triangle T.  This is Eq. (TP) of Sec. 2.2.2 (alpha = q, 2 alpha = p,
 * alpha = 6 in Sec. 2.2.2), discretised with one centroid point per flat
 * triangle; c stands for the prefactor rho/alpha.
 *
 * Arrays are row-major AoS: V[nv][3], F[nt][3], x/nu[nt][3].
 */
#ifndef TP_ORACLE_H
#define TP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* adjacency modes: 0 = exclude every S sharing >= 1 vertex with T (default);
 *                  1 = exclude only S sharing an edge (>= 2 vertices) with T. */

void or_tri_data(const double* V, const int32_t* F, int64_t nt, double* x, double* nu, double* w);

double or_energy(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                 double q, double p, double c, int adj, int nthreads);

int64_t or_admitted_pairs(const int32_t* F, int64_t nt, int adj, int nthreads);

double or_energy_touching(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                          const uint8_t* in_set, double q, double p, double c, int adj, int nthreads);

void or_tri_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t nt,
                  const int64_t* list, int64_t nlist, double q, double p, int adj,
                  double* gw, double* gnu, double* gx, int nthreads);

void or_adjoint(const double* V, const int32_t* F, const int64_t* list, int64_t nlist,
                const double* gw, const double* gnu, const double* gx, double c, double* grad);

int or_lbvh(const double* x, int64_t n, int morton_bits, int leaf_size,
            uint32_t* codes, int32_t* perm, int32_t* left, int32_t* right, int32_t* parent,
            int32_t* first, int32_t* last, int32_t* leaves, int64_t* nleaves);

void or_moments(const double* V, const int32_t* F, const double* x, const double* nu, const double* w,
                int64_t n, const int32_t* perm, const int32_t* left, const int32_t* right,
                double* mom /* [2n-1][13] */, double* box /* [2n-1][6] */);

void or_bh_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t n,
                 const int32_t* perm, const int32_t* left, const int32_t* right,
                 const int32_t* first, const int32_t* last, const int32_t* leaves, int64_t nleaves,
                 const double* mom, const double* box, double theta, int leaf_size,
                 double q, double p, int adj, double* gw, double* gnu, double* gx,
                 int64_t* n_near_pairs, int64_t* n_far_terms, int nthreads);

/* Cluster-cluster (dual-tree) Barnes-Hut form (oracle_dt.c): returns the
 * energy without c; gw/gnu/gx are overwritten with the per-triangle
 * derivatives (without c).  parent[2n-1] from or_lbvh. */
int or_dt_admissible(const double* bA, const double* mA, const double* bB, const double* mB, double theta);
double or_dt_accum(const double* x, const double* nu, const double* w, const int32_t* F, int64_t n,
                   const int32_t* perm, const int32_t* left, const int32_t* right, const int32_t* parent,
                   const int32_t* first, const int32_t* last, const double* mom, const double* box, double theta,
                   int leaf_size, double q, double p, int adj, double* gw, double* gnu, double* gx,
                   int64_t* n_near_pairs, int64_t* n_far_pairs, int64_t* n_far_represented);

/* Confinement energy, Eq. (TPConf), Sec. 2.2 (oracle_conf.c): evolving surface
 * (x, nu, w)[nt], fixed confining surface (centroids y, areas a)[nk]. */
double or_conf_energy(const double* x, const double* nu, const double* w, int64_t nt, const double* y,
                      const double* a, int64_t nk, double q, double p, double c, int nthreads);

void or_conf_accum(const double* x, const double* nu, const double* w, int64_t nt, const double* y, const double* a,
                   int64_t nk, double q, double p, double* gw, double* gnu, double* gx, int nthreads);

/* Multi-point quadrature form (oracle_quad.c): k points per triangle with
 * barycentric coordinates bary[k][3] and weights om[k] (summing to 1). */
void or_quad_points(const double* V, const int32_t* F, int64_t nt, int k, const double* bary, const double* om,
                    double* x, double* nu, double* w, int32_t* Fq);

void or_quad_adjoint(const double* V, const int32_t* F, int64_t nt, int k, const double* bary, const double* om,
                     const double* gw, const double* gnu, const double* gx, double c, double* grad);

#ifdef __cplusplus
}
#endif
#endif
