// tp_dual.cu - cluster-cluster (dual-tree) Barnes-Hut form (TP_BH_DUAL).
//
// Sec. 3.2 clusters only the inner integral (tp_bh.cu); its comparison
// method clusters both.  This form does the latter on the same LBVH and
// moments:
//   - every unordered pair of triangles belongs to exactly one unordered pair
//     of tree nodes {A, B}, found by the recursion from (root, root):
//       A == B: a node of at most leaf_size members (or a primitive) is a
//               near self pair, otherwise (l, l), (r, r), (l, r);
//       A != B: admissible -> far pair; both nodes of at most leaf_size
//               members -> near pair; otherwise the node with more members
//               is split (a node of at most leaf_size members never is);
//     so every node in a near pair is a cluster leaf;
//   - admissible: vertex boxes strictly apart along some axis and
//     max(diag_A, diag_B) < theta |X_A - X_B| (X the area-weighted centroid),
//     in FP64 with separately rounded operations in a fixed order, so the
//     decisions equal the oracle's;
//   - a far pair contributes the cluster monopole of both orderings,
//     A_A A_B (|nubar_A.(X_A - X_B)|^q + |nubar_B.(X_B - X_A)|^q) / |X_A - X_B|^p,
//     a near pair its admitted member pairs exactly;
//   - the gradient is the exact derivative of this energy: a far pair's
//     derivatives with respect to each node's (A, X, nubar) are summed per
//     node and passed down to the member triangles through
//     A = sum w, X = sum w x / A, nubar = sum w nu / A.
//
// GPU organisation:
//   k_dt_expand   one level of the recursion: every node pair of the
//                 frontier is classified (far, near, or split into the next
//                 frontier); lists grow by warp-aggregated atomics and the
//                 host repeats the traversal with larger lists on overflow.
//                 The test reads the tree build's node records (FP64 centroid
//                 quotients and diagonals, outward/inward-rounded FP32 boxes):
//                 an FP32 test with a safety margin decides unless the case
//                 is close, which goes to FP64 on the same quantities as the
//                 oracle.  Several levels run per host synchronisation (each
//                 launch reads its frontier size from device memory);
//   k_dt_far      far terms in FP32 from the records (no division), one
//                 thread per far pair, node derivatives summed with FP64
//                 atomics;
//   k_dt_count/k_dt_fill/k_dt_runs  per cluster leaf, its near partners
//                 (both directions of each near pair) as (first member,
//                 count) in two lists: partners whose FP32 outward vertex box
//                 touches the leaf's (the leaf itself among them) and the
//                 others, the latter cut into runs of at most 128;
//   k_dt_near     one warp per cluster leaf gathers both orderings of every
//                 admitted pair with its touching partners' members (packed
//                 FP32x2, exclusion test on every pair) and stores the leaf's
//                 accumulators (direct kernels' layout); the apart partners
//                 go to the Barnes-Hut near-field kernel (k_near, tp_bh.cu),
//                 which needs no exclusion test and adds with atomics;
//   k_dt_node     per node, the derivatives divided by A and the weight term;
//   k_dt_down     per triangle, the sum over its ancestors added to its
//                 accumulators (Ew += (p/q) w gw, Gn += (p/q)/q gnu,
//                 Gx += (p/q)/q gx), so the direct kernels' adjoint and
//                 energy reduction (Phi = c/2 sum w dPhi/dw: the energy is
//                 homogeneous of degree 2 in the weights) apply unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"
#include "tp_pair_dev.cuh"

namespace {

constexpr int DT_THREADS = 256;
constexpr int DT_NEAR_WARPS = 4;

struct DTTree {
    const int32_t* left;
    const int32_t* right;
    const int32_t* parent;
    const int32_t* first;
    const int32_t* last;
    const int32_t* perm;
    const double* mom;    // [nn][13]
    const double* box;    // [nn][6]
    const double* adm64;  // [nn][4] X (FP64 quotients), diagonal
    const float* adm32;   // [nn][TP_ADM32_W] outward box, X, diagonal (FP32), range, children
    const float* nodef;   // [nn][16] FP32 far-field record (nubar at 6..8)
    int64_t n;
    int leaf;
    unsigned* derr;  // device error word (bounds checks of the TP_DEBUG build)
};

__device__ __forceinline__ bool dt_small(const DTTree& T, int node) {
    return node >= T.n - 1 || (T.last[node] - T.first[node] + 1) <= T.leaf;
}

// Admissibility of {A, B}: vertex boxes strictly apart along some axis and
// max(diag_A, diag_B) < theta |X_A - X_B|.  The FP32 records decide when they
// can: outward-rounded boxes apart -> apart, inward-rounded boxes overlapping
// on every axis -> not apart, the size test outside a 1e-5 relative margin
// (far above the FP32 rounding of the records and of the distance); the other
// cases use FP64 boxes, centroid quotients and diagonals (the oracle's values
// and operations: sqrt(max(dA2, dB2)) = max(sqrt dA2, sqrt dB2) exactly).
__device__ bool dt_admissible(const DTTree& T, int A, int B, double theta, float theta32) {
    const float* cA = T.adm32 + TP_ADM32_W * (int64_t)A;
    const float* cB = T.adm32 + TP_ADM32_W * (int64_t)B;
    bool sure = false, amb = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (cA[3 + a] < cB[a] || cB[3 + a] < cA[a]) sure = true;
        else if (!(tp_inward_hi(cA[3 + a]) >= tp_inward_lo(cB[a]) && tp_inward_hi(cB[3 + a]) >= tp_inward_lo(cA[a])))
            amb = true;
    }
    if (!sure) {
        if (!amb) return false;
        const double* bA = T.box + 6 * (int64_t)A;
        const double* bB = T.box + 6 * (int64_t)B;
        bool disjoint = false;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (bA[3 + a] < bB[a] || bB[3 + a] < bA[a]) disjoint = true;
        if (!disjoint) return false;
    }
    float r2f = 0.f, M = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t = cA[6 + a] - cB[6 + a];
        r2f = fmaf(t, t, r2f);
        M += fabsf(cA[6 + a]) + fabsf(cB[6 + a]);
    }
    const float distf = sqrtf(r2f);
    const float lhsf = fmaxf(cA[9], cB[9]);
    const float rhsf = theta32 * distf;
    const float margin = 1e-5f * (lhsf + theta32 * (distf + M));
    if (lhsf < rhsf - margin) return true;
    if (lhsf > rhsf + margin) return false;
    const double* aA = T.adm64 + 4 * (int64_t)A;
    const double* aB = T.adm64 + 4 * (int64_t)B;
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = __dsub_rn(aA[a], aB[a]);
        r2 = __dadd_rn(r2, __dmul_rn(t, t));
    }
    const double diag = aA[3] > aB[3] ? aA[3] : aB[3];
    return diag < __dmul_rn(theta, __dsqrt_rn(r2));
}

// FP32 outward-rounded vertex boxes strictly apart along some axis: no member
// of A shares a vertex with a member of B
__device__ __forceinline__ bool dt_boxes_apart(const DTTree& T, int A, int B) {
    const float* cA = T.adm32 + TP_ADM32_W * (int64_t)A;
    const float* cB = T.adm32 + TP_ADM32_W * (int64_t)B;
    bool apart = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (cA[3 + a] < cB[a] || cB[3 + a] < cA[a]) apart = true;
    return apart;
}

// Reserve cnt (>= 0) slots of a list for every lane of a warp with one atomic;
// returns this lane's first slot.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned cnt, unsigned long long* counter) {
    const int lane = threadIdx.x & 31;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (incl - cnt);
}

// One level of the pair recursion.  cnt[0] frontier in, cnt[1] frontier out,
// cnt[2] far, cnt[3] near; an append past a capacity sets cnt[4].
// The frontier size is read from n_in_p (the previous level's output count);
// a level whose input overflowed its list (cnt[4] set) does nothing.
__global__ void __launch_bounds__(DT_THREADS) k_dt_expand(DTTree T, double theta, const int2* __restrict__ fin,
                                                          const unsigned long long* __restrict__ n_in_p,
                                                          int64_t cap_in, int2* __restrict__ fout,
                                                          unsigned long long* __restrict__ n_out_p, int64_t cap_out,
                                                          int2* __restrict__ far, int64_t cap_far,
                                                          int2* __restrict__ near, int64_t cap_near,
                                                          unsigned long long* __restrict__ cnt) {
    if (cnt[4]) return;
    const int64_t n_in = (int64_t)*n_in_p < cap_in ? (int64_t)*n_in_p : cap_in;
    const float theta32 = (float)theta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t rounds = (n_in + stride - 1) / stride;
    for (int64_t r = 0; r < rounds; ++r) {  // uniform trip count: every lane reaches the warp reservations
        const int64_t i = r * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        int kind = -1;  // 0 near, 1 far, 2 split A, 3 split B, 4 split self
        int A = 0, B = 0;
        if (i < n_in) {
            const int2 pr = fin[i];
            A = pr.x;
            B = pr.y;
            const bool sA = dt_small(T, A), sB = dt_small(T, B);
            if (A == B) {
                kind = sA ? 0 : 4;
            } else if (dt_admissible(T, A, B, theta, theta32)) {
                kind = 1;
            } else if (sA && sB) {
                kind = 0;
            } else {
                const int cA = T.last[A] - T.first[A], cB = T.last[B] - T.first[B];
                kind = (!sA && (cA >= cB || sB)) ? 2 : 3;
            }
        }
        const unsigned n_out = kind == 4 ? 3u : (kind == 2 || kind == 3) ? 2u : 0u;
        const unsigned long long po = warp_reserve(n_out, n_out_p);
        const unsigned long long pf = warp_reserve(kind == 1 ? 1u : 0u, &cnt[2]);
        const unsigned long long pn = warp_reserve(kind == 0 ? 1u : 0u, &cnt[3]);
        if (kind == 1) {
            if ((int64_t)pf < cap_far) far[pf] = make_int2(A, B);
            else cnt[4] = 1ull;
        } else if (kind == 0) {
            if ((int64_t)pn < cap_near) near[pn] = make_int2(A, B);
            else cnt[4] = 1ull;
        } else if (n_out) {
            if ((int64_t)(po + n_out) <= cap_out) {
                if (kind == 4) {
                    const int l = T.left[A], rr = T.right[A];
                    fout[po] = make_int2(l, l);
                    fout[po + 1] = make_int2(rr, rr);
                    fout[po + 2] = make_int2(l, rr);
                } else if (kind == 2) {
                    fout[po] = make_int2(T.left[A], B);
                    fout[po + 1] = make_int2(T.right[A], B);
                } else {
                    fout[po] = make_int2(A, T.left[B]);
                    fout[po + 1] = make_int2(A, T.right[B]);
                }
            } else {
                cnt[4] = 1ull;
            }
        }
    }
}

// Far pairs: the monopole of both orderings in FP32 from the records (X_A -
// X_B formed in FP64 from the centroid quotients, then rounded; nubar from the
// far-field record), the node derivatives dE/d(A, X[3], nubar[3]) of both
// nodes summed into G[node][7] with FP64 atomics; the represented ordered
// pairs into *rep.
__global__ void __launch_bounds__(DT_THREADS) k_dt_far(DTTree T, const int2* __restrict__ far, int64_t nfar, int q,
                                                       double* __restrict__ G, unsigned long long* __restrict__ rep) {
    unsigned long long my_rep = 0;
    const float pf = 2.0f * (float)q;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfar; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 pr = far[i];
        if (!tp_dbg_ok(pr.x >= 0 && pr.x < 2 * T.n - 1 && pr.y >= 0 && pr.y < 2 * T.n - 1, T.derr)) continue;
        const double* xA = T.adm64 + 4 * (int64_t)pr.x;
        const double* xB = T.adm64 + 4 * (int64_t)pr.y;
        const float* fA = T.nodef + 16 * (int64_t)pr.x;
        const float* fB = T.nodef + 16 * (int64_t)pr.y;
        const float AA = (float)T.mom[13 * (int64_t)pr.x], AB = (float)T.mom[13 * (int64_t)pr.y];
        const float nA[3] = {fA[6], fA[7], fA[8]}, nB[3] = {fB[6], fB[7], fB[8]};
        float d[3], r2 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[a] = (float)(xA[a] - xB[a]);
            r2 = fmaf(d[a], d[a], r2);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            n1 = fmaf(nA[a], d[a], n1);
            n2 = fmaf(-nB[a], d[a], n2);
        }
        // with al = n1 / |d|^2 and be = n2 / |d|^2, n^q |d|^-p = al^q (p = 2q): no
        // power of |d| alone, so nothing overflows for small clusters at large theta
        const float inv = 1.0f / r2, al = n1 * inv, be = n2 * inv;
        float al1 = 1.f, be1 = 1.f;  // al^(q-1), be^(q-1)
        for (int e = 0; e < q - 1; ++e) {
            al1 *= al;
            be1 *= be;
        }
        const float AAB = AA * AB, s = al1 * al + be1 * be;  // al^q + be^q
        const float qa = (float)q * al1 * inv, qb = (float)q * be1 * inv;
        double* GA = G + 7 * (int64_t)pr.x;
        double* GB = G + 7 * (int64_t)pr.y;
        atomicAdd(&GA[0], (double)(AB * s));
        atomicAdd(&GB[0], (double)(AA * s));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float gX = AAB * (qa * nA[k] - qb * nB[k] - pf * s * inv * d[k]);
            atomicAdd(&GA[1 + k], (double)gX);
            atomicAdd(&GB[1 + k], (double)-gX);
            atomicAdd(&GA[4 + k], (double)(AAB * qa * d[k]));
            atomicAdd(&GB[4 + k], (double)(-AAB * qb * d[k]));
        }
        my_rep += 2ull * (unsigned long long)(T.last[pr.x] - T.first[pr.x] + 1) *
                  (unsigned long long)(T.last[pr.y] - T.first[pr.y] + 1);
    }
    for (int o = 16; o > 0; o >>= 1) my_rep += __shfl_xor_sync(0xffffffffu, my_rep, o);
    if ((threadIdx.x & 31) == 0 && my_rep) atomicAdd(rep, my_rep);
}

__global__ void k_dt_leaf_index(const int32_t* __restrict__ leaves, int64_t nleaves, int32_t* __restrict__ node2leaf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nleaves) node2leaf[leaves[i]] = (int32_t)i;
}

// partners per cluster leaf, both directions of every near pair (a self pair
// once): touching partners counted in ct[leaf], apart ones in ca[leaf]
// (the ordered member pairs of the apart node pairs, all admitted, into *apart_pairs)
__global__ void k_dt_count(DTTree T, const int2* __restrict__ near, int64_t nnear,
                           const int32_t* __restrict__ node2leaf, uint32_t* __restrict__ ct,
                           uint32_t* __restrict__ ca, unsigned long long* __restrict__ apart_pairs, unsigned* derr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long np = 0;
    if (i < nnear) {
        const int2 pr = near[i];
        const int la = node2leaf[pr.x], lb = node2leaf[pr.y];
        if (la < 0 || lb < 0) {  // a near node that is not a cluster leaf: the recursion's invariant failed
            tp_dev_error(derr, TP_DERR_INTERNAL);
        } else if (pr.x == pr.y) {
            atomicAdd(&ct[la], 1u);
        } else if (dt_boxes_apart(T, pr.x, pr.y)) {
            atomicAdd(&ca[la], 1u);
            atomicAdd(&ca[lb], 1u);
            np = 2ull * (unsigned long long)(T.last[pr.x] - T.first[pr.x] + 1) *
                 (unsigned long long)(T.last[pr.y] - T.first[pr.y] + 1);
        } else {
            atomicAdd(&ct[la], 1u);
            atomicAdd(&ct[lb], 1u);
        }
    }
    for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
    if ((threadIdx.x & 31) == 0 && np) atomicAdd(apart_pairs, np);
}

__global__ void k_dt_fill(DTTree T, const int2* __restrict__ near, int64_t nnear,
                          const int32_t* __restrict__ node2leaf, const uint32_t* __restrict__ ot,
                          const uint32_t* __restrict__ oa, uint32_t* __restrict__ kt, uint32_t* __restrict__ ka,
                          int2* __restrict__ lt, int2* __restrict__ lap) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnear) return;
    const int2 pr = near[i];
    const int la = node2leaf[pr.x], lb = node2leaf[pr.y];
    if (la < 0 || lb < 0) return;
    const int2 eB = make_int2(T.first[pr.y], T.last[pr.y] - T.first[pr.y] + 1);
    if (pr.x == pr.y) {
        lt[ot[la] + atomicAdd(&kt[la], 1u)] = eB;
        return;
    }
    const int2 eA = make_int2(T.first[pr.x], T.last[pr.x] - T.first[pr.x] + 1);
    if (dt_boxes_apart(T, pr.x, pr.y)) {
        lap[oa[la] + atomicAdd(&ka[la], 1u)] = eB;
        lap[oa[lb] + atomicAdd(&ka[lb], 1u)] = eA;
    } else {
        lt[ot[la] + atomicAdd(&kt[la], 1u)] = eB;
        lt[ot[lb] + atomicAdd(&kt[lb], 1u)] = eA;
    }
}

constexpr int DT_RUN = TP_BH_NEAR;  // apart partners per run of the near-field kernel

__global__ void k_dt_runcount(const uint32_t* __restrict__ ca, int64_t nl, uint32_t* __restrict__ nr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nl) nr[i] = (ca[i] + DT_RUN - 1) / DT_RUN;
}

__global__ void k_dt_runs(const uint32_t* __restrict__ ca, const uint32_t* __restrict__ oa,
                          const uint32_t* __restrict__ orr, int64_t nl, tp_far_run* __restrict__ runs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const uint32_t n = ca[i];
    for (uint32_t j = 0; j * DT_RUN < n; ++j) {
        tp_far_run r;
        r.start = (int64_t)oa[i] + (int64_t)j * DT_RUN;
        r.li = (int32_t)i;
        r.len = (int32_t)min((uint32_t)DT_RUN, n - j * DT_RUN);
        runs[orr[i] + j] = r;
    }
}

__global__ void k_dt_setcount(const int32_t* __restrict__ total, unsigned long long* __restrict__ counter) {
    *counter = (unsigned long long)*total;
}

// One warp per cluster leaf: both orderings of every admitted pair of its
// targets with its touching partners' members, gathered on the target side.
template <int Q>
__global__ void __launch_bounds__(DT_NEAR_WARPS * 32) k_dt_near(const float* __restrict__ soa, int64_t ntp,
                                                                const int32_t* __restrict__ Fs,
                                                                const int32_t* __restrict__ leaves, int64_t nleaves,
                                                                const int32_t* __restrict__ first,
                                                                const int32_t* __restrict__ last, int wide,
                                                                const uint32_t* __restrict__ off,
                                                                const int2* __restrict__ list, int edge_only,
                                                                double* __restrict__ acc,
                                                                unsigned long long* __restrict__ npairs,
                                                                unsigned* __restrict__ derr) {
    __shared__ __align__(16) float s_stg[DT_NEAR_WARPS][16 * BH_PAIR];
    __shared__ int4 s_f[DT_NEAR_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t li = (int64_t)blockIdx.x * DT_NEAR_WARPS + warp;
    if (li >= nleaves) return;
    float* stg = s_stg[warp];
    int4* sf = s_f[warp];
    const int64_t L = leaves[li];
    const int64_t fL = first[L];
    const int cnt = last[L] - first[L] + 1;
    wide = wide && cnt > 16;  // a leaf of up to 16 targets takes two lanes per target in any tree
    const int t = wide ? lane : (lane & 15), half = wide ? 0 : (lane >> 4), nh = wide ? 1 : 2;
    const int64_t k = fL + t;
    const bool active = t < cnt;
    Tgt2 tg;
    int3 tf = make_int3(-2, -2, -2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        tg.h[c] = bh_f2(active ? soa[c * ntp + k] : 0.f);
        tg.l[c] = bh_f2(active ? soa[(3 + c) * ntp + k] : 0.f);
        tg.n[c] = bh_f2(active ? soa[(6 + c) * ntp + k] : 0.f);
    }
    tg.w = bh_f2(active ? soa[9 * ntp + k] : 0.f);
    if (active) tf = make_int3(Fs[3 * k], Fs[3 * k + 1], Fs[3 * k + 2]);
    // the target's sums over the batches: compensated FP32 (value as_ - ac)
    float as_[8], ac[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) as_[c] = ac[c] = 0.f;
    unsigned long long n_adm = 0;
    const uint32_t e0 = off[li], e1 = off[li + 1];
#if TP_DEBUG
    {
        // the leaf's targets and every listed partner range within the triangles
        bool ok = fL >= 0 && cnt >= 1 && cnt <= 32 && fL + cnt <= ntp;
        for (uint32_t j = e0 + lane; j < e1; j += 32) {
            const int2 nd = list[j];
            ok = ok && nd.y >= 1 && nd.y <= 32 && nd.x >= 0 && (int64_t)nd.x + nd.y <= ntp;
        }
        if (!__all_sync(0xffffffffu, tp_dbg_ok(ok, derr))) return;
    }
#else
    (void)derr;
#endif
    uint32_t e = e0;
    while (e < e1) {
        // whole partner leaves while they fit in 32 staging slots
        int nsrc = 0;
        uint32_t e2 = e;
        while (e2 < e1 && nsrc + list[e2].y <= 32) nsrc += list[e2++].y;
        __syncwarp();
        int base = 0;
        for (uint32_t j = e; j < e2; ++j) {
            const int2 nd = list[j];
            if (lane >= base && lane < base + nd.y) {
                const int64_t s = (int64_t)nd.x + (lane - base);
                float v[10];
#pragma unroll
                for (int c = 0; c < 10; ++c) v[c] = soa[c * ntp + s];
                stage_put(stg, lane, v);
                sf[lane] = make_int4(Fs[3 * s], Fs[3 * s + 1], Fs[3 * s + 2], (int)s);
            }
            base += nd.y;
        }
        if (lane == nsrc && (nsrc & 1)) {
            stage_pad(stg, lane);
            sf[lane] = make_int4(-1, -1, -1, -1);
        }
        __syncwarp();
        float2 a2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
        const int np = (nsrc + 1) >> 1;
        for (int pp = half; pp < np; pp += nh) {
            const int4 f0 = sf[2 * pp], f1 = sf[2 * pp + 1];
            const bool v0 = active && f0.w >= 0 && f0.w != (int)k && !adjacent(tf, make_int3(f0.x, f0.y, f0.z), edge_only);
            const bool v1 = active && f1.w >= 0 && f1.w != (int)k && !adjacent(tf, make_int3(f1.x, f1.y, f1.z), edge_only);
            gather_pair2<Q, true>(tg, stg, pp, a2, v0, v1);
            n_adm += (unsigned long long)(v0 + v1);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) ksum_add(as_[c], ac[c], a2[c].x + a2[c].y);
        e = e2;
    }
    double a64[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a64[c] = (double)as_[c] - (double)ac[c];
    if (!wide) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a64[c] += __shfl_xor_sync(0xffffffffu, a64[c], 16);
    }
    if (half == 0 && active) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c * ntp + k] = a64[c];
    }
    for (int o = 16; o > 0; o >>= 1) n_adm += __shfl_xor_sync(0xffffffffu, n_adm, o);
    if (lane == 0 && n_adm) atomicAdd(npairs, n_adm);
}

// Per node: dE/dX / A, dE/dnubar / A, and dE/dA - (dE/dX.X + dE/dnubar.nubar) / A.
__global__ void k_dt_node(const double* __restrict__ G, const double* __restrict__ mom, int64_t nn,
                          double* __restrict__ P) {
    const int64_t N = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (N >= nn) return;
    const double* g = G + 7 * N;
    double gv[7];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        gv[c] = g[c];
        any = any || gv[c] != 0.0;
    }
    if (!any) {  // a node in no far pair (most of them): nothing to pass down
#pragma unroll
        for (int c = 0; c < 7; ++c) P[7 * N + c] = 0.0;
        return;
    }
    const double* m = mom + 13 * N;
    const double ia = 1.0 / m[0];
    double s = gv[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P[7 * N + 1 + a] = gv[1 + a] * ia;
        P[7 * N + 4 + a] = gv[4 + a] * ia;
        s -= (gv[1 + a] * (m[1 + a] * ia) + gv[4 + a] * (m[4 + a] * ia)) * ia;
    }
    P[7 * N] = s;
}

// Per triangle (library position k): the sum of P over the nodes holding it,
// turned into its far-field derivatives and added to its accumulators.
__global__ void k_dt_down(const int32_t* __restrict__ parent, const int32_t* __restrict__ perm, int64_t n,
                          const double* __restrict__ P, const double* __restrict__ x64,
                          const double* __restrict__ nu64, const double* __restrict__ w64, int64_t ntp, double pq,
                          double q, double* __restrict__ acc) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double S[7] = {0, 0, 0, 0, 0, 0, 0};
    int64_t N = n > 1 ? n - 1 + k : 0;
    for (int depth = 0; depth < 4096; ++depth) {
#pragma unroll
        for (int c = 0; c < 7; ++c) S[c] += P[7 * N + c];
        if (N == 0) break;
        N = parent[N];
        if (N < 0) break;
    }
    const int64_t T = perm[k];
    const double w = w64[T];
    double gw = S[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) gw += x64[a * n + T] * S[1 + a] + nu64[a * n + T] * S[4 + a];
    acc[k] += pq * w * gw;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[(2 + a) * ntp + k] += pq / q * w * S[4 + a];
        acc[(5 + a) * ntp + k] += pq / q * w * S[1 + a];
    }
}

inline unsigned dt_blocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

tp_status tp_launch_dual(tp_ctx* ctx, const tp_params* prm) {
    TpRange nvtx_range("tp_launch_dual");
    TP_TRY(tp_ensure_sorted(ctx));
    tp_tree& t = ctx->tree;
    if (t.leaf_size > 32) return tp_set_err(ctx, TP_E_ARG, "leaf_size above 32");
    const int64_t n = ctx->nt, nn = 2 * n - 1;
    DTTree T;
    T.left = t.left;
    T.right = t.right;
    T.parent = t.parent;
    T.first = t.first;
    T.last = t.last;
    T.perm = ctx->perm;
    T.mom = t.mom;
    T.box = t.box;
    T.adm64 = t.adm64;
    T.adm32 = t.adm32;
    T.nodef = t.nodef;
    T.n = n;
    T.leaf = t.leaf_size;
    T.derr = ctx->derr;
    // counters: [2] far pairs, [3] near pairs, [4] overflow, [5] admitted pairs of the
    // touching pass, [6] represented far pairs, [7] pairs of the apart node pairs,
    // [9] runs and [10] work counter of the near-field kernel; from [16] the frontier
    // sizes of DT_LEVELS levels
    constexpr int DT_LEVELS = 4096, DT_SYNC = 8;
    if (!ctx->dt_cnt) TP_TRY(tp_alloc_t(ctx, &ctx->dt_cnt, 16 + DT_LEVELS));
    unsigned long long* cnt = ctx->dt_cnt;
    unsigned long long* fsize = cnt + 16;
    if (ctx->dt_cap == 0) {
        const int64_t c0 = std::max<int64_t>(1 << 16, 64 * t.nleaves);
        TP_TRY(tp_dual_lists(ctx, c0, c0, c0));
    }
    cudaEventRecord(ctx->ev[0], ctx->stream);
    int64_t n_far = 0, n_near = 0;
    const unsigned eblocks = (unsigned)std::max(1, 8 * ctx->num_sms);
    for (int attempt = 0;; ++attempt) {
        // the traversal from (root, root), DT_SYNC levels per host synchronisation
        const int2 root = make_int2(0, 0);
        const unsigned long long one = 1ull;
        TP_CU(cudaMemcpyAsync(ctx->dt_front[0], &root, sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
        TP_CU(cudaMemsetAsync(cnt, 0, (16 + DT_LEVELS) * sizeof(unsigned long long), ctx->stream));
        TP_CU(cudaMemcpyAsync(fsize, &one, sizeof(one), cudaMemcpyHostToDevice, ctx->stream));
        unsigned long long h[5] = {0, 0, 0, 0, 0}, last = 1;
        bool done = false;
        for (int level = 0; level < DT_LEVELS - 1 && !done;) {
            for (int k = 0; k < DT_SYNC && level < DT_LEVELS - 1; ++k, ++level)
                k_dt_expand<<<eblocks, DT_THREADS, 0, ctx->stream>>>(
                    T, prm->theta, ctx->dt_front[level & 1], fsize + level, ctx->dt_cap, ctx->dt_front[(level + 1) & 1],
                    fsize + level + 1, ctx->dt_cap, ctx->dt_far, ctx->dt_far_cap, ctx->dt_near, ctx->dt_near_cap, cnt);
            ctx->nlaunch += DT_SYNC;
            TP_CU(cudaMemcpyAsync(h, cnt, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
            TP_CU(cudaMemcpyAsync(&last, fsize + level, sizeof(last), cudaMemcpyDeviceToHost, ctx->stream));
            TP_CU(cudaStreamSynchronize(ctx->stream));
            done = h[4] != 0 || last == 0;
        }
        if (!h[4] && last == 0) {
            n_far = (int64_t)h[2];
            n_near = (int64_t)h[3];
            break;
        }
        if (attempt > 3 || !h[4]) return tp_set_err(ctx, TP_E_OOM, "dual-tree pair lists keep overflowing");
        // grow every list to twice its size and repeat (an overflowing level stops the traversal,
        // so its count is a lower bound of the need)
        unsigned long long fmax = 0, hf[DT_LEVELS];
        TP_CU(cudaMemcpyAsync(hf, fsize, sizeof(hf), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaStreamSynchronize(ctx->stream));
        for (int l = 0; l < DT_LEVELS; ++l) fmax = std::max(fmax, hf[l]);
        TP_TRY(tp_dual_lists(ctx, std::max<int64_t>(ctx->dt_cap, (int64_t)fmax) * 2,
                             std::max<int64_t>(ctx->dt_far_cap, (int64_t)h[2]) * 2,
                             std::max<int64_t>(ctx->dt_near_cap, (int64_t)h[3]) * 2));
    }
    // per-leaf partner lists: touching ones, apart ones cut into runs
    const int64_t nl = t.nleaves, L1 = nl + 1;
    TP_TRY(tp_dual_leaf_buffers(ctx, nl, nn, 4 * n_near, 2 * n_near / 128 + nl + 1));
    uint32_t* ct = ctx->dt_off;  // counts, then offsets, of the touching lists
    uint32_t* ca = ct + L1;      // ... of the apart lists
    uint32_t* cr = ca + L1;      // ... of the runs
    uint32_t* kt = ctx->dt_cursor;
    uint32_t* ka = kt + L1;
    uint32_t* cat = cr + L1;     // apart counts kept for the runs
    int32_t* tot = reinterpret_cast<int32_t*>(cat + L1);  // [0] apart entries, [1] runs
    TP_CU(cudaMemsetAsync(ctx->dt_node2leaf, 0xff, sizeof(int32_t) * nn, ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->dt_off, 0, sizeof(uint32_t) * (4 * L1 + 2), ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->dt_cursor, 0, sizeof(uint32_t) * 2 * L1, ctx->stream));
    k_dt_leaf_index<<<dt_blocks(nl, 256), 256, 0, ctx->stream>>>(t.leaves, nl, ctx->dt_node2leaf);
    k_dt_count<<<dt_blocks(n_near, 256), 256, 0, ctx->stream>>>(T, ctx->dt_near, n_near, ctx->dt_node2leaf, ct, ca,
                                                                cnt + 7, ctx->derr);
    TP_CU(cudaMemcpyAsync(cat, ca, sizeof(uint32_t) * L1, cudaMemcpyDeviceToDevice, ctx->stream));
    k_dt_runcount<<<dt_blocks(nl, 256), 256, 0, ctx->stream>>>(ca, nl, cr);
    ctx->nlaunch += 3;
    TP_TRY(tp_scan_u32(ctx, ct, ct, L1, false, nullptr));
    TP_TRY(tp_scan_u32(ctx, ca, ca, L1, false, tot));
    TP_TRY(tp_scan_u32(ctx, cr, cr, L1, false, tot + 1));
    int2* list_t = ctx->dt_list;               // at most 2 n_near touching entries
    int2* list_a = ctx->dt_list + 2 * n_near;  // at most 2 n_near apart entries
    k_dt_fill<<<dt_blocks(n_near, 256), 256, 0, ctx->stream>>>(T, ctx->dt_near, n_near, ctx->dt_node2leaf, ct, ca, kt,
                                                               ka, list_t, list_a);
    k_dt_runs<<<dt_blocks(nl, 256), 256, 0, ctx->stream>>>(cat, ca, cr, nl, ctx->dt_runs);
    k_dt_setcount<<<1, 1, 0, ctx->stream>>>(tot + 1, cnt + 8 + 1);
    ctx->nlaunch += 3;
    // near field: touching partners with the exclusion test (each target owned by one warp, stored),
    // then the apart partners in the Barnes-Hut near-field kernel (added)
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    unsigned long long* npairs = cnt + 5;
    unsigned long long* rep = cnt + 6;
    const int wide = t.leaf_size > 16 ? 1 : 0;
    const int edge = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    if (prm->q == 6)
        k_dt_near<6><<<dt_blocks(nl, DT_NEAR_WARPS), DT_NEAR_WARPS * 32, 0, ctx->stream>>>(
            ctx->soa, ctx->ntp, ctx->Fs, t.leaves, nl, t.first, t.last, wide, ct, list_t, edge, ctx->acc, npairs,
            ctx->derr);
    else
        k_dt_near<8><<<dt_blocks(nl, DT_NEAR_WARPS), DT_NEAR_WARPS * 32, 0, ctx->stream>>>(
            ctx->soa, ctx->ntp, ctx->Fs, t.leaves, nl, t.first, t.last, wide, ct, list_t, edge, ctx->acc, npairs,
            ctx->derr);
    ++ctx->nlaunch;
    TP_TRY(tp_launch_near_runs(ctx, prm->q, list_a, 2 * n_near, ctx->dt_runs, ctx->dt_run_cap, cnt + 8));
    // far field: node derivatives, then down to the triangles
    TP_CU(cudaMemsetAsync(ctx->dt_G, 0, sizeof(double) * 7 * nn, ctx->stream));
    if (n_far > 0) {
        k_dt_far<<<(unsigned)std::min<int64_t>(dt_blocks(n_far, DT_THREADS), 16 * ctx->num_sms), DT_THREADS, 0,
                   ctx->stream>>>(T, ctx->dt_far, n_far, prm->q, ctx->dt_G, rep);
        k_dt_node<<<dt_blocks(nn, 256), 256, 0, ctx->stream>>>(ctx->dt_G, t.mom, nn, ctx->dt_P);
        k_dt_down<<<dt_blocks(n, 256), 256, 0, ctx->stream>>>(t.parent, ctx->perm, n, ctx->dt_P, ctx->x64, ctx->nu64,
                                                             ctx->w64, ctx->ntp, (double)prm->p / prm->q,
                                                             (double)prm->q, ctx->acc);
        ctx->nlaunch += 3;
    }
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    unsigned long long h2[3] = {0, 0, 0};
    TP_CU(cudaMemcpyAsync(h2, cnt + 5, sizeof(h2), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    // admitted near pairs: those of the touching pass plus every pair of the apart node pairs
    ctx->stats.pairs_exact = (int64_t)(h2[0] + h2[2]);
    ctx->stats.far_terms = n_far;
    ctx->stats.far_pairs = (int64_t)h2[1];
    ctx->stats.far_rows = n_far;
    return TP_OK;
}

// frontier, far and near lists of the traversal, grown to the given capacities
tp_status tp_dual_lists(tp_ctx* ctx, int64_t cap_front, int64_t cap_far, int64_t cap_near) {
    if (cap_front > ctx->dt_cap) {
        tp_free(ctx, ctx->dt_front[0]);
        tp_free(ctx, ctx->dt_front[1]);
        ctx->dt_front[0] = ctx->dt_front[1] = nullptr;
        ctx->dt_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_front[0], cap_front));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_front[1], cap_front));
        ctx->dt_cap = cap_front;
    }
    if (cap_far > ctx->dt_far_cap) {
        tp_free(ctx, ctx->dt_far);
        ctx->dt_far = nullptr;
        ctx->dt_far_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_far, cap_far));
        ctx->dt_far_cap = cap_far;
    }
    if (cap_near > ctx->dt_near_cap) {
        tp_free(ctx, ctx->dt_near);
        ctx->dt_near = nullptr;
        ctx->dt_near_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_near, cap_near));
        ctx->dt_near_cap = cap_near;
    }
    return TP_OK;
}

// per-leaf partner lists and per-node derivative buffers
tp_status tp_dual_leaf_buffers(tp_ctx* ctx, int64_t nleaves, int64_t nn, int64_t entries, int64_t runs) {
    if (ctx->dt_leaf_cap < nleaves + 1 || ctx->dt_node_cap < nn) {
        for (void* p : {(void*)ctx->dt_off, (void*)ctx->dt_cursor, (void*)ctx->dt_node2leaf, (void*)ctx->dt_G,
                        (void*)ctx->dt_P})
            tp_free(ctx, p);
        ctx->dt_off = ctx->dt_cursor = nullptr;
        ctx->dt_node2leaf = nullptr;
        ctx->dt_G = ctx->dt_P = nullptr;
        ctx->dt_leaf_cap = ctx->dt_node_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_off, 4 * (nleaves + 1) + 2));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_cursor, 2 * (nleaves + 1)));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_node2leaf, nn));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_G, 7 * nn));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_P, 7 * nn));
        ctx->dt_leaf_cap = nleaves + 1;
        ctx->dt_node_cap = nn;
    }
    if (ctx->dt_list_cap < entries) {
        tp_free(ctx, ctx->dt_list);
        ctx->dt_list = nullptr;
        ctx->dt_list_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_list, std::max<int64_t>(entries, 1)));
        ctx->dt_list_cap = entries;
    }
    if (ctx->dt_run_cap < runs) {
        tp_free(ctx, ctx->dt_runs);
        ctx->dt_runs = nullptr;
        ctx->dt_run_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_runs, std::max<int64_t>(runs, 1)));
        ctx->dt_run_cap = runs;
    }
    return TP_OK;
}
