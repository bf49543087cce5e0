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
//                 host repeats the traversal with larger lists on overflow;
//   k_dt_far      FP64 far terms, one thread per far pair, node derivatives
//                 summed with FP64 atomics;
//   k_dt_count/k_dt_fill  per cluster leaf, the list of its near partners
//                 (both directions of each near pair) as (first member, count);
//   k_dt_near     one warp per cluster leaf gathers both orderings of every
//                 admitted pair with its partners' members (packed FP32x2,
//                 FP64 per partner batch), exclusion test on every pair, and
//                 stores the leaf's accumulators (direct kernels' layout);
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
    const double* mom;  // [nn][13]
    const double* box;  // [nn][6]
    int64_t n;
    int leaf;
};

__device__ __forceinline__ bool dt_small(const DTTree& T, int node) {
    return node >= T.n - 1 || (T.last[node] - T.first[node] + 1) <= T.leaf;
}

__device__ __forceinline__ double dt_diag2(const double* b) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double e = __dsub_rn(b[3 + a], b[a]);
        s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return s;
}

__device__ bool dt_admissible(const double* bA, const double* mA, const double* bB, const double* mB, double theta) {
    bool disjoint = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (bA[3 + a] < bB[a] || bB[3 + a] < bA[a]) disjoint = true;
    if (!disjoint) return false;
    const double dA2 = dt_diag2(bA), dB2 = dt_diag2(bB);
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = __dsub_rn(__ddiv_rn(mA[1 + a], mA[0]), __ddiv_rn(mB[1 + a], mB[0]));
        r2 = __dadd_rn(r2, __dmul_rn(t, t));
    }
    const double diag = __dsqrt_rn(dA2 > dB2 ? dA2 : dB2);
    return diag < __dmul_rn(theta, __dsqrt_rn(r2));
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
__global__ void __launch_bounds__(DT_THREADS) k_dt_expand(DTTree T, double theta, const int2* __restrict__ fin,
                                                          int64_t n_in, int2* __restrict__ fout, int64_t cap_out,
                                                          int2* __restrict__ far, int64_t cap_far,
                                                          int2* __restrict__ near, int64_t cap_near,
                                                          unsigned long long* __restrict__ cnt) {
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
            } else if (dt_admissible(T.box + 6 * (int64_t)A, T.mom + 13 * (int64_t)A, T.box + 6 * (int64_t)B,
                                     T.mom + 13 * (int64_t)B, theta)) {
                kind = 1;
            } else if (sA && sB) {
                kind = 0;
            } else {
                const int cA = T.last[A] - T.first[A], cB = T.last[B] - T.first[B];
                kind = (!sA && (cA >= cB || sB)) ? 2 : 3;
            }
        }
        const unsigned n_out = kind == 4 ? 3u : (kind == 2 || kind == 3) ? 2u : 0u;
        const unsigned long long po = warp_reserve(n_out, &cnt[1]);
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

// Far pairs in FP64: the node derivatives dE/d(A, X[3], nubar[3]) of both
// nodes into G[node][7]; the represented ordered pairs into *rep.
__global__ void __launch_bounds__(DT_THREADS) k_dt_far(DTTree T, const int2* __restrict__ far, int64_t nfar, int q,
                                                       double p, double* __restrict__ G,
                                                       unsigned long long* __restrict__ rep) {
    unsigned long long my_rep = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfar; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 pr = far[i];
        const double* mA = T.mom + 13 * (int64_t)pr.x;
        const double* mB = T.mom + 13 * (int64_t)pr.y;
        const double AA = mA[0], AB = mB[0];
        double d[3], nA[3], nB[3], r2 = 0.0, n1 = 0.0, n2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[a] = mA[1 + a] / AA - mB[1 + a] / AB;
            nA[a] = mA[4 + a] / AA;
            nB[a] = mB[4 + a] / AB;
            r2 += d[a] * d[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            n1 += nA[a] * d[a];
            n2 -= nB[a] * d[a];
        }
        const double inv = 1.0 / r2;
        double rp = 1.0;  // |d|^-p, p even
        for (int e = 0; e < (int)(p / 2); ++e) rp *= inv;
        double b1 = (double)q, b2 = (double)q;  // q n^(q-1)
        for (int e = 0; e < q - 1; ++e) {
            b1 *= n1;
            b2 *= n2;
        }
        const double a1 = b1 * n1 / q, a2 = b2 * n2 / q;  // n^q
        const double AAB = AA * AB, s = a1 + a2;
        double* GA = G + 7 * (int64_t)pr.x;
        double* GB = G + 7 * (int64_t)pr.y;
        atomicAdd(&GA[0], AB * s * rp);
        atomicAdd(&GB[0], AA * s * rp);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double gX = AAB * rp * (b1 * nA[k] - b2 * nB[k] - p * s * inv * d[k]);
            atomicAdd(&GA[1 + k], gX);
            atomicAdd(&GB[1 + k], -gX);
            atomicAdd(&GA[4 + k], AAB * b1 * rp * d[k]);
            atomicAdd(&GB[4 + k], -AAB * b2 * rp * d[k]);
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

// partners per cluster leaf: both directions of every near pair (a self pair once)
__global__ void k_dt_count(const int2* __restrict__ near, int64_t nnear, const int32_t* __restrict__ node2leaf,
                           uint32_t* __restrict__ count, unsigned* derr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnear) return;
    const int2 pr = near[i];
    const int la = node2leaf[pr.x], lb = node2leaf[pr.y];
    if (la < 0 || lb < 0) {  // a near node that is not a cluster leaf: the recursion's invariant failed
        tp_dev_error(derr, TP_DERR_INTERNAL);
        return;
    }
    atomicAdd(&count[la], 1u);
    if (pr.x != pr.y) atomicAdd(&count[lb], 1u);
}

__global__ void k_dt_fill(const int2* __restrict__ near, int64_t nnear, const int32_t* __restrict__ node2leaf,
                          const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                          const uint32_t* __restrict__ off, uint32_t* __restrict__ cursor, int2* __restrict__ list) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnear) return;
    const int2 pr = near[i];
    const int la = node2leaf[pr.x], lb = node2leaf[pr.y];
    if (la < 0 || lb < 0) return;
    list[off[la] + atomicAdd(&cursor[la], 1u)] = make_int2(first[pr.y], last[pr.y] - first[pr.y] + 1);
    if (pr.x != pr.y) list[off[lb] + atomicAdd(&cursor[lb], 1u)] = make_int2(first[pr.x], last[pr.x] - first[pr.x] + 1);
}

// One warp per cluster leaf: both orderings of every admitted pair of its
// targets with its near partners' members, gathered on the target side.
template <int Q>
__global__ void __launch_bounds__(DT_NEAR_WARPS * 32) k_dt_near(const float* __restrict__ soa, int64_t ntp,
                                                                const int32_t* __restrict__ Fs,
                                                                const int32_t* __restrict__ leaves, int64_t nleaves,
                                                                const int32_t* __restrict__ first,
                                                                const int32_t* __restrict__ last, int wide,
                                                                const uint32_t* __restrict__ off,
                                                                const int2* __restrict__ list, int edge_only,
                                                                double* __restrict__ acc,
                                                                unsigned long long* __restrict__ npairs) {
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
    double a64[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long n_adm = 0;
    const uint32_t e0 = off[li], e1 = off[li + 1];
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
        for (int c = 0; c < 8; ++c) a64[c] += (double)(a2[c].x + a2[c].y);
        e = e2;
    }
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
    const double* m = mom + 13 * N;
    const double A = m[0];
    double s = g[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P[7 * N + 1 + a] = g[1 + a] / A;
        P[7 * N + 4 + a] = g[4 + a] / A;
        s -= (g[1 + a] * (m[1 + a] / A) + g[4 + a] * (m[4 + a] / A)) / A;
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
    T.n = n;
    T.leaf = t.leaf_size;
    if (!ctx->dt_cnt) TP_TRY(tp_alloc_t(ctx, &ctx->dt_cnt, 8));
    unsigned long long* cnt = ctx->dt_cnt;
    if (ctx->dt_cap == 0) {
        const int64_t c0 = std::max<int64_t>(1 << 16, 64 * t.nleaves);
        TP_TRY(tp_dual_lists(ctx, c0, c0, c0));
    }
    cudaEventRecord(ctx->ev[0], ctx->stream);
    int64_t n_far = 0, n_near = 0;
    for (int attempt = 0;; ++attempt) {
        // the traversal, level by level from (root, root)
        const int2 root = make_int2(0, 0);
        TP_CU(cudaMemcpyAsync(ctx->dt_front[0], &root, sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
        TP_CU(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), ctx->stream));
        int64_t n_in = 1;
        int cur = 0;
        bool overflow = false;
        unsigned long long h[5] = {0, 0, 0, 0, 0};
        for (int level = 0; n_in > 0 && level < 4096; ++level) {
            TP_CU(cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned long long), ctx->stream));
            const unsigned blocks = (unsigned)std::min<int64_t>(dt_blocks(n_in, DT_THREADS), 8 * ctx->num_sms);
            k_dt_expand<<<blocks, DT_THREADS, 0, ctx->stream>>>(T, prm->theta, ctx->dt_front[cur], n_in,
                                                                 ctx->dt_front[cur ^ 1], ctx->dt_cap, ctx->dt_far,
                                                                 ctx->dt_far_cap, ctx->dt_near, ctx->dt_near_cap, cnt);
            ++ctx->nlaunch;
            TP_CU(cudaMemcpyAsync(h, cnt, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
            TP_CU(cudaStreamSynchronize(ctx->stream));
            if (h[4]) {
                overflow = true;
                break;
            }
            n_in = (int64_t)h[1];
            cur ^= 1;
        }
        if (!overflow) {
            n_far = (int64_t)h[2];
            n_near = (int64_t)h[3];
            break;
        }
        if (attempt > 3) return tp_set_err(ctx, TP_E_OOM, "dual-tree pair lists keep overflowing");
        // grow the list that overflowed (the counters passed the capacities) and repeat
        TP_TRY(tp_dual_lists(ctx, std::max<int64_t>(ctx->dt_cap, (int64_t)h[1]) * 2,
                             std::max<int64_t>(ctx->dt_far_cap, (int64_t)h[2]) * 2,
                             std::max<int64_t>(ctx->dt_near_cap, (int64_t)h[3]) * 2));
    }
    // per-leaf partner lists
    const int64_t nl = t.nleaves;
    TP_TRY(tp_dual_leaf_buffers(ctx, nl, nn, 2 * n_near));
    TP_CU(cudaMemsetAsync(ctx->dt_node2leaf, 0xff, sizeof(int32_t) * nn, ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->dt_off, 0, sizeof(uint32_t) * (nl + 1), ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->dt_cursor, 0, sizeof(uint32_t) * nl, ctx->stream));
    k_dt_leaf_index<<<dt_blocks(nl, 256), 256, 0, ctx->stream>>>(t.leaves, nl, ctx->dt_node2leaf);
    k_dt_count<<<dt_blocks(n_near, 256), 256, 0, ctx->stream>>>(ctx->dt_near, n_near, ctx->dt_node2leaf, ctx->dt_off,
                                                                ctx->derr);
    TP_TRY(tp_scan_u32(ctx, ctx->dt_off, ctx->dt_off, nl + 1, false, nullptr));
    k_dt_fill<<<dt_blocks(n_near, 256), 256, 0, ctx->stream>>>(ctx->dt_near, n_near, ctx->dt_node2leaf, t.first,
                                                               t.last, ctx->dt_off, ctx->dt_cursor, ctx->dt_list);
    ctx->nlaunch += 3;
    // near field: every target owned by one warp, stored without atomics
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    unsigned long long* npairs = cnt + 5;
    unsigned long long* rep = cnt + 6;
    const int wide = t.leaf_size > 16 ? 1 : 0;
    const int edge = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    if (prm->q == 6)
        k_dt_near<6><<<dt_blocks(nl, DT_NEAR_WARPS), DT_NEAR_WARPS * 32, 0, ctx->stream>>>(
            ctx->soa, ctx->ntp, ctx->Fs, t.leaves, nl, t.first, t.last, wide, ctx->dt_off, ctx->dt_list, edge,
            ctx->acc, npairs);
    else
        k_dt_near<8><<<dt_blocks(nl, DT_NEAR_WARPS), DT_NEAR_WARPS * 32, 0, ctx->stream>>>(
            ctx->soa, ctx->ntp, ctx->Fs, t.leaves, nl, t.first, t.last, wide, ctx->dt_off, ctx->dt_list, edge,
            ctx->acc, npairs);
    ++ctx->nlaunch;
    // far field: node derivatives, then down to the triangles
    TP_CU(cudaMemsetAsync(ctx->dt_G, 0, sizeof(double) * 7 * nn, ctx->stream));
    if (n_far > 0) {
        k_dt_far<<<(unsigned)std::min<int64_t>(dt_blocks(n_far, DT_THREADS), 16 * ctx->num_sms), DT_THREADS, 0,
                   ctx->stream>>>(T, ctx->dt_far, n_far, prm->q, (double)prm->p, ctx->dt_G, rep);
        k_dt_node<<<dt_blocks(nn, 256), 256, 0, ctx->stream>>>(ctx->dt_G, t.mom, nn, ctx->dt_P);
        k_dt_down<<<dt_blocks(n, 256), 256, 0, ctx->stream>>>(t.parent, ctx->perm, n, ctx->dt_P, ctx->x64, ctx->nu64,
                                                             ctx->w64, ctx->ntp, (double)prm->p / prm->q,
                                                             (double)prm->q, ctx->acc);
        ctx->nlaunch += 3;
    }
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    unsigned long long h2[2] = {0, 0};
    TP_CU(cudaMemcpyAsync(h2, cnt + 5, sizeof(h2), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.pairs_exact = (int64_t)h2[0];
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
tp_status tp_dual_leaf_buffers(tp_ctx* ctx, int64_t nleaves, int64_t nn, int64_t entries) {
    if (ctx->dt_leaf_cap < nleaves + 1 || ctx->dt_node_cap < nn) {
        for (void* p : {(void*)ctx->dt_off, (void*)ctx->dt_cursor, (void*)ctx->dt_node2leaf, (void*)ctx->dt_G,
                        (void*)ctx->dt_P})
            tp_free(ctx, p);
        ctx->dt_off = ctx->dt_cursor = nullptr;
        ctx->dt_node2leaf = nullptr;
        ctx->dt_G = ctx->dt_P = nullptr;
        ctx->dt_leaf_cap = ctx->dt_node_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_off, nleaves + 1));
        TP_TRY(tp_alloc_t(ctx, &ctx->dt_cursor, nleaves + 1));
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
    return TP_OK;
}
