// tp_lbvh.cu - cluster tree for the Barnes-Hut form: linear BVH over Morton
// codes, cluster leaves and FP64 cluster moments.
//
// Sec. 3.2 clusters the inner integral with "precomputed averages over a
// patch of mesh elements" and an admissibility condition after Yu et al.;
// the paper does not name its tree.  This file builds a linear BVH:
//   1. Morton codes of the FP64 centroids (tp_tri.cu, k_morton) sorted as
//      (code, triangle index) keys;
//   2. the binary radix tree of the sorted keys, one thread per internal
//      node: node i covers a key range with i at one end; the direction of
//      the range follows the longer common prefix with a neighbour, its
//      extent is found by exponential then binary search on the common
//      prefix length, and its split is the last position sharing more than
//      the node's common prefix with key i (Karras 2012 numbering: the
//      children of a node split at g are node g, or primitive g when the
//      range [first, g] has one key, and node g+1, or primitive g+1);
//   3. cluster leaves: nodes with at most leaf_size triangles whose parent
//      has more, listed in ascending order of their first triangle;
//   4. moments bottom-up: a primitive holds w, w x (3), w nu (3),
//      (w nu_a) nu_b (6) and its vertex box; an internal node holds
//      left + right, added by the second thread to reach it (atomic visit
//      counter, no waiting: in shared memory while the node's range lies in
//      the block's slice of primitives, in global memory above that).  Every
//      FP64 operation is separately rounded in a fixed order, so the moments
//      are bit-exact with the oracle.  A second pass writes the far-field
//      and admissibility records of the nodes the traversal can reach.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t key_at(const uint32_t* __restrict__ codes_sorted,
                                           const int32_t* __restrict__ perm, int64_t i) {
    return ((uint64_t)codes_sorted[i] << 32) | (uint32_t)perm[i];
}

// common prefix length of keys i and j, -1 outside [0, n)
__device__ __forceinline__ int prefix(const uint32_t* __restrict__ cs, const int32_t* __restrict__ perm, int64_t n,
                                      int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    return __clzll(key_at(cs, perm, i) ^ key_at(cs, perm, j));
}

__global__ void k_radix_tree(const uint32_t* __restrict__ cs, const int32_t* __restrict__ perm, int64_t n,
                             int32_t* __restrict__ left, int32_t* __restrict__ right, int32_t* __restrict__ parent,
                             int32_t* __restrict__ first, int32_t* __restrict__ last) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (prefix(cs, perm, n, i, i + 1) - prefix(cs, perm, n, i, i - 1)) > 0 ? 1 : -1;
    const int dmin = prefix(cs, perm, n, i, i - d);
    int64_t lmax = 2;
    while (prefix(cs, perm, n, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (prefix(cs, perm, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = prefix(cs, perm, n, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
        t = (t + 1) / 2;
        if (prefix(cs, perm, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t g = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int64_t lc = (lo == g) ? (n - 1 + g) : g;
    const int64_t rc = (hi == g + 1) ? (n - 1 + g + 1) : (g + 1);
    left[i] = (int32_t)lc;
    right[i] = (int32_t)rc;
    parent[lc] = (int32_t)i;
    parent[rc] = (int32_t)i;
    first[i] = (int32_t)lo;
    last[i] = (int32_t)hi;
}

__global__ void k_prim_ranges(int64_t n, int32_t* __restrict__ first, int32_t* __restrict__ last,
                              int32_t* __restrict__ parent) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    first[n - 1 + k] = (int32_t)k;
    last[n - 1 + k] = (int32_t)k;
    if (n == 1) parent[0] = -1;
}

__global__ void k_root_parent(int32_t* parent) { parent[0] = -1; }

// start_node[first[v]] = v for every cluster leaf v
__global__ void k_mark_leaves(int64_t n, int leaf_size, const int32_t* __restrict__ first,
                              const int32_t* __restrict__ last, const int32_t* __restrict__ parent,
                              int32_t* __restrict__ start_node) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= 2 * n - 1) return;
    const int64_t cnt = (int64_t)last[v] - first[v] + 1;
    if (cnt > leaf_size) return;
    const int32_t p = (v == 0) ? -1 : parent[v];
    if (p >= 0 && (int64_t)last[p] - first[p] + 1 <= leaf_size) return;
    start_node[first[v]] = (int32_t)v;
}


constexpr int MOM_B = 64;   // primitives per block of the bottom-up pass
constexpr int MOM_W = 19;   // values per node: 13 moments + 6 box bounds

// The records derived from a node's moments and box:
//   nodef[v] = X - centre split hi/lo (6), nubar = sum(w nu)/A (3), sqrt(p/q) A (1)
//              in FP32 for the far-field terms;
//   adm64[v] = (X_C[3] = sum(w x)/A, diag_C = |box extent|) in FP64, with exactly
//              the operations and order of the oracle's admissibility test;
//   adm32[v] = box rounded outward (min down, max up) [6], X_C [3], diag_C [1]
//              in FP32 for the pre-test that settles all but borderline cases
//              (tp_bh.cu), then the member range and the children (int bits,
//              -1 for a single-triangle node).
__device__ __forceinline__ void node_records(int64_t v, const double* __restrict__ m, const double* __restrict__ b,
                                             const double* __restrict__ c3, float* __restrict__ nodef,
                                             double* __restrict__ adm64, float* __restrict__ adm32, int first,
                                             int last, int left, int right) {
    double dc2 = 0.0;
    double X[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double ec = __dsub_rn(b[3 + a], b[a]);
        dc2 = __dadd_rn(dc2, __dmul_rn(ec, ec));
        X[a] = __ddiv_rn(m[1 + a], m[0]);
    }
    const double dc = __dsqrt_rn(dc2);
    double2* a64 = reinterpret_cast<double2*>(adm64 + 4 * v);
    a64[0] = make_double2(X[0], X[1]);
    a64[1] = make_double2(X[2], dc);
    float4* a32 = reinterpret_cast<float4*>(adm32 + TP_ADM32_W * v);
    a32[0] = make_float4(__double2float_rd(b[0]), __double2float_rd(b[1]), __double2float_rd(b[2]),
                         __double2float_ru(b[3]));
    a32[1] = make_float4(__double2float_ru(b[4]), __double2float_ru(b[5]), (float)X[0], (float)X[1]);
    a32[2] = make_float4((float)X[2], (float)dc, __int_as_float(first), __int_as_float(last));
    a32[3] = make_float4(__int_as_float(left), __int_as_float(right), 0.f, 0.f);
    float hi[3], lo[3], nb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double Xc = X[a] - c3[a];
        hi[a] = (float)Xc;
        lo[a] = (float)(Xc - (double)hi[a]);
        nb[a] = (float)(__ddiv_rn(m[4 + a], m[0]));
    }
    float4* r = reinterpret_cast<float4*>(nodef + 16 * v);
    r[0] = make_float4(hi[0], hi[1], hi[2], lo[0]);
    r[1] = make_float4(lo[1], lo[2], nb[0], nb[1]);
    r[2] = make_float4(nb[2], (float)(1.4142135623730951 * m[0]), 0.0f, 0.0f);
    r[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ void node_store(int64_t v, const double* __restrict__ m, double* __restrict__ mom,
                                           double* __restrict__ box) {
    double* mo = mom + 13 * v;
#pragma unroll
    for (int c = 0; c < 13; ++c) mo[c] = m[c];
    double2* bo = reinterpret_cast<double2*>(box + 6 * v);
    bo[0] = make_double2(m[13], m[14]);
    bo[1] = make_double2(m[15], m[16]);
    bo[2] = make_double2(m[17], m[18]);
}

// Order-preserving integer key of a finite double, with -0 and +0 equal:
// key(l) < key(r) exactly when l < r.  The boxes' min/max selections below
// keep the FP64 comparison's result (ties pick the same operand) but run on
// the integer pipe instead of the narrow FP64 pipe.  Positions are finite
// (checked at upload).
__device__ __forceinline__ long long ord_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (long long)(0x8000000000000000ULL - (unsigned long long)b);
}
__device__ __forceinline__ double lo_of(double l, double r) { return ord_key(l) < ord_key(r) ? l : r; }
__device__ __forceinline__ double hi_of(double l, double r) { return ord_key(l) > ord_key(r) ? l : r; }

// parent = left + right (moments), box = union with the left child's value
// kept on ties, as in the oracle
__device__ __forceinline__ void node_combine(double* __restrict__ own, const double* __restrict__ sib, int stride,
                                             bool own_left) {
#pragma unroll
    for (int c = 0; c < 13; ++c) own[c] = __dadd_rn(own[c], sib[c * stride]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double o0 = own[13 + a], s0 = sib[(13 + a) * stride];
        const double o1 = own[16 + a], s1 = sib[(16 + a) * stride];
        const double l0 = own_left ? o0 : s0, r0 = own_left ? s0 : o0;
        const double l1 = own_left ? o1 : s1, r1 = own_left ? s1 : o1;
        own[13 + a] = lo_of(l0, r0);
        own[16 + a] = hi_of(l1, r1);
    }
}

// Primitive moments and the bottom-up pass.
// Block b owns primitives [b MOM_B, (b+1) MOM_B): a node whose key range lies
// inside that slice is added up in shared memory (CTA counters), one whose
// range spans slices through global memory (device counters); in both the
// second thread to reach a node adds its children and carries on.
__global__ void __launch_bounds__(MOM_B) k_moments(
    const double* __restrict__ V, const int32_t* __restrict__ F, const double* __restrict__ x64,
    const double* __restrict__ nu64, const double* __restrict__ w64, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ left, const int32_t* __restrict__ right, const int32_t* __restrict__ parent,
    const int32_t* __restrict__ first, const int32_t* __restrict__ last, int64_t n, int32_t* __restrict__ counter,
    double* __restrict__ mom, double* __restrict__ box) {
    __shared__ double vs[MOM_W][2 * MOM_B];  // slot t: primitive base+t; slot MOM_B+i: internal node base+i
    __shared__ int cnt_s[MOM_B];
    const int t = threadIdx.x;
    const int64_t base = blockIdx.x * (int64_t)MOM_B;
    cnt_s[t] = 0;
    __syncthreads();
    const int64_t k = base + t;
    if (k >= n) return;
    double own[MOM_W];
    {
        const int64_t T = perm[k];
        const double w = w64[T];
        double nu[3];
        for (int a = 0; a < 3; ++a) nu[a] = nu64[a * n + T];
        own[0] = w;
        for (int a = 0; a < 3; ++a) own[1 + a] = __dmul_rn(w, x64[a * n + T]);
        for (int a = 0; a < 3; ++a) own[4 + a] = __dmul_rn(w, nu[a]);
        int o = 7;
        for (int a = 0; a < 3; ++a)
            for (int c = a; c < 3; ++c) own[o++] = __dmul_rn(__dmul_rn(w, nu[a]), nu[c]);
        const int64_t f0 = 3 * (int64_t)F[3 * T], f1 = 3 * (int64_t)F[3 * T + 1], f2 = 3 * (int64_t)F[3 * T + 2];
        for (int a = 0; a < 3; ++a) {
            const double p0 = V[f0 + a], p1 = V[f1 + a], p2 = V[f2 + a];
            // lo = p0, then p1 and p2 replace it when smaller (hi: larger)
            own[13 + a] = lo_of(p2, lo_of(p1, p0));
            own[16 + a] = hi_of(p2, hi_of(p1, p0));
        }
    }
    int64_t v = n - 1 + k;
    node_store(v, own, mom, box);
    if (n == 1) return;
    int slot = t;
    bool local = true;
    while (true) {
        const int64_t p = parent[v];
        if (p < 0) break;
        const int64_t lc = left[p], rc = right[p];
        const bool own_left = lc == v;
        const int64_t sib = own_left ? rc : lc;
        if (local && first[p] >= base && last[p] < base + MOM_B) {
#pragma unroll
            for (int c = 0; c < MOM_W; ++c) vs[c][slot] = own[c];
            __threadfence_block();
            if (atomicAdd(&cnt_s[p - base], 1) == 0) break;
            __threadfence_block();
            const int ss = sib >= n - 1 ? (int)(sib - (n - 1) - base) : MOM_B + (int)(sib - base);
            node_combine(own, &vs[0][ss], 2 * MOM_B, own_left);
            slot = MOM_B + (int)(p - base);
        } else {
            local = false;
            __threadfence();
            if (atomicAdd(&counter[p], 1) == 0) break;
            __threadfence();
            double sv[MOM_W];
            const double* ms = mom + 13 * sib;
            const double* bs = box + 6 * sib;
#pragma unroll
            for (int c = 0; c < 13; ++c) sv[c] = __ldcg(ms + c);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                sv[13 + a] = __ldcg(bs + a);
                sv[16 + a] = __ldcg(bs + 3 + a);
            }
            node_combine(own, sv, 1, own_left);
        }
        v = p;
        node_store(v, own, mom, box);
    }
}

// far-field and admissibility records of every node the traversal can reach
__global__ void __launch_bounds__(TP_NODE_THREADS) k_node_out(
    const double* __restrict__ mom, const double* __restrict__ box, const int32_t* __restrict__ parent,
    const int32_t* __restrict__ first, const int32_t* __restrict__ last, const int32_t* __restrict__ left,
    const int32_t* __restrict__ right, int leaf_size, const double* __restrict__ center, int64_t nn,
    float* __restrict__ nodef, double* __restrict__ adm64, float* __restrict__ adm32) {
    __shared__ int32_t list[TP_NODE_BLK];
    __shared__ int cnt;
    const int n = tp_reachable_list(parent, first, last, leaf_size, blockIdx.x * (int64_t)TP_NODE_BLK, nn, list,
                                    &cnt);
    const double c3[3] = {center[0], center[1], center[2]};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t v = list[i];
        double m[13], b[6];
#pragma unroll
        for (int c = 0; c < 13; ++c) m[c] = mom[13 * v + c];
        const double2* bi = reinterpret_cast<const double2*>(box + 6 * v);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 x = bi[c];
            b[2 * c] = x.x;
            b[2 * c + 1] = x.y;
        }
        const int64_t n = (nn + 1) / 2;  // triangles; nodes below n - 1 are internal
        node_records(v, m, b, c3, nodef, adm64, adm32, first[v], last[v], v < n - 1 ? left[v] : -1,
                     v < n - 1 ? right[v] : -1);
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

tp_status tp_launch_tree_build(tp_ctx* ctx, int leaf_size, int morton_bits) {
    TpRange nvtx_range("tp_launch_tree_build");
    const int64_t n = ctx->nt;
    const int64_t nn = 2 * n - 1;
    tp_tree& t = ctx->tree;
    if (t.cap < n) {
        tp_free(ctx, t.left);
        tp_free(ctx, t.right);
        tp_free(ctx, t.parent);
        tp_free(ctx, t.first);
        tp_free(ctx, t.last);
        tp_free(ctx, t.leaves);
        tp_free(ctx, t.counter);
        tp_free(ctx, t.mom);
        tp_free(ctx, t.box);
        tp_free(ctx, t.nodef);
        tp_free(ctx, t.nleaves_d);
        tp_free(ctx, t.adm64);
        tp_free(ctx, t.adm32);
        tp_free(ctx, t.nodeft);
        t.left = t.right = t.parent = t.first = t.last = t.leaves = t.counter = t.nleaves_d = nullptr;
        t.mom = t.box = t.adm64 = nullptr;
        t.nodef = t.adm32 = t.nodeft = nullptr;
        TP_TRY(tp_alloc_t(ctx, &t.left, n));
        TP_TRY(tp_alloc_t(ctx, &t.right, n));
        TP_TRY(tp_alloc_t(ctx, &t.parent, nn));
        TP_TRY(tp_alloc_t(ctx, &t.first, nn));
        TP_TRY(tp_alloc_t(ctx, &t.last, nn));
        TP_TRY(tp_alloc_t(ctx, &t.leaves, n));
        TP_TRY(tp_alloc_t(ctx, &t.counter, n));
        TP_TRY(tp_alloc_t(ctx, &t.mom, 13 * nn));
        TP_TRY(tp_alloc_t(ctx, &t.box, 6 * nn));
        TP_TRY(tp_alloc_t(ctx, &t.nodef, 16 * nn));
        TP_TRY(tp_alloc_t(ctx, &t.nleaves_d, 4));
        TP_TRY(tp_alloc_t(ctx, &t.adm64, 4 * nn));
        TP_TRY(tp_alloc_t(ctx, &t.adm32, TP_ADM32_W * nn));
        TP_TRY(tp_alloc_t(ctx, &t.nodeft, 16 * nn));
        t.cap = n;
    }
    t.leaf_size = leaf_size;
    t.morton_bits = morton_bits;
    // 1. Morton order of the current centroids; refresh the library-order data
    TP_TRY(tp_launch_morton_order(ctx, morton_bits));
    TP_TRY(tp_launch_sorted_soa(ctx));
    ctx->flags_stale = 2;  // the direct kernels' item lists follow the new order when next needed
    // 2. radix tree
    if (n > 1) {
        k_radix_tree<<<nblk(n - 1, 256), 256, 0, ctx->stream>>>(ctx->codes_sorted, ctx->perm, n, t.left, t.right,
                                                               t.parent, t.first, t.last);
        ++ctx->nlaunch;
        k_root_parent<<<1, 1, 0, ctx->stream>>>(t.parent);
        ++ctx->nlaunch;
    }
    k_prim_ranges<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, t.first, t.last, t.parent);
    ++ctx->nlaunch;
    // 3. cluster leaves in ascending order of their first triangle
    int32_t* start_node = ctx->idx_tmp;
    TP_CU(cudaMemsetAsync(start_node, 0xff, sizeof(int32_t) * n, ctx->stream));
    k_mark_leaves<<<nblk(nn, 256), 256, 0, ctx->stream>>>(n, leaf_size, t.first, t.last, t.parent, start_node);
    ++ctx->nlaunch;
    TP_TRY(tp_compact_nonneg(ctx, start_node, n, t.leaves, t.nleaves_d));
    // 4. moments
    if (n > 1) TP_CU(cudaMemsetAsync(t.counter, 0, sizeof(int32_t) * (n - 1), ctx->stream));
    k_moments<<<nblk(n, MOM_B), MOM_B, 0, ctx->stream>>>(ctx->V64, ctx->F, ctx->x64, ctx->nu64, ctx->w64, ctx->perm,
                                                         t.left, t.right, t.parent, t.first, t.last, n, t.counter,
                                                         t.mom, t.box);
    ++ctx->nlaunch;
    k_node_out<<<nblk(nn, TP_NODE_BLK), TP_NODE_THREADS, 0, ctx->stream>>>(
        t.mom, t.box, t.parent, t.first, t.last, t.left, t.right, leaf_size, ctx->center, nn, t.nodef, t.adm64,
        t.adm32);
    ++ctx->nlaunch;
    t.feat_stale = true;  // the network's node features are computed when the learned form needs them
    int32_t h = 0;
    TP_CU(cudaMemcpyAsync(&h, t.nleaves_d, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    TP_CU(cudaGetLastError());
    t.nleaves = h;
    return TP_OK;
}
