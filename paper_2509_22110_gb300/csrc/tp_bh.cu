// tp_bh.cu - Barnes-Hut form: only the inner sum is clustered (Sec. 3.2).
//
// For every target triangle T the library needs the derivatives of
// sum_S (e_TS + e_ST) with respect to T's own centroid, normal and area (the
// inner integrals of Eq. (dTP_reordered), Sec. 3.2, are functions of the
// outer point only).  The inner sum over S is split by the cluster tree:
//   - a cluster C that is admissible for the target's leaf L (vertex boxes
//     strictly disjoint along some axis, and
//     diag(C) < theta (|X_C - c_L| - diag(L)/2), decided in FP64 with
//     separately rounded operations) contributes one far term built from
//     its moments: area A_C, area-weighted centroid X_C and area-averaged
//     normal nubar_C = sum(w nu)/A_C (not renormalised), both orderings;
//   - a non-admissible cluster leaf contributes its member pairs exactly,
//     skipping T itself and triangles sharing a vertex with T;
//   - a non-admissible internal node is opened.
// Derivatives are not propagated into the cluster moments.  theta = 0
// admits no cluster and reproduces the direct sum.
//
// GPU organisation.  k_bh: one warp per target cluster leaf (at most 32
// targets per leaf, 16 by default).  The admissibility test depends on (L, C)
// only, so the traversal is warp-uniform: the warp pops up to 32 nodes from a
// shared-memory stack, each lane tests one, and ballots sort them into a far
// list, two near lists and nodes to open.  A near cluster whose vertex box is
// apart from the leaf's can hold no triangle adjacent to a target: those are
// listed for k_near, which sums them without exclusion tests (and forms d from
// the hi parts alone when the boxes are at least TP_PRECISE_GAP_REL of the
// mesh's box diagonal apart, the direct kernels' FAST rule).  Near clusters
// whose box touches the leaf's (the leaf itself among them) are evaluated in
// k_bh with the test on every pair, and so are the far terms of the plain
// form.  These sweeps run in packed FP32x2 arithmetic, one target against two
// staged sources per instruction, with lanes split as (target = lane % 16,
// half = lane / 16) for leaves of up to 16 targets (each half taking every
// other source pair) or one target per lane for larger leaves.  Per-target
// partials are FP32 per list flush and FP64 across flushes; each target is
// owned by one warp, so k_bh stores its results without atomics in the
// accumulator layout of the direct kernels (see tp_direct.cu); k_near (and
// k_far) add to them, and the same adjoint applies.
//
// Learned form (TP_LEARNED).  The traversal lists the far nodes of every leaf
// (runs of up to 256 nodes, reserved with one atomic per run) instead of
// evaluating them; the network runs on the listed (leaf, cluster) pairs, and
// k_far evaluates each far term once with the network's channel factors.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "tp_internal.cuh"
#include "tp_mlp_dev.cuh"
#include "tp_pair_dev.cuh"

namespace {

constexpr int BH_WARPS = 4;
constexpr int BH_STACK = 1024;
constexpr int BH_FAR = 256;
constexpr int BH_NEAR = TP_BH_NEAR;  // clusters per near-field run (k_bh's list of clusters apart from the leaf)
constexpr int BH_TOUCH = 128;        // touching clusters gathered before k_bh sweeps them
#ifndef TP_NEAR_FAST
#define TP_NEAR_FAST 1  // near clusters far enough apart take the hi-part difference only
#endif
#ifndef TP_FAR_FAST
#define TP_FAR_FAST 1  // the same for the far nodes of the plain form
#endif
#ifndef TP_BH_MINB
#define TP_BH_MINB 5  // resident blocks per SM asked of the register allocator (20 warps)
#endif

struct BHArgs {
    const float* soa;
    int64_t ntp;
    const int32_t* Fs;
    const int32_t* left;
    const int32_t* right;
    const int32_t* first;
    const int32_t* last;
    const int32_t* leaves;
    int64_t nleaves;
    int64_t n;
    const double* mom;
    const double* box;
    const float* nodef;
    const double* adm64;
    const float* adm32;
    const double* bounds;        // mesh bounding box (min[3], max[3]) of the tree build
    double theta;
    int leaf_size;
    int edge_only;
    double* acc;
    unsigned* derr;
    unsigned long long* counts;  // [0] near pairs, [1] far terms, [2] far pairs, [3] learned terms
    unsigned long long* far_rows;  // (leaf, cluster) far pairs
    unsigned long long* near_listed;  // ordered pairs listed for k_near: [0] all, [1] with hi-only differences
    // learned far field
    const float* nodeft;         // [nn][16] f32 feature records
    const __nv_bfloat16* wb;     // network weights (BF16 block)
    const float* mbias;          // network biases
    const float* mnorm;          // [4][24] feature mean, std, lo, hi
    // far field: far node ids listed for k_far, in runs of one leaf
    int32_t* far_list;
    int32_t* far_leaf;           // the leaf (index into leaves) of each listed row
    tp_far_run* far_runs;
    unsigned long long* far_count;  // [0] rows, [1] runs listed (past the capacities), [2] k_far work counter
    int64_t far_cap, run_cap;
    // near field: clusters apart from the leaf, listed for k_near
    const float* src;            // [ntp][TP_SRCW] source records (each value twice)
    int2* near_list;             // (first member, count) per listed cluster
    tp_far_run* near_runs;       // runs of one leaf
    unsigned long long* near_count;  // [0] entries, [1] runs listed (past the capacities), [2] k_near work counter
    int64_t near_cap, nrun_cap;
    // sampling of far pairs (RECORD mode)
    uint32_t keep_u;
    uint64_t seed;
    int2* rec_out;
    int64_t rec_cap;
    int32_t* rec_count;
};

// M_BH: the evaluation pass of the plain form (evaluates the far nodes and
// the touching near clusters, lists the near clusters apart from the leaf for
// k_near); M_LIST: the same for the learned form, with the far nodes listed
// for the network and k_far instead of evaluated; M_RECORD: sample far pairs
// for training only.
enum { M_BH = 0, M_LIST = 1, M_RECORD = 2 };

// A pair of targets (one per half of t) against one source record of the
// direct kernels' layout (each value stored twice: x_hi[3], x_lo[3], nu[3], w~),
// without the target weights (k_near multiplies its sums by them).
template <int Q, bool HILO>
__device__ __forceinline__ void near_pair2(const Tgt2& t, const float* rec, float2 acc[8]) {
    const float4* r = reinterpret_cast<const float4*>(rec);
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
    const float2 sh[3] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w), make_float2(r1.x, r1.y)};
    const float2 sl[3] = {make_float2(r1.z, r1.w), make_float2(r2.x, r2.y), make_float2(r2.z, r2.w)};
    const float2 sn[3] = {make_float2(r3.x, r3.y), make_float2(r3.z, r3.w), make_float2(r4.x, r4.y)};
    pair_core<Q, false, HILO, true>(t.h, t.l, t.n, t.w, sh, sl, sn, make_float2(r4.z, r4.w), acc, true, true);
}

// Target-leaf constants of the admissibility test.
struct LeafAdm {
    double bl[6];      // FP64 vertex box
    double cl[3];      // box centre (bl_min + bl_max) * 0.5
    double dl;         // box diagonal
    float out[6], in[6], cl32[3], dl32;
    float fast2;       // squared box gap from which a near cluster's pairs take the hi parts only
};

__device__ __forceinline__ void leaf_adm(const double* box, const double* bounds, LeafAdm& L) {
    double dl2 = 0.0, md2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double e = bounds[3 + a] - bounds[a];
        md2 += e * e;
    }
    const float delta = TP_PRECISE_GAP_REL * (float)sqrt(md2);
    L.fast2 = TP_NEAR_FAST ? delta * delta : INFINITY;
#pragma unroll
    for (int a = 0; a < 6; ++a) L.bl[a] = box[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double el = __dsub_rn(L.bl[3 + a], L.bl[a]);
        dl2 = __dadd_rn(dl2, __dmul_rn(el, el));
        L.cl[a] = __dmul_rn(__dadd_rn(L.bl[a], L.bl[3 + a]), 0.5);
        L.out[a] = __double2float_rd(L.bl[a]);
        L.out[3 + a] = __double2float_ru(L.bl[3 + a]);
        L.in[a] = __double2float_ru(L.bl[a]);
        L.in[3 + a] = __double2float_rd(L.bl[3 + a]);
        L.cl32[a] = (float)L.cl[a];
    }
    L.dl = __dsqrt_rn(dl2);
    L.dl32 = (float)L.dl;
}

__device__ __forceinline__ uint64_t bh_mix(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// Admissibility of cluster C for target leaf L:
//   boxes strictly disjoint along some axis, and
//   diag(C) < theta * (|X_C - c_L| - diag(L)/2),
// with every quantity in FP64, separately rounded, in a fixed order.  An FP32
// pre-test settles the decision whenever its error bound allows (outward and
// inward rounded boxes for the strict comparisons; a 1e-5 relative margin for
// the size test, far above FP32 rounding); otherwise the FP64 test decides.
__device__ __forceinline__ bool admissible(const LeafAdm& L, const float* c32, const double* bc,
                                           const double* c64, double theta, float theta32) {
    bool sure = false, amb = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (L.out[3 + a] < c32[a] || c32[3 + a] < L.out[a]) sure = true;
        else if (!(L.in[3 + a] >= tp_inward_lo(c32[a]) && tp_inward_hi(c32[3 + a]) >= L.in[a])) amb = true;
    }
    if (!sure) {
        if (!amb) return false;
        bool disjoint = false;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (L.bl[3 + a] < bc[a] || bc[3 + a] < L.bl[a]) disjoint = true;
        if (!disjoint) return false;
    }
    float r2f = 0.f, M = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t = c32[6 + a] - L.cl32[a];
        r2f = fmaf(t, t, r2f);
        M += fabsf(c32[6 + a]) + fabsf(L.cl32[a]);
    }
    // sqrt.approx: the margin below (1e-5 relative) is far above its error
    float distf;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(distf) : "f"(r2f));
    const float rhsf = theta32 * (distf - 0.5f * L.dl32);
    const float lhsf = c32[9];
    const float margin = 1e-5f * (lhsf + theta32 * (distf + L.dl32 + M));
    if (lhsf < rhsf - margin) return true;
    if (lhsf > rhsf + margin) return false;
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = __dsub_rn(c64[a], L.cl[a]);
        r2 = __dadd_rn(r2, __dmul_rn(t, t));
    }
    const double dist = __dsqrt_rn(r2);
    const double rhs = __dmul_rn(theta, __dsub_rn(dist, __dmul_rn(0.5, L.dl)));
    return c64[3] < rhs;
}


// Squared gap between the leaf's and a cluster's FP32 outward-rounded vertex
// boxes (a lower bound of the true gap).  Near clusters at least
// TP_PRECISE_GAP_REL of the mesh's box diagonal away form d from the hi parts
// alone, as the direct kernels' FAST items do: the relative error of d is then
// at most about 2^-24 |x| / gap.
__device__ __forceinline__ float box_gap2(const LeafAdm& L, const float* c32) {
    float g2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float g = fmaxf(0.f, fmaxf(c32[a] - L.out[3 + a], L.out[a] - c32[3 + a]));
        g2 = fmaf(g, g, g2);
    }
    return g2;
}

// FP32 outward-rounded vertex boxes strictly apart along some axis.  Two
// triangles that share a vertex lie in vertex boxes that both hold it, so a
// near cluster whose box is apart from the target leaf's has no member
// adjacent to any target and needs no exclusion test.
__device__ __forceinline__ bool boxes_apart(const LeafAdm& L, const float* c32) {
    bool apart = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (L.out[3 + a] < c32[a] || c32[3 + a] < L.out[a]) apart = true;
    return apart;
}

template <int Q, int MODE>
__global__ void __launch_bounds__(BH_WARPS * 32, TP_BH_MINB) k_bh(BHArgs A) {
    __shared__ int32_t s_stack[BH_WARPS][BH_STACK];
    __shared__ int32_t s_far[BH_WARPS][BH_FAR];
    __shared__ int2 s_near[BH_WARPS][BH_NEAR];    // (first member, count) of clusters apart from the leaf
    __shared__ int2 s_touch[BH_WARPS][BH_TOUCH];  // (first member, count) of clusters touching it
    __shared__ __align__(16) float s_stg[BH_WARPS][16 * BH_PAIR];
    __shared__ int4 s_stg_f[BH_WARPS][32];
    __shared__ LeafAdm s_la[BH_WARPS];  // the leaf's admissibility constants (read by every test)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t li = (int64_t)blockIdx.x * BH_WARPS + warp;
    if (li >= A.nleaves) return;
    int32_t* st = s_stack[warp];
    int32_t* far = s_far[warp];
    float* stg = s_stg[warp];
    int4* stg_f = s_stg_f[warp];
    const int64_t L = A.leaves[li];
    const int64_t fL = A.first[L];
    const int cnt = A.last[L] - A.first[L] + 1;
    if (lane == 0) leaf_adm(A.box + 6 * L, A.bounds, s_la[warp]);
    __syncwarp();
    const LeafAdm& la = s_la[warp];
    const float theta32 = (float)A.theta;
    // a leaf of up to 16 targets (in a tree of any leaf size): lanes t and
    // t + 16 share target t and take alternate source pairs; a larger leaf:
    // one target per lane
    const bool wide = cnt > 16;
    const int t = wide ? lane : (lane & 15);
    const int half = wide ? 0 : (lane >> 4);
    const int nh = wide ? 1 : 2;
    const bool active = t < cnt;
    const int64_t k = fL + t;
    Tgt2 tg;
    int3 tf = make_int3(-2, -2, -2);
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tg.h[c] = bh_f2(A.soa[c * A.ntp + k]);
            tg.l[c] = bh_f2(A.soa[(3 + c) * A.ntp + k]);
            tg.n[c] = bh_f2(A.soa[(6 + c) * A.ntp + k]);
        }
        tg.w = bh_f2(A.soa[9 * A.ntp + k]);
        tf = make_int3(A.Fs[3 * k], A.Fs[3 * k + 1], A.Fs[3 * k + 2]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) tg.h[c] = tg.l[c] = tg.n[c] = bh_f2(0.f);
        tg.w = bh_f2(0.f);
    }
    // the target's sums over the flushes: compensated FP32 (value as - ac)
    float as_[8], ac[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) as_[c] = ac[c] = 0.f;
    // statistics: pair counts of far terms and of near pairs without exclusion
    // tests are taken per node in the traversal (lane of the node), those of
    // touching near nodes per admitted pair
    unsigned long long n_near = 0, n_far = 0, n_farp = 0;
    const unsigned lt = (1u << lane) - 1u;

    // far nodes of the learned form: one run of node ids for the network and
    // the far-field kernel (k_far),
    // reserved with one atomic per run; a run whose ids do not fit is recorded
    // with no rows (the host sees the overflow in the counts and repeats the
    // evaluation)
    auto emit_far = [&](int nf) {
        if (nf == 0) return;
        unsigned long long pos = 0, run = 0;
        if (lane == 0) {
            pos = atomicAdd(&A.far_count[0], (unsigned long long)nf);
            run = atomicAdd(&A.far_count[1], 1ull);
        }
        pos = __shfl_sync(0xffffffffu, pos, 0);
        run = __shfl_sync(0xffffffffu, run, 0);
        const bool fits = pos + (unsigned long long)nf <= (unsigned long long)A.far_cap;
        if (fits)
            for (int i = lane; i < nf; i += 32) {
                A.far_list[pos + i] = far[i];
                A.far_leaf[pos + i] = (int32_t)li;
            }
        if (lane == 0 && run < (unsigned long long)A.run_cap) {
            tp_far_run fr;
            fr.start = fits ? (int64_t)pos : 0;
            fr.li = (int32_t)li;
            fr.len = fits ? nf : 0;
            A.far_runs[run] = fr;
        }
    };
    // far nodes of the plain form: stage 32 node records at a time, then
    // sweep them in pairs (one target against two records per packed step).
    // The list holds nodes whose boxes are at least TP_PRECISE_GAP_REL of the
    // mesh diagonal from the leaf's at its back (far[BH_FAR - 1 - i], i < nff):
    // their differences take the hi parts alone, as k_near's.  The others sit
    // at its front (far[i], i < nfp).  The target weight is applied to the sums.
    auto sweep_far = [&](auto hilo, int nb0, float2 (&a2)[8]) {
        constexpr bool HILO = decltype(hilo)::value;
        for (int b0 = 0; b0 < nb0; b0 += 32) {
            const int nb = nb0 - b0 < 32 ? nb0 - b0 : 32;
            __syncwarp();
            if (lane < nb) {
                const int node = HILO ? far[b0 + lane] : far[BH_FAR - 1 - (b0 + lane)];
                const float4* r = reinterpret_cast<const float4*>(A.nodef + 16 * (int64_t)node);
                const float4 r0 = r[0], r1 = r[1], r2 = r[2];
                const float v[10] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y};
                stage_put(stg, lane, v);
            } else if (lane == nb && (nb & 1)) {
                stage_pad(stg, lane);
            }
            __syncwarp();
            const int np = (nb + 1) >> 1;
            for (int p = half; p < np; p += nh) gather_pair2<Q, false, HILO, true>(tg, stg, p, a2);
        }
    };
    auto flush_far = [&](int nfp, int nff) {
        if constexpr (MODE == M_LIST) {
            emit_far(nfp);
        } else {
            float2 a2[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
            sweep_far(std::true_type{}, nfp, a2);
            sweep_far(std::false_type{}, nff, a2);
            const float tw = tg.w.x;
#pragma unroll
            for (int c = 0; c < 8; ++c) ksum_add(as_[c], ac[c], (a2[c].x + a2[c].y) * tw);
        }
    };
    // near clusters apart from the leaf: one run of (first member, count)
    // entries for the near-field kernel (k_near), reserved with one atomic per
    // run; a run whose entries do not fit is recorded with no entries (the
    // host sees the overflow in the counts and repeats the evaluation)
    auto emit_near = [&](int nn) {
        if (nn == 0) return;
        unsigned long long pos = 0, run = 0;
        if (lane == 0) {
            pos = atomicAdd(&A.near_count[0], (unsigned long long)nn);
            run = atomicAdd(&A.near_count[1], 1ull);
        }
        pos = __shfl_sync(0xffffffffu, pos, 0);
        run = __shfl_sync(0xffffffffu, run, 0);
        const bool fits = pos + (unsigned long long)nn <= (unsigned long long)A.near_cap;
        // the run's ordered pairs (all, and those with hi-only differences) for the statistics
        unsigned int rp = 0, rh = 0;
        for (int i = lane; i < nn; i += 32) {
            const int c = s_near[warp][i].y;
            rp += (unsigned)(c < 0 ? -c : c);
            if (c < 0) rh += (unsigned)-c;
        }
        for (int o = 16; o > 0; o >>= 1) {
            rp += __shfl_xor_sync(0xffffffffu, rp, o);
            rh += __shfl_xor_sync(0xffffffffu, rh, o);
        }
        if (lane == 0) {
            atomicAdd(&A.near_listed[0], (unsigned long long)rp * (unsigned long long)cnt);
            atomicAdd(&A.near_listed[1], (unsigned long long)rh * (unsigned long long)cnt);
        }
        if (fits) {
            // the clusters with hi/lo differences first, then the hi-only ones, so
            // that k_near's slots (one kind each) stay full
            int o = 0;
            for (int kind = 0; kind < 2; ++kind)
                for (int i0 = 0; i0 < nn; i0 += 32) {
                    const int i = i0 + lane;
                    const int2 e = i < nn ? s_near[warp][i] : make_int2(0, 0);
                    const bool take = i < nn && (e.y < 0) == (kind == 1);
                    const unsigned bal = __ballot_sync(0xffffffffu, take);
                    if (take) A.near_list[pos + o + __popc(bal & lt)] = e;
                    o += __popc(bal);
                }
        }
        if (lane == 0 && run < (unsigned long long)A.nrun_cap) {
            tp_far_run nr;
            nr.start = fits ? (int64_t)pos : 0;
            nr.li = (int32_t)li;
            nr.len = fits ? nn : 0;
            A.near_runs[run] = nr;
        }
    };
    // near clusters whose box touches the leaf's: stage the members of up to
    // 32 sources at a time (whole clusters), then sweep them in pairs with the
    // exclusion test on every pair
    auto flush_touch = [&](const int2* nl, int nn) {
        float2 a2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
        int i = 0;
        while (i < nn) {
            // take whole nodes while they fit in 32 slots
            int nsrc = 0, i1 = i;
            while (i1 < nn && nsrc + nl[i1].y <= 32) nsrc += nl[i1++].y;
            __syncwarp();
            // lane -> (node, member) by walking the taken nodes
            {
                int base = 0;
                for (int j = i; j < i1; ++j) {
                    const int2 nd = nl[j];
                    if (lane >= base && lane < base + nd.y) {
                        const int64_t s = (int64_t)nd.x + (lane - base);
                        float v[10];
#pragma unroll
                        for (int c = 0; c < 10; ++c) v[c] = A.soa[c * A.ntp + s];
                        stage_put(stg, lane, v);
                        stg_f[lane] = make_int4(A.Fs[3 * s], A.Fs[3 * s + 1], A.Fs[3 * s + 2], (int)s);
                    }
                    base += nd.y;
                }
                if (lane == nsrc && (nsrc & 1)) {
                    stage_pad(stg, lane);
                    stg_f[lane] = make_int4(-1, -1, -1, -1);
                }
            }
            __syncwarp();
            const int np = (nsrc + 1) >> 1;
            for (int p = half; p < np; p += nh) {
                const int4 f0 = stg_f[2 * p], f1 = stg_f[2 * p + 1];
                const bool v0 = active && f0.w >= 0 && f0.w != (int)k &&
                                !adjacent(tf, make_int3(f0.x, f0.y, f0.z), A.edge_only);
                const bool v1 = active && f1.w >= 0 && f1.w != (int)k &&
                                !adjacent(tf, make_int3(f1.x, f1.y, f1.z), A.edge_only);
                gather_pair2<Q, true>(tg, stg, p, a2, v0, v1);
                n_near += (unsigned long long)(v0 + v1);
            }
            i = i1;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) ksum_add(as_[c], ac[c], a2[c].x + a2[c].y);
    };

    int sp = 1, nfp = 0, nff = 0, nn[2] = {0, 0};
    if (lane == 0) st[0] = 0;  // root
    __syncwarp();
    bool overflow = false;
    while (sp > 0) {
        const int m = sp < 32 ? sp : 32;
        const int node = lane < m ? st[sp - 1 - lane] : -1;
        __syncwarp();
        sp -= m;
        bool is_far = false, is_near = false, is_open = false, touch = false, fast = false, ffast = false;
        int firstc = 0, cntc = 0, lc = 0, rc = 0;
        if (node >= 0 && tp_dbg_ok(node < 2 * A.n - 1, A.derr)) {
            // everything the test and the push need, in one round of four 16-byte
            // loads of the node's record: box, centroid, diagonal, member range
            // and children
            const float4* c4 = reinterpret_cast<const float4*>(A.adm32 + TP_ADM32_W * (int64_t)node);
            const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2], q3 = c4[3];
            firstc = __float_as_int(q2.z);
            const int lastc = __float_as_int(q2.w);
            lc = __float_as_int(q3.x);
            rc = __float_as_int(q3.y);
            cntc = lastc - firstc + 1;
            const float c32[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                                   q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
            if (admissible(la, c32, A.box + 6 * (int64_t)node, A.adm64 + 4 * (int64_t)node, A.theta, theta32)) {
                is_far = true;
                ffast = TP_FAR_FAST && MODE == M_BH && box_gap2(la, c32) >= la.fast2;
                n_far += (unsigned long long)cnt;
                n_farp += (unsigned long long)cnt * (unsigned long long)cntc;
            } else if (cntc <= A.leaf_size || node >= A.n - 1) {
                is_near = true;
                touch = !boxes_apart(la, c32);
                if (!touch) {
                    n_near += (unsigned long long)cnt * (unsigned long long)cntc;
                    fast = box_gap2(la, c32) >= la.fast2;
                }
            } else {
                is_open = tp_dbg_ok(lc >= 0 && lc < 2 * A.n - 1 && rc >= 0 && rc < 2 * A.n - 1 &&
                                        A.first[node] == firstc && A.last[node] == lastc,
                                    A.derr);
            }
        }
        const unsigned bfp = __ballot_sync(0xffffffffu, is_far && !ffast);
        const unsigned bff = __ballot_sync(0xffffffffu, is_far && ffast);
        const unsigned bn0 = __ballot_sync(0xffffffffu, is_near && !touch);
        const unsigned bn1 = __ballot_sync(0xffffffffu, is_near && touch);
        const unsigned bo = __ballot_sync(0xffffffffu, is_open);
        if (sp + 2 * __popc(bo) > BH_STACK) {
            overflow = true;
            break;
        }
        if (MODE == M_RECORD) {
            if (is_far) {
                const uint64_t h = bh_mix(A.seed ^ (((uint64_t)li << 32) | (uint32_t)node));
                if ((uint32_t)(h >> 32) < A.keep_u || A.keep_u == 0xffffffffu) {
                    const int32_t pos = atomicAdd(A.rec_count, 1);
                    if (pos < A.rec_cap) A.rec_out[pos] = make_int2((int)li, node);
                }
            }
        } else {
            if (is_far && !ffast) far[nfp + __popc(bfp & lt)] = node;
            if (is_far && ffast) far[BH_FAR - 1 - (nff + __popc(bff & lt))] = node;
            // (first member, count); a negative count marks a cluster whose pairs take the hi parts only
            if (is_near && !touch) s_near[warp][nn[0] + __popc(bn0 & lt)] = make_int2(firstc, fast ? -cntc : cntc);
            if (is_near && touch) s_touch[warp][nn[1] + __popc(bn1 & lt)] = make_int2(firstc, cntc);
        }
        if (is_open) {
            const int pos = sp + 2 * __popc(bo & lt);
            st[pos] = rc;
            st[pos + 1] = lc;
        }
        if (MODE != M_RECORD) {
            nfp += __popc(bfp);
            nff += __popc(bff);
            nn[0] += __popc(bn0);
            nn[1] += __popc(bn1);
        }
        sp += 2 * __popc(bo);
        __syncwarp();
        if (nfp + nff > BH_FAR - 32) {
            flush_far(nfp, nff);
            nfp = nff = 0;
        }
        if (nn[0] > BH_NEAR - 32) {
            emit_near(nn[0]);
            nn[0] = 0;
        }
        if (nn[1] > BH_TOUCH - 32) {
            flush_touch(s_touch[warp], nn[1]);
            nn[1] = 0;
        }
        __syncwarp();
    }
    if (overflow) {
        if (lane == 0) tp_dev_error(A.derr, TP_DERR_STACK);
        return;
    }
    if (MODE == M_RECORD) return;
    flush_far(nfp, nff);
    emit_near(nn[0]);
    flush_touch(s_touch[warp], nn[1]);
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = (double)as_[c] - (double)ac[c];
    if (!wide) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
    }
    if (half == 0 && active) {
#pragma unroll
        for (int c = 0; c < 8; ++c) A.acc[c * A.ntp + k] = acc[c];
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_near += __shfl_xor_sync(0xffffffffu, n_near, o);
        n_far += __shfl_xor_sync(0xffffffffu, n_far, o);
        n_farp += __shfl_xor_sync(0xffffffffu, n_farp, o);
    }
    if (lane == 0) {
        atomicAdd(&A.counts[0], n_near);
        atomicAdd(&A.counts[1], n_far);
        atomicAdd(&A.counts[2], n_farp);
        atomicAdd(A.far_rows, n_far / (unsigned long long)cnt);  // far terms = cnt x far nodes of this leaf
    }
}

// ------------------------------------------------------------ near field
// The near clusters apart from a leaf (listed by k_bh in runs of up to
// BH_NEAR clusters) are summed by k_near, one warp per run (taken from a work
// counter).  Lanes are (target pair, source stream), sized to the leaf: its
// cnt targets make np = ceil(cnt / 2) pairs and the warp runs 32 / np streams
// (a leaf of 11 triangles: 6 pairs x 5 streams), so few lanes idle; each lane
// evaluates its two targets against every ns-th source in packed FP32x2
// arithmetic.  Sources are the direct kernels' records (80 B, each value
// twice, so one record feeds both halves): whole clusters are copied into a
// two-slot ring of NR_SLOT records per warp with cp.async.bulk, completion on
// an mbarrier per slot (bounded waits), so the next slot's copies run while
// this one is evaluated.  The energy channel is folded into FP64 after every
// slot; at the end of the run the streams are summed through shared memory
// (the ring, free by then) and the targets' FP64 accumulators are updated
// atomically (runs of one leaf may be
// in flight in several warps, after k_bh has stored its own part).
#ifndef TP_NR_SLOT
#define TP_NR_SLOT 56
#endif
#ifndef TP_NR_BPS
#define TP_NR_BPS 5  // k_near blocks per SM: 5 x 40 KB of shared memory, 20 warps
#endif
constexpr int NR_WARPS = 4;
constexpr int NR_SLOT = TP_NR_SLOT;  // source records per ring slot
static_assert(NR_SLOT >= 32, "a slot must hold the largest cluster leaf (32 triangles)");

struct NearWarpSmem {
    float rec[2][NR_SLOT * TP_SRCW];
    int2 ent[BH_NEAR];
    uint64_t bar[2];
};

template <int Q>
__global__ void __launch_bounds__(NR_WARPS * 32, TP_NR_BPS) k_near(BHArgs A) {
    __shared__ __align__(128) NearWarpSmem s_w[NR_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    NearWarpSmem& S = s_w[warp];
    if (lane == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t ph0 = 0u, ph1 = 0u;  // phase parities of the two slots' mbarriers (scalars: no local memory)
    const unsigned long long nr = A.near_count[1];
    const int64_t nruns = nr < (unsigned long long)A.nrun_cap ? (int64_t)nr : A.nrun_cap;
    bool failed = false;
    while (!failed) {
        int64_t run = 0;
        if (lane == 0) run = (int64_t)atomicAdd(&A.near_count[2], 1ull);
        run = __shfl_sync(0xffffffffu, run, 0);
        if (run >= nruns) break;
        const tp_far_run R = A.near_runs[run];
        if (R.len <= 0 || R.len > BH_NEAR || R.li < 0 || (int64_t)R.li >= A.nleaves || R.start < 0 ||
            R.start + R.len > A.near_cap)
            continue;  // a run whose entries overflowed the list (the evaluation is repeated)
        const int64_t L = A.leaves[R.li];
        const int64_t fL = A.first[L];
        const int cnt = A.last[L] - A.first[L] + 1;
#if TP_DEBUG
        {
            // the leaf's targets and every listed member range within the triangles
            bool ok = fL >= 0 && cnt >= 1 && cnt <= 32 && fL + cnt <= A.ntp;
            for (int i = lane; i < R.len; i += 32) {
                const int2 e = A.near_list[R.start + i];
                const int c = e.y < 0 ? -e.y : e.y;
                ok = ok && c >= 1 && c <= 32 && e.x >= 0 && (int64_t)e.x + c <= A.ntp;
            }
            if (!__all_sync(0xffffffffu, tp_dbg_ok(ok, A.derr))) continue;
        }
#endif
        const int npair = (cnt + 1) >> 1;           // target pairs
        const int ng = 32 / npair;                  // source streams
        const int tpl = lane % npair, g = lane / npair;  // this lane's pair and stream (g >= ng: idle)
        for (int i = lane; i < R.len; i += 32) S.ent[i] = A.near_list[R.start + i];
        // this lane's two targets, fL + 2 tpl + h (h = 0, 1); absent ones have zero weight
        Tgt2 tg;
        bool act[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 2 * tpl + h;
            act[h] = t < cnt && g < ng;
            const int64_t k = fL + (act[h] ? t : 0);
            float v[10];
#pragma unroll
            for (int c = 0; c < 10; ++c) v[c] = act[h] ? A.soa[c * A.ntp + k] : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                (h ? tg.h[c].y : tg.h[c].x) = v[c];
                (h ? tg.l[c].y : tg.l[c].x) = v[3 + c];
                (h ? tg.n[c].y : tg.n[c].x) = v[6 + c];
            }
            (h ? tg.w.y : tg.w.x) = v[9];
        }
        __syncwarp();
        // slot planning: whole clusters of one kind (a negative count marks a
        // cluster whose pairs take the hi parts only) while they fit.  The warp
        // plans up to 32 entries at a time: a ballot finds where the kind
        // changes, a scan of the counts where the slot is full, and every lane
        // of the taken prefix issues its own cluster's copy (at most two rounds:
        // a slot holds at most NR_SLOT <= 64 clusters of one record).
        static_assert(NR_SLOT <= 64, "two planning rounds of 32 entries fill a slot");
        int next = 0, ns0 = 0, ns1 = 0;  // records planned into slot 0 / 1 and not yet consumed
        bool hi0 = false, hi1 = false;   // the slot's clusters take the hi parts only
        auto plan = [&](int b) {
            int n = 0;
            const bool hi = next < R.len && S.ent[next].y < 0;
            int my_e[2] = {-1, -1}, my_o[2] = {0, 0};  // this lane's entries and their record offsets
#pragma unroll
            for (int round = 0; round < 2; ++round) {
                if (next >= R.len) break;  // warp-uniform
                const int e = next + lane;
                const int2 en = e < R.len ? S.ent[e] : make_int2(0, 0);
                const int c = abs(en.y);
                const bool same = e < R.len && (en.y < 0) == hi;
                const unsigned brk = __ballot_sync(0xffffffffu, !same);
                const int f = brk ? __ffs(brk) - 1 : 32;  // entries of the slot's kind: lanes < f
                int incl = lane < f ? c : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                // counts are >= 1, so the entries that fit form a prefix
                const bool take = lane < f && n + incl <= NR_SLOT;
                const int m = __popc(__ballot_sync(0xffffffffu, take));
                if (take) {
                    my_e[round] = e;
                    my_o[round] = n + incl - c;
                }
                n += m ? __shfl_sync(0xffffffffu, incl, m - 1) : 0;
                next += m;
                if (m < 32) break;
            }
            if (b) {
                ns1 = n;
                hi1 = hi;
            } else {
                ns0 = n;
                hi0 = hi;
            }
            if (n == 0) {
                // a cluster larger than a slot cannot occur (leaves hold at most 32)
                if (next < R.len && lane == 0) tp_dev_error(A.derr, TP_DERR_INTERNAL);
                return;
            }
            if (lane == 0) mbar_expect_tx(&S.bar[b], (uint32_t)(n * TP_SRCW * 4));
            __syncwarp();  // the expected bytes are set before any copy can complete
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (my_e[r] < 0) continue;
                const int2 en = S.ent[my_e[r]];
                tma_load_1d(S.rec[b] + my_o[r] * TP_SRCW, A.src + (int64_t)en.x * TP_SRCW,
                            (uint32_t)(abs(en.y) * TP_SRCW * 4), &S.bar[b]);
            }
        };
        plan(0);
        plan(1);
        float2 a2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
        KSum2 ek = {bh_f2(0.f), bh_f2(0.f)};  // the energy channel, folded after every slot
        for (int slot = 0;; ++slot) {
            const int b = slot & 1;
            const int n = b ? ns1 : ns0;
            if (n == 0) break;  // nothing planned (an empty run)
            const bool ok = mbar_wait_bounded(&S.bar[b], b ? ph1 : ph0);
            if (!__all_sync(0xffffffffu, ok)) {  // the same decision in every lane
                failed = true;
                break;
            }
            if (b) {
                ph1 ^= 1u;
                ns1 = 0;  // consumed (planned again below)
            } else {
                ph0 ^= 1u;
                ns0 = 0;
            }
            const float* rb = S.rec[b];
            if (g < ng) {
                if (b ? hi1 : hi0)
                    for (int j = g; j < n; j += ng) near_pair2<Q, false>(tg, rb + j * TP_SRCW, a2);
                else
                    for (int j = g; j < n; j += ng) near_pair2<Q, true>(tg, rb + j * TP_SRCW, a2);
            }
            ksum2_add(ek, a2[0]);
            a2[0] = bh_f2(0.f);
            __syncwarp();  // every lane is done with slot b before it is refilled
            plan(b);
            if (ns0 == 0 && ns1 == 0) break;
        }
        if (failed) {
            // copies of either slot may still be in flight: wait for them (bounded,
            // the phases of slots not yet consumed) before this warp stops using
            // its shared memory
            if (lane == 0) tp_dev_error(A.derr, TP_DERR_TIMEOUT);
            if (ns0 > 0) mbar_wait_bounded(&S.bar[0], ph0);
            if (ns1 > 0) mbar_wait_bounded(&S.bar[1], ph1);
            break;
        }
        // sum the source streams through shared memory (the ring is free: every
        // planned slot has been consumed) and add to the targets
        float* red = S.rec[0];  // [32 lanes][16] channel partials of both targets
        double* ered = reinterpret_cast<double*>(S.rec[1]);  // [32 lanes][2] energies
#pragma unroll
        for (int c = 1; c < 8; ++c) {
            red[lane * 16 + 2 * c] = a2[c].x;
            red[lane * 16 + 2 * c + 1] = a2[c].y;
        }
        double e64[2] = {(double)ek.s.x - (double)ek.c.x, (double)ek.s.y - (double)ek.c.y};
        ered[2 * lane] = e64[0];
        ered[2 * lane + 1] = e64[1];
        __syncwarp();
        if (lane < npair) {
            for (int gg = 1; gg < ng; ++gg) {
                const int o = gg * npair + lane;
#pragma unroll
                for (int c = 1; c < 8; ++c) {
                    a2[c].x += red[o * 16 + 2 * c];
                    a2[c].y += red[o * 16 + 2 * c + 1];
                }
                e64[0] += ered[2 * o];
                e64[1] += ered[2 * o + 1];
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!act[h]) continue;
                const int64_t k = fL + 2 * tpl + h;
                const float w = h ? tg.w.y : tg.w.x;  // the target weight left out of the pair terms
                atomicAdd(&A.acc[k], e64[h] * (double)w);
#pragma unroll
                for (int c = 1; c < 8; ++c)
                    atomicAdd(&A.acc[c * A.ntp + k], (double)(h ? a2[c].y : a2[c].x) * (double)w);
            }
        }
        __syncwarp();  // the entry list is reused by the next run
    }
}

// Block-wide form of k_near (see TP_NR_BLOCK): one run per block of 128 threads,
// lanes (target pair, source stream) over the whole block, so a leaf of cnt
// targets keeps ceil(cnt/2) x floor(128 / pairs) threads busy (22 targets: 121
// of 128, where a warp keeps 22 of 32); one ring of two slots of NB_SLOT
// records per block.  Warp 0 plans the slots and issues the copies; a block
// barrier per slot orders the reuse of a slot.  Numerics as in k_near.
#ifndef TP_NR_BLOCK
#define TP_NR_BLOCK 2  // 0: k_near always; 1: k_near_blk always; 2: k_near_blk for trees with leaves of more than 16
#endif
// Measured on the level-7 sphere: with leaves of 32 the block-wide form took the
// near-field launch from 19.2 to 17.4 ms (theta 0.085, six blocks per SM); with
// leaves of 16, whose runs are shorter and whose warps are already well filled,
// it was slower (22.2 against 28.3 ms at theta 0.0625).
__host__ __device__ constexpr bool near_block_form(int leaf_size) {
    return TP_NR_BLOCK == 1 || (TP_NR_BLOCK == 2 && leaf_size > 16);
}
#ifndef TP_NB_BPS
#define TP_NB_BPS 6  // k_near_blk blocks per SM: 6 x 37 KB of shared memory, at most 85 registers
#endif
#ifndef TP_NB_SLOT
#define TP_NB_SLOT 216  // with 256-entry runs: 6 x 37.7 KB of shared memory per SM
#endif
constexpr int NB_THREADS = NR_WARPS * 32;
constexpr int NB_SLOT = TP_NB_SLOT;  // records per ring slot

struct NearBlockSmem {
    float rec[2][NB_SLOT * TP_SRCW];
    int2 ent[BH_NEAR];
    uint64_t bar[2];
    int ns[2];  // records planned into each slot and not yet consumed (0: none)
    int hi[2];  // the slot's clusters take the hi parts only
    long long work;
};

template <int Q>
__global__ void __launch_bounds__(NB_THREADS, TP_NB_BPS) k_near_blk(BHArgs A) {
    __shared__ __align__(128) NearBlockSmem S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t ph0 = 0u, ph1 = 0u;  // phase parities of the two slots' mbarriers
    const unsigned long long nr = A.near_count[1];
    const int64_t nruns = nr < (unsigned long long)A.nrun_cap ? (int64_t)nr : A.nrun_cap;
    while (true) {
        if (tid == 0) S.work = (long long)atomicAdd(&A.near_count[2], 1ull);
        __syncthreads();
        const int64_t run = S.work;
        __syncthreads();  // every thread has read the item before thread 0 takes the next
        if (run >= nruns) break;
        const tp_far_run R = A.near_runs[run];
        if (R.len <= 0 || R.len > BH_NEAR || R.li < 0 || (int64_t)R.li >= A.nleaves || R.start < 0 ||
            R.start + R.len > A.near_cap)
            continue;  // a run whose entries overflowed the list (the evaluation is repeated)
        const int64_t L = A.leaves[R.li];
        const int64_t fL = A.first[L];
        const int cnt = A.last[L] - A.first[L] + 1;
#if TP_DEBUG
        {
            bool ok = fL >= 0 && cnt >= 1 && cnt <= 32 && fL + cnt <= A.ntp;
            for (int i = tid; i < R.len; i += NB_THREADS) {
                const int2 e = A.near_list[R.start + i];
                const int c = e.y < 0 ? -e.y : e.y;
                ok = ok && c >= 1 && c <= 32 && e.x >= 0 && (int64_t)e.x + c <= A.ntp;
            }
            if (!__syncthreads_and(tp_dbg_ok(ok, A.derr))) continue;
        }
#endif
        const int npair = (cnt + 1) >> 1;                // target pairs
        const int ng = NB_THREADS / npair;               // source streams
        const int tpl = tid % npair, g = tid / npair;    // this thread's pair and stream (g >= ng: idle)
        for (int i = tid; i < R.len; i += NB_THREADS) S.ent[i] = A.near_list[R.start + i];
        Tgt2 tg;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 2 * tpl + h;
            const bool act = t < cnt && g < ng;
            const int64_t k = fL + (act ? t : 0);
            float v[10];
#pragma unroll
            for (int c = 0; c < 10; ++c) v[c] = act ? A.soa[c * A.ntp + k] : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                (h ? tg.h[c].y : tg.h[c].x) = v[c];
                (h ? tg.l[c].y : tg.l[c].x) = v[3 + c];
                (h ? tg.n[c].y : tg.n[c].x) = v[6 + c];
            }
            (h ? tg.w.y : tg.w.x) = v[9];
        }
        __syncthreads();  // the entries are in shared memory
        // slot planning by warp 0, as in k_near (at most two rounds of 32
        // entries per slot); `next` lives in warp 0's registers
        int next = 0;
        auto plan = [&](int b) {
            int n = 0;
            const bool hi = next < R.len && S.ent[next].y < 0;
            int my_e[2] = {-1, -1}, my_o[2] = {0, 0};
#pragma unroll
            for (int round = 0; round < 2; ++round) {
                if (next >= R.len) break;
                const int e = next + lane;
                const int2 en = e < R.len ? S.ent[e] : make_int2(0, 0);
                const int c = abs(en.y);
                const bool same = e < R.len && (en.y < 0) == hi;
                const unsigned brk = __ballot_sync(0xffffffffu, !same);
                const int f = brk ? __ffs(brk) - 1 : 32;
                int incl = lane < f ? c : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const bool take = lane < f && n + incl <= NB_SLOT;
                const int m = __popc(__ballot_sync(0xffffffffu, take));
                if (take) {
                    my_e[round] = e;
                    my_o[round] = n + incl - c;
                }
                n += m ? __shfl_sync(0xffffffffu, incl, m - 1) : 0;
                next += m;
                if (m < 32) break;
            }
            if (lane == 0) {
                S.ns[b] = n;
                S.hi[b] = hi ? 1 : 0;
            }
            if (n == 0) {
                if (next < R.len && lane == 0) tp_dev_error(A.derr, TP_DERR_INTERNAL);
                return;
            }
            if (lane == 0) mbar_expect_tx(&S.bar[b], (uint32_t)(n * TP_SRCW * 4));
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (my_e[r] < 0) continue;
                const int2 en = S.ent[my_e[r]];
                tma_load_1d(S.rec[b] + my_o[r] * TP_SRCW, A.src + (int64_t)en.x * TP_SRCW,
                            (uint32_t)(abs(en.y) * TP_SRCW * 4), &S.bar[b]);
            }
        };
        if (warp == 0) {
            plan(0);
            plan(1);
        }
        __syncthreads();  // the slot sizes are in shared memory
        float2 a2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
        KSum2 ek = {bh_f2(0.f), bh_f2(0.f)};
        bool failed = false;
        for (int slot = 0;; ++slot) {
            const int b = slot & 1;
            const int n = S.ns[b];  // planned before the last block barrier
            if (n == 0) break;
            // a thread whose wait gave up still reads the slot (in bounds, values
            // undefined); the barrier below, which also orders the slot's reuse,
            // makes every thread see the failure, and the run is abandoned
            const bool ok = mbar_wait_bounded(&S.bar[b], b ? ph1 : ph0);
            const float* rb = S.rec[b];
            if (g < ng) {
                if (S.hi[b])
                    for (int j = g; j < n; j += ng) near_pair2<Q, false>(tg, rb + j * TP_SRCW, a2);
                else
                    for (int j = g; j < n; j += ng) near_pair2<Q, true>(tg, rb + j * TP_SRCW, a2);
            }
            ksum2_add(ek, a2[0]);
            a2[0] = bh_f2(0.f);
            // every thread is done with slot b before it is planned again
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            if (b) ph1 ^= 1u;
            else ph0 ^= 1u;
            if (warp == 0) plan(b);
        }
        if (failed) {
            // copies of either slot may still be in flight: wait for them (bounded)
            // before the block leaves its shared memory
            if (tid == 0) {
                tp_dev_error(A.derr, TP_DERR_TIMEOUT);
                if (S.ns[0] > 0) mbar_wait_bounded(&S.bar[0], ph0);
                if (S.ns[1] > 0) mbar_wait_bounded(&S.bar[1], ph1);
            }
            break;
        }
        // the streams' sums through shared memory (the ring is free), then one
        // thread per (target pair, channel) adds both targets' totals
        float* red = S.rec[0];                               // [128][16] channel partials
        double* ered = reinterpret_cast<double*>(S.rec[1]);  // [128][2] energies
#pragma unroll
        for (int c = 1; c < 8; ++c) {
            red[tid * 16 + 2 * c] = a2[c].x;
            red[tid * 16 + 2 * c + 1] = a2[c].y;
        }
        ered[2 * tid] = (double)ek.s.x - (double)ek.c.x;
        ered[2 * tid + 1] = (double)ek.s.y - (double)ek.c.y;
        __syncthreads();
        for (int item = tid; item < 8 * npair; item += NB_THREADS) {
            const int p = item % npair, c = item / npair;
            double v[2] = {0.0, 0.0};
            float f[2] = {0.f, 0.f};
            for (int gg = 0; gg < ng; ++gg) {
                const int o = gg * npair + p;
                if (c == 0) {
                    v[0] += ered[2 * o];
                    v[1] += ered[2 * o + 1];
                } else {
                    f[0] += red[o * 16 + 2 * c];
                    f[1] += red[o * 16 + 2 * c + 1];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = 2 * p + h;
                if (t >= cnt) continue;
                const int64_t k = fL + t;
                const double w = (double)A.soa[9 * A.ntp + k];  // the target weight left out of the pair terms
                atomicAdd(&A.acc[c * A.ntp + k], (c == 0 ? v[h] : (double)f[h]) * w);
            }
        }
        __syncthreads();  // the entries and the ring are reused by the next run
    }
}

// ------------------------------------------------------------ learned far field
// In the learned form the far nodes of every leaf (listed by k_bh in runs of
// up to BH_FAR nodes) are evaluated by k_far after the network, one warp per
// run (taken from a work counter), with the same leaf-sized lanes as k_near:
// (target pair, record stream).  Each batch of 32 listed nodes is staged in
// shared memory in the duplicated record layout with the network's channel
// factors; the next batch's records are loaded into registers while this one
// is evaluated.  The channels of the far term are scaled by the factors
// f_c = exp(y_c) of its (leaf, cluster) row (1 outside the training ranges):
// E = wts (f0 al^q + f1 be^q), U: f2 A5, Gx: f4 B5 nubar - k d,
// k = (p/q) wts inv (f5 al^q + f6 be^q).  The normal-derivative channel Gn
// keeps the monopole A5 d: its factor is fitted to the channel's projection on
// the target-cluster direction, and applied to the whole vector it doubled the
// gradient error (level-7 sphere, theta = 0.25, a model trained at theta =
// 0.25 and 0.5: 8.3e-3 with it, 3.9e-3 without, 4.4e-3 for plain Barnes-Hut).  (The plain form evaluates its far
// nodes inside k_bh, straight from the traversal's staged list.)
// EO (energy only): fk[0], fk[1] hold f0 - 1 and f1 - 1, every accumulator
// takes the monopole, and the energy correction wts ((f0-1) al^q + (f1-1) be^q)
// goes to dacc.
template <int Q, bool EO>
__device__ __forceinline__ void far_pair2_learned(const Tgt2& t, const float* rec, const float* fk, float2 acc[8],
                                                  float2& dacc) {
    const float4* r = reinterpret_cast<const float4*>(rec);
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
    const float2 sh[3] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w), make_float2(r1.x, r1.y)};
    const float2 sl[3] = {make_float2(r1.z, r1.w), make_float2(r2.x, r2.y), make_float2(r2.z, r2.w)};
    const float2 sn[3] = {make_float2(r3.x, r3.y), make_float2(r3.z, r3.w), make_float2(r4.x, r4.y)};
    const float2 sw = make_float2(r4.z, r4.w);
    const float4 f03 = reinterpret_cast<const float4*>(fk)[0], f47 = reinterpret_cast<const float4*>(fk)[1];
    float2 d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = bh_add2(bh_add2(t.h[k], bh_neg2(sh[k])), bh_add2(t.l[k], bh_neg2(sl[k])));
    float2 r2s = bh_mul2(d[0], d[0]);
    r2s = bh_fma2(d[1], d[1], r2s);
    r2s = bh_fma2(d[2], d[2], r2s);
    const float2 wts = bh_mul2(t.w, sw);
    const float2 inv = make_float2(bh_rcp(r2s.x), bh_rcp(r2s.y));
    float2 a = bh_mul2(t.n[0], d[0]);
    a = bh_fma2(t.n[1], d[1], a);
    a = bh_fma2(t.n[2], d[2], a);
    float2 b = bh_mul2(sn[0], d[0]);
    b = bh_fma2(sn[1], d[1], b);
    b = bh_fma2(sn[2], d[2], b);
    const float2 al = bh_mul2(a, inv), be = bh_mul2(b, inv);
    const float2 al2 = bh_mul2(al, al), be2 = bh_mul2(be, be);
    const float2 al4 = bh_mul2(al2, al2), be4 = bh_mul2(be2, be2);
    float2 alq, beq, al5, be5;
    if (Q == 6) {
        alq = bh_mul2(al4, al2);
        beq = bh_mul2(be4, be2);
        al5 = bh_mul2(al4, al);
        be5 = bh_mul2(be4, be);
    } else {
        alq = bh_mul2(al4, al4);
        beq = bh_mul2(be4, be4);
        al5 = bh_mul2(bh_mul2(al4, al2), al);
        be5 = bh_mul2(bh_mul2(be4, be2), be);
    }
    const float2 wi = bh_mul2(wts, inv);
    const float2 A5 = bh_mul2(wi, al5), B5 = bh_mul2(wi, be5);
    if constexpr (EO) {
        const float2 s6 = bh_add2(alq, beq);
        const float2 nk = bh_mul2(bh_mul2(wi, s6), bh_f2(-2.0f));
        acc[0] = bh_fma2(wts, s6, acc[0]);
        dacc = bh_fma2(wts, bh_fma2(bh_f2(f03.y), beq, bh_mul2(bh_f2(f03.x), alq)), dacc);
        acc[1] = bh_add2(acc[1], A5);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[2 + k] = bh_fma2(A5, d[k], acc[2 + k]);
            acc[5 + k] = bh_fma2(nk, d[k], bh_fma2(B5, sn[k], acc[5 + k]));
        }
        return;
    }
    const float2 se = bh_fma2(bh_f2(f03.y), beq, bh_mul2(bh_f2(f03.x), alq));
    const float2 sk = bh_fma2(bh_f2(f47.z), beq, bh_mul2(bh_f2(f47.y), alq));
    const float2 nk = bh_mul2(bh_mul2(wi, sk), bh_f2(-2.0f));  // -(p/q) wts inv (f5 al^q + f6 be^q)
    const float2 gB = bh_mul2(bh_f2(f47.x), B5);  // (f3, the Gn factor, is not applied)
    acc[0] = bh_fma2(wts, se, acc[0]);
    acc[1] = bh_fma2(bh_f2(f03.z), A5, acc[1]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[2 + k] = bh_fma2(A5, d[k], acc[2 + k]);
        acc[5 + k] = bh_fma2(nk, d[k], bh_fma2(gB, sn[k], acc[5 + k]));
    }
}

constexpr int FAR_WARPS = 8;

// first index i in the sorted a[0, n) with a[i] >= v
__device__ __forceinline__ int64_t bh_lower_bound(const int64_t* a, int64_t n, int64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The runs (in first-row order) that hold rows of the window [w0, w1): the runs
// tile the listed rows, so they are the run holding w0 up to the last one
// starting below w1.
__device__ __forceinline__ void window_runs(const int64_t* skey, int64_t nruns, int64_t w0, int64_t w1, int64_t& lo,
                                            int64_t& hi) {
    lo = bh_lower_bound(skey, nruns, w0 + 1) - 1;
    if (lo < 0) lo = 0;
    hi = bh_lower_bound(skey, nruns, w1);
}

// Window boundaries of the learned passes, moved onto run starts: bnd[k] is
// the first row of the first run starting at or after row k win (the listed
// rows if none).  No run is then split between windows, so its FP32 sums do
// not depend on where the listing placed its rows.  A window holds fewer
// than win + BH_FAR rows.
__global__ void k_window_bounds(const int64_t* __restrict__ skey, int64_t nruns, int64_t win, int64_t nwin,
                                int64_t rows, int64_t* __restrict__ bnd) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > nwin) return;
    if (k == 0 || k == nwin) {
        bnd[k] = k == 0 ? 0 : rows;
        return;
    }
    const int64_t i = bh_lower_bound(skey, nruns, k * win);
    bnd[k] = i < nruns ? skey[i] : rows;
}

__global__ void k_run_keys(const tp_far_run* __restrict__ runs, int64_t nruns, int64_t* __restrict__ key,
                           int32_t* __restrict__ ord) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nruns) return;
    key[i] = runs[i].start;
    ord[i] = (int32_t)i;
}


// EO (TP_LEARNED_ENERGY): every per-target sum takes the plain monopole (the
// gradient is that of plain Barnes-Hut) and the network's correction of the
// two energy channels, sum of wts ((f0-1) al^q + (f1-1) be^q), is added to
// *de, which the energy reduction adds to the sum of the per-target energies.
template <int Q, bool EO>
__global__ void __launch_bounds__(FAR_WARPS * 32) k_far(BHArgs A, const float* __restrict__ kf, int64_t w0,
                                                         int64_t w1, const int64_t* __restrict__ skey,
                                                         const int32_t* __restrict__ sord, double* __restrict__ de) {
    __shared__ __align__(16) float s_rec[FAR_WARPS][32 * TP_SRCW];  // duplicated records of a batch
    __shared__ __align__(16) float s_fk[FAR_WARPS][32 * 8];         // channel factors of a batch
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* rec = s_rec[warp];
    float* fk = s_fk[warp];
    const unsigned long long nr = A.far_count[1];
    const int64_t nruns = nr < (unsigned long long)A.run_cap ? (int64_t)nr : A.run_cap;
    int64_t rlo, rhi;
    window_runs(skey, nruns, w0, w1, rlo, rhi);
    unsigned long long n_learn = 0;  // (target, row) pairs with the range flag set, counted by lane 0
    while (true) {
        int64_t run = 0;
        if (lane == 0) run = rlo + (int64_t)atomicAdd(&A.far_count[2], 1ull);
        run = __shfl_sync(0xffffffffu, run, 0);
        if (run >= rhi) break;
        const tp_far_run R = A.far_runs[sord[run]];
        if (R.len <= 0 || R.len > BH_FAR || R.li < 0 || (int64_t)R.li >= A.nleaves || R.start < 0 ||
            R.start + R.len > A.far_cap)
            continue;  // a run whose rows overflowed the list (the evaluation is repeated)
        // the run's rows inside this window of rows [w0, w1); kf holds the window's rows
        const int64_t r0 = R.start > w0 ? R.start : w0;
        const int64_t r1 = R.start + R.len < w1 ? R.start + R.len : w1;
        if (r0 >= r1) continue;
        const int rlen = (int)(r1 - r0);
        const int64_t L = A.leaves[R.li];
        const int64_t fL = A.first[L];
        const int cnt = A.last[L] - A.first[L] + 1;
#if TP_DEBUG
        {
            // the leaf's targets within the triangles and the run's listed nodes within the tree
            bool ok = fL >= 0 && cnt >= 1 && cnt <= 32 && fL + cnt <= A.ntp;
            for (int i = lane; i < rlen; i += 32) {
                const int nd = A.far_list[r0 + i];
                ok = ok && nd >= 0 && nd < 2 * A.n - 1;
            }
            if (!__all_sync(0xffffffffu, tp_dbg_ok(ok, A.derr))) continue;
        }
#endif
        const int npair = (cnt + 1) >> 1;
        const int ng = 32 / npair;
        const int tpl = lane % npair, g = lane / npair;
        Tgt2 tg;
        bool act[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 2 * tpl + h;
            act[h] = t < cnt && g < ng;
            const int64_t k = fL + (act[h] ? t : 0);
            float v[10];
#pragma unroll
            for (int c = 0; c < 10; ++c) v[c] = act[h] ? A.soa[c * A.ntp + k] : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                (h ? tg.h[c].y : tg.h[c].x) = v[c];
                (h ? tg.l[c].y : tg.l[c].x) = v[3 + c];
                (h ? tg.n[c].y : tg.n[c].x) = v[6 + c];
            }
            (h ? tg.w.y : tg.w.x) = v[9];
        }
        float2 a2[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a2[c] = bh_f2(0.f);
        KSum2 ek = {bh_f2(0.f), bh_f2(0.f)};   // the energy channel, folded after every batch
        KSum2 kde = {bh_f2(0.f), bh_f2(0.f)};  // EO: the energy correction, likewise
        // this lane's row of a batch, loaded one batch ahead
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0, k0 = q0, k1 = q0;
        auto load_row = [&](int b0, int nb) {
            if (lane < nb) {
                const int64_t row = r0 + b0 + lane;
                const float4* r = reinterpret_cast<const float4*>(A.nodef + 16 * (int64_t)A.far_list[row]);
                q0 = r[0];
                q1 = r[1];
                q2 = r[2];
                const float4* kr = reinterpret_cast<const float4*>(kf + (row - w0) * 8);
                k0 = kr[0];
                k1 = kr[1];
            }
        };
        int nb = rlen < 32 ? rlen : 32;
        load_row(0, nb);
        for (int b0 = 0; b0 < rlen; b0 += 32) {
            __syncwarp();  // the previous batch has been evaluated
            if (lane < nb) {
                float4* d = reinterpret_cast<float4*>(rec + lane * TP_SRCW);
                d[0] = make_float4(q0.x, q0.x, q0.y, q0.y);  // x_hi
                d[1] = make_float4(q0.z, q0.z, q0.w, q0.w);  // x_hi[2], x_lo[0]
                d[2] = make_float4(q1.x, q1.x, q1.y, q1.y);  // x_lo[1..2]
                d[3] = make_float4(q1.z, q1.z, q1.w, q1.w);  // nubar[0..1]
                d[4] = make_float4(q2.x, q2.x, q2.y, q2.y);  // nubar[2], area
                // factors exp(y_c) = 1 + (exp(y_c) - 1); the network wrote exp(y_c) - 1
                float4* f = reinterpret_cast<float4*>(fk + lane * 8);
                if (EO) {
                    f[0] = make_float4(k0.x, k0.y, 1.f, 1.f);  // f0 - 1, f1 - 1
                    f[1] = make_float4(1.f, 1.f, 1.f, k1.w);
                } else {
                    f[0] = make_float4(1.f + k0.x, 1.f + k0.y, 1.f + k0.z, 1.f + k0.w);
                    f[1] = make_float4(1.f + k1.x, 1.f + k1.y, 1.f + k1.z, k1.w);
                }
            }
            const unsigned fb = __ballot_sync(0xffffffffu, lane < nb && k1.w != 0.f);
            if (lane == 0) n_learn += (unsigned long long)__popc(fb) * (unsigned long long)cnt;
            __syncwarp();
            const int n = nb;
            if (b0 + 32 < rlen) {
                nb = rlen - (b0 + 32) < 32 ? rlen - (b0 + 32) : 32;
                load_row(b0 + 32, nb);
            }
            float2 dacc = bh_f2(0.f);
            if (g < ng) {
                for (int j = g; j < n; j += ng) far_pair2_learned<Q, EO>(tg, rec + j * TP_SRCW, fk + j * 8, a2, dacc);
            }
            ksum2_add(ek, a2[0]);
            a2[0] = bh_f2(0.f);
            if (EO) ksum2_add(kde, dacc);
        }
        // sum the streams through shared memory and add to the targets
        __syncwarp();
        float* red = rec;                                // [32 lanes][16]
        double* ered = reinterpret_cast<double*>(fk);    // [32 lanes][2]
#pragma unroll
        for (int c = 1; c < 8; ++c) {
            red[lane * 16 + 2 * c] = a2[c].x;
            red[lane * 16 + 2 * c + 1] = a2[c].y;
        }
        double e64[2] = {(double)ek.s.x - (double)ek.c.x, (double)ek.s.y - (double)ek.c.y};
        ered[2 * lane] = e64[0];
        ered[2 * lane + 1] = e64[1];
        __syncwarp();
        if (lane < npair) {
            for (int gg = 1; gg < ng; ++gg) {
                const int o = gg * npair + lane;
#pragma unroll
                for (int c = 1; c < 8; ++c) {
                    a2[c].x += red[o * 16 + 2 * c];
                    a2[c].y += red[o * 16 + 2 * c + 1];
                }
                e64[0] += ered[2 * o];
                e64[1] += ered[2 * o + 1];
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!act[h]) continue;
                const int64_t k = fL + 2 * tpl + h;
                atomicAdd(&A.acc[k], e64[h]);
#pragma unroll
                for (int c = 1; c < 8; ++c) atomicAdd(&A.acc[c * A.ntp + k], (double)(h ? a2[c].y : a2[c].x));
            }
        }
        if (EO) {
            double de_lane = ((double)kde.s.x - (double)kde.c.x) + ((double)kde.s.y - (double)kde.c.y);
            for (int o = 16; o > 0; o >>= 1) de_lane += __shfl_xor_sync(0xffffffffu, de_lane, o);
            if (lane == 0 && de_lane != 0.0) atomicAdd(de, de_lane);
        }
        __syncwarp();  // the staging buffers are reused by the next run
    }
    if (lane == 0 && n_learn) atomicAdd(&A.counts[3], n_learn);
}

// ------------------------------------------------------------ learned correction
// The network scales each channel of the far term of a listed (leaf L,
// cluster C) pair by a factor.  One pass over the listed pairs comes before
// k_far applies the factors: k_mlp_tc<true> (tp_tc.cu) builds each row's 24
// normalised features from the feature records of L and C as a BF16 row in
// shared memory (column 31 = 1 when the raw features lie in the training
// ranges, else 0) and runs the network on 128-row tiles on the
// 5th-generation tensor cores (tcgen05.mma, operands in shared memory, FP32
// accumulators in tensor memory): exp(y_c) - 1 per channel (0 outside the
// ranges).
BHArgs make_bh_args(tp_ctx* ctx, double theta, int edge_only) {
    tp_tree& t = ctx->tree;
    BHArgs A;
    memset(&A, 0, sizeof(A));
    A.soa = ctx->soa;
    A.ntp = ctx->ntp;
    A.Fs = ctx->Fs;
    A.left = t.left;
    A.right = t.right;
    A.first = t.first;
    A.last = t.last;
    A.leaves = t.leaves;
    A.nleaves = t.nleaves;
    A.n = ctx->nt;
    A.mom = t.mom;
    A.box = t.box;
    A.nodef = t.nodef;
    A.adm64 = t.adm64;
    A.adm32 = t.adm32;
    A.bounds = ctx->bounds;
    A.nodeft = t.nodeft;
    A.theta = theta;
    A.leaf_size = t.leaf_size;
    A.edge_only = edge_only;
    A.acc = ctx->acc;
    A.derr = ctx->derr;
    return A;
}

}  // namespace

tp_status tp_launch_bh(tp_ctx* ctx, const tp_params* prm, bool learned) {
    TpRange nvtx_range("tp_launch_bh");
    TP_TRY(tp_ensure_sorted(ctx));
    tp_tree& t = ctx->tree;
    if (t.leaf_size > 32) return tp_set_err(ctx, TP_E_ARG, "leaf_size above 32");
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ctx->scalar + 2);
    unsigned long long* far_rows = reinterpret_cast<unsigned long long*>(ctx->scalar + 7);
    BHArgs A = make_bh_args(ctx, prm->theta, (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0);
    A.counts = counts;
    A.far_rows = far_rows;
    const unsigned blocks = (unsigned)((t.nleaves + BH_WARPS - 1) / BH_WARPS);
    // pair lists, first sized for about 256 near clusters and 1024 far nodes per
    // leaf, then to the counted need
    if (!ctx->near_count) TP_TRY(tp_alloc_t(ctx, &ctx->near_count, 3));
    if (!ctx->far_count) TP_TRY(tp_alloc_t(ctx, &ctx->far_count, 3));
    auto alloc_near = [&](int64_t ents, int64_t runs) -> tp_status {
        TP_TRY(tp_alloc_t(ctx, &ctx->near_list, ents));
        TP_TRY(tp_alloc_t(ctx, &ctx->near_runs, runs));
        ctx->near_cap = ents;
        ctx->nrun_cap = runs;
        return TP_OK;
    };
    auto alloc_far = [&](int64_t rows, int64_t runs) -> tp_status {
        rows = (rows + 31) / 32 * 32;  // whole 32-row network batches
        TP_TRY(tp_alloc_t(ctx, &ctx->far_list, rows));
        TP_TRY(tp_alloc_t(ctx, &ctx->far_leaf, rows));
        TP_TRY(tp_alloc_t(ctx, &ctx->far_runs, runs));
        for (void* p : {(void*)ctx->run_key, (void*)ctx->run_key_s, (void*)ctx->run_ord, (void*)ctx->run_ord_s})
            tp_free(ctx, p);
        ctx->run_key = ctx->run_key_s = nullptr;
        ctx->run_ord = ctx->run_ord_s = nullptr;
        TP_TRY(tp_alloc_t(ctx, &ctx->run_key, runs));
        TP_TRY(tp_alloc_t(ctx, &ctx->run_key_s, runs));
        TP_TRY(tp_alloc_t(ctx, &ctx->run_ord, runs));
        TP_TRY(tp_alloc_t(ctx, &ctx->run_ord_s, runs));
        ctx->far_cap = rows;
        ctx->run_cap = runs;
        return TP_OK;
    };
    if (!ctx->near_list) {
        const int64_t ents = std::max<int64_t>(1 << 20, t.nleaves * 256);
        TP_TRY(alloc_near(ents, ents / 32 + t.nleaves + 1024));
    }
    if (!ctx->far_list) {
        const int64_t rows = std::max<int64_t>(1 << 20, t.nleaves * 1024);
        TP_TRY(alloc_far(rows, rows / 32 + t.nleaves + 1024));
    }
    const bool nblk = near_block_form(t.leaf_size);
    const unsigned nblocks = (unsigned)std::max(1, ctx->num_sms * (nblk ? TP_NB_BPS : TP_NR_BPS));
    const unsigned fblocks = (unsigned)std::max(1, ctx->num_sms * 4);
    // ordered pairs listed for k_near ([0]) and those of them with hi-only differences ([1])
    unsigned long long* near_listed = reinterpret_cast<unsigned long long*>(ctx->scalar + 10);
    A.near_listed = near_listed;
    int64_t listed_rows = 0, listed_runs = 0;
    unsigned long long h[4] = {0, 0, 0, 0}, h_rows = 0, h_lst[2] = {0, 0};
    for (int attempt = 0;; ++attempt) {
        TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
        TP_CU(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), ctx->stream));
        TP_CU(cudaMemsetAsync(far_rows, 0, sizeof(unsigned long long), ctx->stream));
        TP_CU(cudaMemsetAsync(near_listed, 0, 2 * sizeof(unsigned long long), ctx->stream));
        TP_CU(cudaMemsetAsync(ctx->near_count, 0, 3 * sizeof(unsigned long long), ctx->stream));
        TP_CU(cudaMemsetAsync(ctx->far_count, 0, 3 * sizeof(unsigned long long), ctx->stream));
        A.src = ctx->src;
        A.near_list = ctx->near_list;
        A.near_runs = ctx->near_runs;
        A.near_count = ctx->near_count;
        A.near_cap = ctx->near_cap;
        A.nrun_cap = ctx->nrun_cap;
        A.far_list = ctx->far_list;
        A.far_leaf = ctx->far_leaf;
        A.far_runs = ctx->far_runs;
        A.far_count = ctx->far_count;
        A.far_cap = ctx->far_cap;
        A.run_cap = ctx->run_cap;
        // the traversal (far nodes evaluated or listed, touching near clusters
        // evaluated, the other near clusters listed), then the listed near clusters
        // (the near-field kernel is the timed one: ev[0] .. ev[1])
        if (prm->q == 6) {
            if (learned) k_bh<6, M_LIST><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
            else k_bh<6, M_BH><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
            cudaEventRecord(ctx->ev[0], ctx->stream);
            if (nblk) k_near_blk<6><<<nblocks, NB_THREADS, 0, ctx->stream>>>(A);
            else k_near<6><<<nblocks, NR_WARPS * 32, 0, ctx->stream>>>(A);
        } else {
            if (learned) k_bh<8, M_LIST><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
            else k_bh<8, M_BH><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
            cudaEventRecord(ctx->ev[0], ctx->stream);
            if (nblk) k_near_blk<8><<<nblocks, NB_THREADS, 0, ctx->stream>>>(A);
            else k_near<8><<<nblocks, NR_WARPS * 32, 0, ctx->stream>>>(A);
        }
        cudaEventRecord(ctx->ev[1], ctx->stream);
        ctx->nlaunch += 2;
        TP_CU(cudaGetLastError());
        unsigned long long nc[2] = {0, 0}, fc[2] = {0, 0};
        TP_CU(cudaMemcpyAsync(nc, ctx->near_count, sizeof(nc), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaMemcpyAsync(fc, ctx->far_count, sizeof(fc), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaMemcpyAsync(&h_rows, far_rows, sizeof(h_rows), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaMemcpyAsync(h_lst, near_listed, sizeof(h_lst), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaStreamSynchronize(ctx->stream));
        const bool near_ok = (int64_t)nc[0] <= ctx->near_cap && (int64_t)nc[1] <= ctx->nrun_cap;
        const bool far_ok = (int64_t)fc[0] <= ctx->far_cap && (int64_t)fc[1] <= ctx->run_cap;
        if (near_ok && far_ok) {
            listed_rows = (int64_t)fc[0];
            listed_runs = (int64_t)fc[1];
            break;
        }
        if (attempt > 0) return tp_set_err(ctx, TP_E_OOM, "Barnes-Hut pair list overflow");
        // enlarge the lists that overflowed to the counted need (with slack) and repeat
        if (!near_ok) {
            tp_free(ctx, ctx->near_list);
            tp_free(ctx, ctx->near_runs);
            ctx->near_list = nullptr;
            ctx->near_runs = nullptr;
            TP_TRY(alloc_near((int64_t)(nc[0] + nc[0] / 4 + 1024), (int64_t)(nc[1] + nc[1] / 4 + 1024)));
        }
        if (!far_ok) {
            tp_free(ctx, ctx->far_list);
            tp_free(ctx, ctx->far_leaf);
            tp_free(ctx, ctx->far_runs);
            ctx->far_list = nullptr;
            ctx->far_leaf = nullptr;
            ctx->far_runs = nullptr;
            TP_TRY(alloc_far((int64_t)(fc[0] + fc[0] / 4 + 1024), (int64_t)(fc[1] + fc[1] / 4 + 1024)));
        }
    }
    if (learned) {
        TP_TRY(tp_ensure_node_features(ctx));
        TP_CU(cudaMemsetAsync(ctx->scalar + 6, 0, sizeof(double), ctx->stream));
        // factors of the listed (leaf, cluster) pairs, for one window of at most
        // ctx->learned_window rows at a time
        const int64_t win = std::min<int64_t>(std::max<int64_t>(listed_rows, 32), ctx->learned_window);
        const int64_t xcap = win + BH_FAR;  // a window ends on a run start, at most BH_FAR - 1 rows late
        if (ctx->far_xcap < xcap) {
            tp_free(ctx, ctx->far_kf);
            ctx->far_kf = nullptr;
            ctx->far_xcap = 0;
            TP_TRY(tp_alloc_t(ctx, &ctx->far_kf, xcap * 8));
            ctx->far_xcap = xcap;
        }
        A.wb = static_cast<const __nv_bfloat16*>(tp_mlp_weights(ctx));
        A.mbias = tp_mlp_bias(ctx);
        A.mnorm = tp_mlp_norm(ctx);
        // the runs in first-row order, so that a window visits only its own runs
        if (listed_runs > 0) {
            k_run_keys<<<(unsigned)((listed_runs + 255) / 256), 256, 0, ctx->stream>>>(
                ctx->far_runs, listed_runs, ctx->run_key, ctx->run_ord);
            ++ctx->nlaunch;
            int end_bit = 1;
            while (end_bit < 63 && ((int64_t)1 << end_bit) <= listed_rows) ++end_bit;
            TP_TRY(tp_sort_pairs_u64(ctx, reinterpret_cast<const uint64_t*>(ctx->run_key), ctx->run_ord,
                                     reinterpret_cast<uint64_t*>(ctx->run_key_s), ctx->run_ord_s, listed_runs,
                                     end_bit));
        }
        // window boundaries on run starts (read back once when there are several windows)
        const int64_t nwin = (listed_rows + win - 1) / win;
        std::vector<int64_t> bnd = {0, listed_rows};
        if (nwin > 1) {
            if (ctx->win_bnd_cap < nwin + 1) {
                tp_free(ctx, ctx->win_bnd);
                ctx->win_bnd = nullptr;
                ctx->win_bnd_cap = 0;
                TP_TRY(tp_alloc_t(ctx, &ctx->win_bnd, nwin + 1));
                ctx->win_bnd_cap = nwin + 1;
            }
            k_window_bounds<<<(unsigned)((nwin + 256) / 256), 256, 0, ctx->stream>>>(
                ctx->run_key_s, listed_runs, win, nwin, listed_rows, ctx->win_bnd);
            ++ctx->nlaunch;
            bnd.resize(nwin + 1);
            TP_CU(cudaMemcpyAsync(bnd.data(), ctx->win_bnd, sizeof(int64_t) * (nwin + 1), cudaMemcpyDeviceToHost,
                                  ctx->stream));
            TP_CU(cudaStreamSynchronize(ctx->stream));
        }
        // per window: the network's factors of the listed far terms, then the far terms with them
        tp_feat_src fs;
        fs.nodeft = t.nodeft;
        fs.far_list = ctx->far_list;
        fs.far_leaf = ctx->far_leaf;
        fs.leaves = t.leaves;
        fs.mnorm = A.mnorm;
        fs.nleaves = t.nleaves;
        fs.nnodes = 2 * ctx->nt - 1;
        for (size_t wi = 0; wi + 1 < bnd.size(); ++wi) {
            const int64_t w0 = bnd[wi], w1 = bnd[wi + 1];
            if (w1 <= w0) continue;
            if (w1 - w0 > ctx->far_xcap)  // cannot happen while runs hold at most BH_FAR rows
                return tp_set_err(ctx, TP_E_STATE, "internal: learned window of %lld rows above %lld",
                                  (long long)(w1 - w0), (long long)ctx->far_xcap);
            TP_TRY(tp_launch_mlp_tc_feat(ctx, A.wb, A.mbias, fs, w0, w1, ctx->far_kf));
            TP_CU(cudaMemsetAsync(ctx->far_count + 2, 0, sizeof(unsigned long long), ctx->stream));
            double* de = ctx->scalar + 6;  // energy correction of TP_LEARNED_ENERGY (zeroed per evaluation)
            if (prm->flags & TP_LEARNED_ENERGY) {
                if (prm->q == 6)
                    k_far<6, true><<<fblocks, FAR_WARPS * 32, 0, ctx->stream>>>(A, ctx->far_kf, w0, w1,
                                                                              ctx->run_key_s, ctx->run_ord_s, de);
                else
                    k_far<8, true><<<fblocks, FAR_WARPS * 32, 0, ctx->stream>>>(A, ctx->far_kf, w0, w1,
                                                                              ctx->run_key_s, ctx->run_ord_s, de);
            } else {
                if (prm->q == 6)
                    k_far<6, false><<<fblocks, FAR_WARPS * 32, 0, ctx->stream>>>(A, ctx->far_kf, w0, w1,
                                                                               ctx->run_key_s, ctx->run_ord_s, de);
                else
                    k_far<8, false><<<fblocks, FAR_WARPS * 32, 0, ctx->stream>>>(A, ctx->far_kf, w0, w1,
                                                                               ctx->run_key_s, ctx->run_ord_s, de);
            }
            ++ctx->nlaunch;
        }
        TP_CU(cudaGetLastError());
        TP_CU(cudaMemcpyAsync(h + 3, counts + 3, sizeof(h[3]), cudaMemcpyDeviceToHost, ctx->stream));
    }
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.pairs_exact = (int64_t)h[0];
    ctx->stats.kernel_pairs = (int64_t)h_lst[0];  // ordered pairs of the timed near-field launch
    ctx->stats.far_terms = (int64_t)h[1];
    ctx->stats.far_pairs = (int64_t)h[2];
    ctx->stats.learned_terms = (int64_t)h[3];
    ctx->stats.far_rows = (int64_t)h_rows;
    return TP_OK;
}

// The Barnes-Hut near-field kernel on given runs of (first member, count)
// entries whose clusters have vertex boxes apart from their run's leaf (so no
// exclusion test is needed): adds to ctx->acc with FP64 atomics.  counters[1]
// holds the number of runs, counters[2] is the work counter (zeroed here).
tp_status tp_launch_near_runs(tp_ctx* ctx, int q, const int2* list, int64_t list_len, const tp_far_run* runs,
                              int64_t run_cap, unsigned long long* counters) {
    BHArgs A = make_bh_args(ctx, 0.0, 0);
    A.src = ctx->src;
    A.near_list = const_cast<int2*>(list);
    A.near_runs = const_cast<tp_far_run*>(runs);
    A.near_count = counters;
    A.near_cap = list_len;
    A.nrun_cap = run_cap;
    TP_CU(cudaMemsetAsync(counters + 2, 0, sizeof(unsigned long long), ctx->stream));
    const bool nblk = near_block_form(ctx->tree.leaf_size);
    const unsigned nblocks = (unsigned)std::max(1, ctx->num_sms * (nblk ? TP_NB_BPS : TP_NR_BPS));
    if (nblk) {
        if (q == 6) k_near_blk<6><<<nblocks, NB_THREADS, 0, ctx->stream>>>(A);
        else k_near_blk<8><<<nblocks, NB_THREADS, 0, ctx->stream>>>(A);
    } else {
        if (q == 6) k_near<6><<<nblocks, NR_WARPS * 32, 0, ctx->stream>>>(A);
        else k_near<8><<<nblocks, NR_WARPS * 32, 0, ctx->stream>>>(A);
    }
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_bh_sample(tp_ctx* ctx, double theta, uint32_t keep_u, uint64_t seed, int2* out, int64_t cap,
                              int32_t* counter) {
    TpRange nvtx_range("tp_launch_bh_sample");
    TP_TRY(tp_ensure_sorted(ctx));
    tp_tree& t = ctx->tree;
    BHArgs A = make_bh_args(ctx, theta, 0);
    A.keep_u = keep_u;
    A.seed = seed;
    A.rec_out = out;
    A.rec_cap = cap;
    A.rec_count = counter;
    const unsigned blocks = (unsigned)((t.nleaves + BH_WARPS - 1) / BH_WARPS);
    k_bh<6, M_RECORD><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}
