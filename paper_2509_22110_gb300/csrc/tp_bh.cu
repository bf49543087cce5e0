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
// GPU organisation.  One warp per target cluster leaf (at most 32 targets
// per leaf, 16 by default).  The admissibility test depends on (L, C)
// only, so the traversal is warp-uniform: the warp pops up to 32 nodes from
// a shared-memory stack, each lane tests one, and ballots sort them into a
// far list, a near list and nodes to open.  The lists are evaluated with
// lanes split as (target = lane % 16, half = lane / 16), each half taking
// every other far node or near member.  Per-target partials are FP32 per
// list flush and FP64 across flushes; each target is owned by one warp, so
// results are stored without atomics in the same accumulator layout as the
// direct kernels (see tp_direct.cu), and the same adjoint applies.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"

namespace {

constexpr int BH_WARPS = 4;
constexpr int BH_STACK = 1024;
constexpr int BH_FAR = 256;
constexpr int BH_NEAR = 128;

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
    double theta;
    int leaf_size;
    int edge_only;
    double* acc;
    unsigned* derr;
    unsigned long long* counts;  // [0] near pairs, [1] far terms, [2] far pairs
};

__device__ __forceinline__ float bh_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Tgt {
    float h[3], l[3], n[3], w;
};

// T-side derivatives of e_TS + e_ST for one source (or cluster) with data
// (sh, sl, sn, sw), accumulated in the direct kernels' convention.
template <int Q>
__device__ __forceinline__ void gather_pair(const Tgt& t, const float* sh, const float* sl, const float* sn, float sw,
                                            float acc[8]) {
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = (t.h[k] - sh[k]) + (t.l[k] - sl[k]);
    float inv = bh_rcp(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float a = t.n[0] * d[0] + t.n[1] * d[1] + t.n[2] * d[2];
    float b = sn[0] * d[0] + sn[1] * d[1] + sn[2] * d[2];
    float al = a * inv, be = b * inv;
    float al2 = al * al, be2 = be * be, al4 = al2 * al2, be4 = be2 * be2;
    float alq, beq, al5, be5;
    if (Q == 6) {
        alq = al4 * al2;
        beq = be4 * be2;
        al5 = al4 * al;
        be5 = be4 * be;
    } else {
        alq = al4 * al4;
        beq = be4 * be4;
        al5 = al4 * al2 * al;
        be5 = be4 * be2 * be;
    }
    float wts = t.w * sw;
    float s6 = alq + beq;
    float wi = wts * inv;
    float A5 = wi * al5, B5 = wi * be5, k = 2.0f * wi * s6;  // (p/q) = 2
    acc[0] += wts * s6;
    acc[1] += A5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[2 + c] += A5 * d[c];
        acc[5 + c] += B5 * sn[c] - k * d[c];
    }
}

// Target-leaf constants of the admissibility test.
struct LeafAdm {
    double bl[6];      // FP64 vertex box
    double cl[3];      // box centre (bl_min + bl_max) * 0.5
    double dl;         // box diagonal
    float out[6], in[6], cl32[3], dl32;
};

__device__ __forceinline__ void leaf_adm(const double* box, LeafAdm& L) {
    double dl2 = 0.0;
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
        else if (!(L.in[3 + a] >= c32[6 + a] && c32[9 + a] >= L.in[a])) amb = true;
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
        const float t = c32[12 + a] - L.cl32[a];
        r2f = fmaf(t, t, r2f);
        M += fabsf(c32[12 + a]) + fabsf(L.cl32[a]);
    }
    const float distf = sqrtf(r2f);
    const float rhsf = theta32 * (distf - 0.5f * L.dl32);
    const float lhsf = c32[15];
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

__device__ __forceinline__ bool adjacent(int3 a, int3 b, int edge_only) {
    int k = (a.x == b.x) + (a.x == b.y) + (a.x == b.z) + (a.y == b.x) + (a.y == b.y) + (a.y == b.z) + (a.z == b.x) +
            (a.z == b.y) + (a.z == b.z);
    return edge_only ? k >= 2 : k >= 1;
}

template <int Q>
__global__ void __launch_bounds__(BH_WARPS * 32) k_bh(BHArgs A) {
    __shared__ int32_t s_stack[BH_WARPS][BH_STACK];
    __shared__ int32_t s_far[BH_WARPS][BH_FAR];
    __shared__ int32_t s_near[BH_WARPS][BH_NEAR];
    __shared__ __align__(16) float s_stg[BH_WARPS][32 * 16];
    __shared__ int32_t s_stg_cnt[BH_WARPS][32];
    __shared__ int4 s_stg_f[BH_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t li = (int64_t)blockIdx.x * BH_WARPS + warp;
    if (li >= A.nleaves) return;
    int32_t* st = s_stack[warp];
    int32_t* far = s_far[warp];
    int32_t* nearl = s_near[warp];
    float* stg = s_stg[warp];
    int32_t* stg_cnt = s_stg_cnt[warp];
    int4* stg_f = s_stg_f[warp];
    const int64_t L = A.leaves[li];
    const int64_t fL = A.first[L];
    const int cnt = A.last[L] - A.first[L] + 1;
    LeafAdm la;
    leaf_adm(A.box + 6 * L, la);
    const float theta32 = (float)A.theta;
    const int t = lane & 15, half = lane >> 4;
    const int64_t k = fL + t;
    const bool active = t < cnt;
    Tgt tg;
    int3 tf = make_int3(-2, -2, -2);
    if (active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tg.h[c] = A.soa[c * A.ntp + k];
            tg.l[c] = A.soa[(3 + c) * A.ntp + k];
            tg.n[c] = A.soa[(6 + c) * A.ntp + k];
        }
        tg.w = A.soa[9 * A.ntp + k];
        tf = make_int3(A.Fs[3 * k], A.Fs[3 * k + 1], A.Fs[3 * k + 2]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) tg.h[c] = tg.l[c] = tg.n[c] = 0.f;
        tg.w = 0.f;
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long n_near = 0, n_far = 0, n_farp = 0;
    const unsigned lt = (1u << lane) - 1u;

    // far list: stage 32 node records at a time in shared memory, then every
    // half-warp sweeps them (half h takes records h, h+2, ...)
    auto flush_far = [&](int nf) {
        float a32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int b0 = 0; b0 < nf; b0 += 32) {
            const int nb = nf - b0 < 32 ? nf - b0 : 32;
            __syncwarp();
            if (lane < nb) {
                const int32_t C = far[b0 + lane];
                const float4* r = reinterpret_cast<const float4*>(A.nodef + 16 * (int64_t)C);
                float4* d = reinterpret_cast<float4*>(stg + lane * 16);
                d[0] = r[0];
                d[1] = r[1];
                d[2] = r[2];
                stg_cnt[lane] = A.last[C] - A.first[C] + 1;
            }
            __syncwarp();
            for (int i = half; i < nb; i += 2) {
                const float* r = stg + i * 16;
                if (active) {
                    gather_pair<Q>(tg, r, r + 3, r + 6, r[9], a32);
                    n_far += 1;
                    n_farp += (unsigned long long)stg_cnt[i];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += (double)a32[c];
    };
    // near list: stage the members of up to 32 sources at a time (whole near
    // nodes) in shared memory, then every half-warp sweeps them
    auto flush_near = [&](int nn) {
        float a32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int i = 0;
        while (i < nn) {
            // take whole nodes while they fit in 32 slots
            int nsrc = 0, i1 = i;
            while (i1 < nn) {
                const int m = A.last[nearl[i1]] - A.first[nearl[i1]] + 1;
                if (nsrc + m > 32) break;
                nsrc += m;
                ++i1;
            }
            __syncwarp();
            // lane -> (node, member) by walking the taken nodes
            {
                int base = 0;
                for (int j = i; j < i1; ++j) {
                    const int64_t C = nearl[j];
                    const int64_t f = A.first[C];
                    const int m = A.last[C] - A.first[C] + 1;
                    if (lane >= base && lane < base + m) {
                        const int64_t s = f + (lane - base);
                        float* d = stg + lane * 16;
#pragma unroll
                        for (int c = 0; c < 10; ++c) d[c] = A.soa[c * A.ntp + s];
                        stg_f[lane] = make_int4(A.Fs[3 * s], A.Fs[3 * s + 1], A.Fs[3 * s + 2], (int)s);
                    }
                    base += m;
                }
            }
            __syncwarp();
            for (int j = half; j < nsrc; j += 2) {
                const float* r = stg + j * 16;
                const int4 sf = stg_f[j];
                if (active && sf.w != (int)k && !adjacent(tf, make_int3(sf.x, sf.y, sf.z), A.edge_only)) {
                    gather_pair<Q>(tg, r, r + 3, r + 6, r[9], a32);
                    n_near += 1;
                }
            }
            i = i1;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += (double)a32[c];
    };

    int sp = 1, nf = 0, nn = 0;
    if (lane == 0) st[0] = 0;  // root
    __syncwarp();
    bool overflow = false;
    while (sp > 0) {
        const int m = sp < 32 ? sp : 32;
        const int node = lane < m ? st[sp - 1 - lane] : -1;
        __syncwarp();
        sp -= m;
        bool is_far = false, is_near = false, is_open = false;
        if (node >= 0) {
            const int cntc = A.last[node] - A.first[node] + 1;
            if (admissible(la, A.adm32 + 16 * (int64_t)node, A.box + 6 * (int64_t)node, A.adm64 + 4 * (int64_t)node,
                           A.theta, theta32))
                is_far = true;
            else if (cntc <= A.leaf_size || node >= A.n - 1) is_near = true;
            else is_open = true;
        }
        const unsigned bf = __ballot_sync(0xffffffffu, is_far);
        const unsigned bn = __ballot_sync(0xffffffffu, is_near);
        const unsigned bo = __ballot_sync(0xffffffffu, is_open);
        if (sp + 2 * __popc(bo) > BH_STACK) {
            overflow = true;
            break;
        }
        if (is_far) far[nf + __popc(bf & lt)] = node;
        if (is_near) nearl[nn + __popc(bn & lt)] = node;
        if (is_open) {
            const int pos = sp + 2 * __popc(bo & lt);
            st[pos] = A.right[node];
            st[pos + 1] = A.left[node];
        }
        nf += __popc(bf);
        nn += __popc(bn);
        sp += 2 * __popc(bo);
        __syncwarp();
        if (nf > BH_FAR - 32) {
            flush_far(nf);
            nf = 0;
        }
        if (nn > BH_NEAR - 32) {
            flush_near(nn);
            nn = 0;
        }
        __syncwarp();
    }
    if (overflow) {
        if (lane == 0) tp_dev_error(A.derr, TP_DERR_STACK);
        return;
    }
    flush_far(nf);
    flush_near(nn);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
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
    }
}

}  // namespace

tp_status tp_launch_bh(tp_ctx* ctx, const tp_params* prm, bool learned) {
    if (learned) return tp_set_err(ctx, TP_E_STATE, "TP_LEARNED is not available in this build");
    tp_tree& t = ctx->tree;
    if (t.leaf_size > 32) return tp_set_err(ctx, TP_E_ARG, "leaf_size above 32");
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ctx->scalar + 2);
    TP_CU(cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), ctx->stream));
    BHArgs A;
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
    A.theta = prm->theta;
    A.leaf_size = t.leaf_size;
    A.edge_only = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    A.acc = ctx->acc;
    A.derr = ctx->derr;
    A.counts = counts;
    const unsigned blocks = (unsigned)((t.nleaves + BH_WARPS - 1) / BH_WARPS);
    cudaEventRecord(ctx->ev[0], ctx->stream);
    if (prm->q == 6)
        k_bh<6><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
    else
        k_bh<8><<<blocks, BH_WARPS * 32, 0, ctx->stream>>>(A);
    ++ctx->nlaunch;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    unsigned long long h[3] = {0, 0, 0};
    TP_CU(cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->stats.pairs_exact = (int64_t)h[0];
    ctx->stats.far_terms = (int64_t)h[1];
    ctx->stats.far_pairs = (int64_t)h[2];
    return TP_OK;
}
