// tp_pair_dev.cuh - packed FP32x2 pair arithmetic shared by the clustered
// forms (the Barnes-Hut kernels of tp_bh.cu and the cluster-cluster kernels
// of tp_dual.cu): one lane evaluates one target (duplicated in both halves)
// against two staged sources at a time, or two targets against one source,
// and accumulates the target-side derivatives of e_TS + e_ST in the direct
// kernels' convention (Ew, U, Gn[3], Gx[3], all carrying the factor p/q).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ float bh_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 arithmetic: one lane evaluates one target against two sources
// at a time (the target's data duplicated in both halves).
__device__ __forceinline__ float2 bh_f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 bh_neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 bh_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bh_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 bh_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Compensated FP32 running sums (Kahan), one per half: the value is s - c.
// The clustered kernels fold their per-batch FP32 partials into these
// instead of into FP64 sums: FP64 arithmetic runs at a small fraction of the
// FP32 rate on this part, and its pipe stalled the warps that issued the
// folds.  (t - s) - y is formed with FMAs by -1, which no compiler
// contraction can change.
struct KSum2 {
    float2 s, c;
};

__device__ __forceinline__ void ksum2_add(KSum2& k, float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 y = __ffma2_rn(k.c, m1, x);
    const float2 t = __fadd2_rn(k.s, y);
    k.c = __ffma2_rn(y, m1, __ffma2_rn(k.s, m1, t));
    k.s = t;
}

// The same for one scalar sum.
__device__ __forceinline__ void ksum_add(float& s, float& c, float x) {
    const float y = __fmaf_rn(c, -1.f, x);
    const float t = __fadd_rn(s, y);
    c = __fmaf_rn(y, -1.f, __fmaf_rn(s, -1.f, t));
    s = t;
}

struct Tgt2 {
    float2 h[3], l[3], n[3], w;
};

// Staged sources (near members or far-node records) are kept in pairs: the
// ten values (x_hi[3], x_lo[3], nu[3], w~) of sources 2i and 2i+1 interleaved,
// so that one 16-byte shared load gives two values of both sources.
constexpr int BH_PAIR = 20;  // floats per staged source pair

__device__ __forceinline__ void stage_put(float* stg, int j, const float v[10]) {
    float* d = stg + (j >> 1) * BH_PAIR + (j & 1);
#pragma unroll
    for (int c = 0; c < 10; ++c) d[2 * c] = v[c];
}

// A padding source: zero weight, far from every target, so that its terms
// vanish without a test (no zero distance, no overflow).
__device__ __forceinline__ void stage_pad(float* stg, int j) {
    const float v[10] = {1e18f, 1e18f, 1e18f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    stage_put(stg, j, v);
}

// T-side derivatives of e_TS + e_ST for two (target, source) pairs at once,
// one per half of the float2 operands (targets th..tw, sources sh..sw),
// accumulated in the direct kernels' convention.  SEL: per-half admission
// (v0, v1); an excluded half gets 1/|d|^2 = 0 and weight 0, so its terms are
// exact zeros (d itself stays finite: a coincident centroid or a padding
// source's large offset never reaches a power).  HILO: d = (hi_T - hi_S) +
// (lo_T - lo_S); without it d = hi_T - hi_S (pairs far enough apart).  TW1:
// the target weights are left out (every accumulated term carries its
// target's weight as a factor, which the caller applies to the sums).
template <int Q, bool SEL, bool HILO = true, bool TW1 = false>
__device__ __forceinline__ void pair_core(const float2 (&th)[3], const float2 (&tl)[3], const float2 (&tn)[3],
                                          float2 tw, const float2 (&sh)[3], const float2 (&sl)[3],
                                          const float2 (&sn)[3], float2 sw, float2 acc[8], bool v0, bool v1) {
    float2 d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        d[k] = HILO ? bh_add2(bh_add2(th[k], bh_neg2(sh[k])), bh_add2(tl[k], bh_neg2(sl[k])))
                    : bh_add2(th[k], bh_neg2(sh[k]));
    float2 r2 = bh_mul2(d[0], d[0]);
    r2 = bh_fma2(d[1], d[1], r2);
    r2 = bh_fma2(d[2], d[2], r2);
    float2 wts = TW1 ? sw : bh_mul2(tw, sw);
    float2 inv = make_float2(bh_rcp(r2.x), bh_rcp(r2.y));
    if (SEL) {
        inv = make_float2(v0 ? inv.x : 0.f, v1 ? inv.y : 0.f);
        wts = make_float2(v0 ? wts.x : 0.f, v1 ? wts.y : 0.f);
    }
    float2 a = bh_mul2(tn[0], d[0]);
    a = bh_fma2(tn[1], d[1], a);
    a = bh_fma2(tn[2], d[2], a);
    float2 b = bh_mul2(sn[0], d[0]);
    b = bh_fma2(sn[1], d[1], b);
    b = bh_fma2(sn[2], d[2], b);
    const float2 al = bh_mul2(a, inv), be = bh_mul2(b, inv);
    const float2 al2 = bh_mul2(al, al), be2 = bh_mul2(be, be);
    const float2 al4 = bh_mul2(al2, al2), be4 = bh_mul2(be2, be2);
    float2 al5, be5;
    if (Q == 6) {
        al5 = bh_mul2(al4, al);
        be5 = bh_mul2(be4, be);
    } else {
        al5 = bh_mul2(bh_mul2(al4, al2), al);
        be5 = bh_mul2(bh_mul2(be4, be2), be);
    }
    const float2 wi = bh_mul2(wts, inv);
    const float2 A5 = bh_mul2(wi, al5), B5 = bh_mul2(wi, be5);
#if TP_PAIR_T
    // wi s6 = A5 al + B5 be, and the pair energy wts s6 = (wi s6) |d|^2
    const float2 ws6 = bh_fma2(A5, al, bh_mul2(B5, be));
    const float2 nk = bh_mul2(ws6, bh_f2(-2.0f));  // -(p/q) wts inv s6, p = 2q
    acc[0] = bh_fma2(ws6, r2, acc[0]);
#else
    const float2 s6 = Q == 6 ? bh_fma2(be4, be2, bh_mul2(al4, al2)) : bh_fma2(be4, be4, bh_mul2(al4, al4));
    const float2 nk = bh_mul2(bh_mul2(wi, s6), bh_f2(-2.0f));  // -(p/q) wts inv s6, p = 2q
    acc[0] = bh_fma2(wts, s6, acc[0]);
#endif
    acc[1] = bh_add2(acc[1], A5);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[2 + k] = bh_fma2(A5, d[k], acc[2 + k]);
        acc[5 + k] = bh_fma2(nk, d[k], bh_fma2(B5, sn[k], acc[5 + k]));
    }
}

// One target (duplicated in both halves of t) against the staged source pair
// p (data at stg + p * BH_PAIR); HILO and TW1 as in pair_core.
template <int Q, bool SEL, bool HILO = true, bool TW1 = false>
__device__ __forceinline__ void gather_pair2(const Tgt2& t, const float* stg, int p, float2 acc[8], bool v0 = true,
                                             bool v1 = true) {
    const float4* r = reinterpret_cast<const float4*>(stg + p * BH_PAIR);
    const float4 q0 = r[0], q1 = r[1], q2 = r[2], q3 = r[3], q4 = r[4];
    const float2 sh[3] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y)};
    const float2 sl[3] = {make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
    const float2 sn[3] = {make_float2(q3.x, q3.y), make_float2(q3.z, q3.w), make_float2(q4.x, q4.y)};
    pair_core<Q, SEL, HILO, TW1>(t.h, t.l, t.n, t.w, sh, sl, sn, make_float2(q4.z, q4.w), acc, v0, v1);
}

__device__ __forceinline__ bool adjacent(int3 a, int3 b, int edge_only) {
    int k = (a.x == b.x) + (a.x == b.y) + (a.x == b.z) + (a.y == b.x) + (a.y == b.y) + (a.y == b.z) + (a.z == b.x) +
            (a.z == b.y) + (a.z == b.z);
    return edge_only ? k >= 2 : k >= 1;
}

}  // namespace
