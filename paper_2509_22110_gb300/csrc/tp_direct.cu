// tp_direct.cu - direct all-pairs tangent-point energy and its per-triangle
// derivatives (Eq. TP, Sec. 2.2.2; the "full integration" scheme of Sec. 3.2
// with one centroid point per flat triangle).
//
// Symmetric scheme.  Each unordered pair {T,S} of admitted triangles is
// evaluated once; both orderings are formed from the shared geometry
//     d = x_T - x_S,  r2 = |d|^2,  inv = 1/r2,  a = nu_T.d,  b = nu_S.d,
//     al = a*inv, be = b*inv   (so al^6 = a^6/r^12: no overflow of r^-12)
//     s6 = al^6 + be^6,  wts = w~_T w~_S  (w~ = sqrt(p/q) w, p = 2q)
//     E = wts s6 = (p/q)(e_TS + e_ST),  A5 = wts inv al^5,  B5 = wts inv be^5,
//     k = (p/q) wts inv s6
// and added to per-triangle accumulators (all carrying the factor p/q):
//     T: Ew += E, U += A5, Gn += A5 d, Gx += B5 nu_S - k d
//     S: Ew += E, U -= B5, Gn += B5 d, Gx += -A5 nu_T + k d
// from which dPhi/dw = Ew/((p/q) w), dPhi/dnu = q Gn/(p/q),
// dPhi/dx = q (Gx + U nu)/(p/q) (exact chain rule of the discrete sum; the
// two-sided accumulation is the discrete counterpart of the reordered
// variation Eq. (dTP_reordered), Sec. 3.2).  Written for q = 6, p = 12 and
// q = 8, p = 16.
//
// Work decomposition.  Triangles are in Morton order, padded to super-tiles
// of 1536.  A work item is a super-tile pair (I <= J).  A persistent block
// (one per SM) keeps the 1536 targets of I in registers (each lane NP packed
// pairs of consecutive targets, FP32x2 arithmetic) and streams the 1536
// sources of J through shared memory in chunks of 128 with cp.async.bulk
// (TMA bulk copies, completion on an mbarrier, bounded waits).  Per source
// every lane adds its 2 NP pair contributions to packed target
// accumulators; the source contributions of the warp are reduced by a
// butterfly transpose (8 values over 32 lanes in 9 shuffles), software-
// pipelined beside the next source's arithmetic, and written once per warp;
// per chunk the block sums its warps and promotes to FP64 with one global
// atomic add per source and accumulator.  Target partials (FP32 over one
// item) are promoted to FP64 with one global atomic add per target and
// accumulator per item.
//
// Three kinds of items, two launches:
//   FAST    - super-tiles far apart: d = x_hi,T - x_hi,S (FP32 centroids);
//   PRECISE - super-tiles closer than a fraction of the mesh size:
//             d = (hi_T - hi_S) + (lo_T - lo_S), which removes the FP32
//             cancellation of nearby centroids;
//   MASKED  - a pair of triangles sharing a vertex inside (and all diagonal
//             items): the 128 x 128 blocks that hold a vertex-sharing pair
//             (and the diagonal blocks) take a per-pair exclusion test,
//             the other blocks the PRECISE arithmetic.
// FAST and PRECISE items run 8 warps x 3 pairs per lane (a prefetched
// source record in registers); MASKED items 12 warps x 2 pairs per lane
// (face indices in registers for the exclusion test).
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"

namespace {

constexpr int WARPS = 12;  // energy kernel: 12 warps, each lane 2 packed target pairs
constexpr int THREADS = WARPS * 32;
constexpr int NCHUNK = TP_SUPER / TP_CHUNK;                // chunks per super-tile
constexpr int CHUNK_BYTES = TP_CHUNK * TP_SRCW * 4;        // 10 KB
constexpr int SMEM_ENERGY = 2 * CHUNK_BYTES + 64 + WARPS * 8;  // chunks, mbarriers + item slot, warp sums
static_assert(TP_SUPER == WARPS * 128, "a warp owns 128 targets of the super-tile");

enum { K_FAST = 0, K_PRECISE = 1, K_MASKED = 2 };

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct DirectArgs {
    const float* soa;         // 10 planes of ntp: x_hi[3], x_lo[3], nu[3], w~
    const float* src;         // [ntp][TP_SRCW]
    const int32_t* Fs;        // [ntp][3]
    double* acc;              // [TP_NACC][ntp]
    const int32_t* mlist;     // MASKED items (I << 16 | J)
    const int32_t* plist;     // PRECISE items
    const int32_t* flist;     // FAST items
    const unsigned* bmask;    // per super-tile pair: 128 x 128 blocks holding a vertex-sharing pair
    int nsup;                 // super-tiles
    int nm, np, nf;           // their counts; the work queue is mlist, plist, flist in that order
    unsigned* work;           // dynamic work counter (zeroed before the launch)
    int64_t ntp;
    int edge_only;
    unsigned* derr;
    // energy kernel: per-block energy partials; masked gradient kernel: a device
    // array of three pointers to the exclusion bits (xmask [slot][128 targets][4
    // words], xeff per masked item, xbase per masked item).  One field serves
    // both so that the argument block of the other kernels stays as it is.
    double* partial;
};

struct SrcRec {
    float2 h[3], l[3], n[3], w;
};

template <bool LO>
__device__ __forceinline__ void load_src(const float* rec, SrcRec& s) {
    const float4* r = reinterpret_cast<const float4*>(rec);
    float4 a = r[0], b = r[1], d = r[3], e = r[4];
    s.h[0] = make_float2(a.x, a.y);
    s.h[1] = make_float2(a.z, a.w);
    s.h[2] = make_float2(b.x, b.y);
    if (LO) {
        float4 c = r[2];
        s.l[0] = make_float2(b.z, b.w);
        s.l[1] = make_float2(c.x, c.y);
        s.l[2] = make_float2(c.z, c.w);
    }
    s.n[0] = make_float2(d.x, d.y);
    s.n[1] = make_float2(d.z, d.w);
    s.n[2] = make_float2(e.x, e.y);
    s.w = make_float2(e.z, e.w);
}

struct TgtPair {
    float2 h[3], l[3], n[3], w;
};

template <bool LO>
__device__ __forceinline__ void load_tgt(const float* soa, int64_t ntp, int64_t t0, TgtPair& t) {
    // t0 even: (t0, t0+1) from each plane as one float2
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        t.h[k] = *reinterpret_cast<const float2*>(soa + (0 + k) * ntp + t0);
        if (LO) t.l[k] = *reinterpret_cast<const float2*>(soa + (3 + k) * ntp + t0);
        t.n[k] = *reinterpret_cast<const float2*>(soa + (6 + k) * ntp + t0);
    }
    t.w = *reinterpret_cast<const float2*>(soa + 9 * ntp + t0);
}

struct Acc8 {
    float2 v[TP_NACC];  // Ew, U, Gn[3], Gx[3]
};

template <int Q>
__device__ __forceinline__ float2 powq_m1(float2 x, float2& xq) {
    // returns x^(Q-1), sets xq = x^Q (Q even: 6 or 8)
    float2 x2 = mul2(x, x);
    float2 x4 = mul2(x2, x2);
    if (Q == 6) {
        xq = mul2(x4, x2);
        return mul2(x4, x);
    } else {
        float2 x8 = mul2(x4, x4);
        xq = x8;
        return mul2(mul2(x4, x2), x);
    }
}

#ifndef TP_DIFF_FMA
#define TP_DIFF_FMA 0
#endif
template <bool LO>
__device__ __forceinline__ void pair_diff(const TgtPair& t, const SrcRec& s, float2 d[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#if TP_DIFF_FMA
        const float2 m1 = f2(-1.0f);
        if (LO) d[k] = add2(fma2(s.h[k], m1, t.h[k]), fma2(s.l[k], m1, t.l[k]));
        else d[k] = fma2(s.h[k], m1, t.h[k]);
#else
        if (LO) d[k] = add2(add2(t.h[k], neg2(s.h[k])), add2(t.l[k], neg2(s.l[k])));
        else d[k] = add2(t.h[k], neg2(s.h[k]));
#endif
    }
}

// x^(Q-1) (Q even: 6 or 8)
template <int Q>
__device__ __forceinline__ float2 powm1(float2 x) {
    float2 x2 = mul2(x, x);
    float2 x4 = mul2(x2, x2);
    if (Q == 6) return mul2(x4, x);
    return mul2(mul2(x4, x2), x);
}


// x^(Q-1) into xm1 and x^Q + addend into sum (the last product fused with the add)
template <int Q>
__device__ __forceinline__ void powq_m1_fma(float2 x, float2 addend, float2& xm1, float2& sum) {
    float2 x2 = mul2(x, x);
    float2 x4 = mul2(x2, x2);
    if (Q == 6) {
        sum = fma2(x4, x2, addend);
        xm1 = mul2(x4, x);
    } else {
        sum = fma2(x4, x4, addend);
        xm1 = mul2(mul2(x4, x2), x);
    }
}

// Geometry of one packed evaluation that does not depend on the normals:
// d = x_T - x_S and inv = 1/|d|^2 (computed one source ahead in the
// pipelined loop, so the reciprocal's latency overlaps other work).
struct PairPre {
    float2 d[3];
    float2 inv;
    float2 r2;
};

template <int KIND>
__device__ __forceinline__ void pair_pre(const TgtPair& t, const SrcRec& s, PairPre& p) {
    pair_diff<KIND != K_FAST>(t, s, p.d);
    float2 r2 = mul2(p.d[0], p.d[0]);
    r2 = fma2(p.d[1], p.d[1], r2);
    r2 = fma2(p.d[2], p.d[2], r2);
    p.r2 = r2;
    p.inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
}

// The rest of one packed evaluation: target pair t against one source s (both
// halves share s).  valid: per half 1 admitted, 0 excluded (MASKED only).
// FIRST: the source partials `as` are initialised by this call instead of
// accumulated.  Source-side sign convention: `as` carries +B5 in slot 1 and
// +(A5 nu_T + nk d) in slots 5..7, i.e. the negatives of the U and Gx
// contributions to S; the chunk epilogue flips their sign (no per-pair
// negations).
template <int Q, int KIND, bool FIRST>
__device__ __forceinline__ void pair_post(const TgtPair& t, const SrcRec& s, const PairPre& p, Acc8& at, Acc8& as,
                                          float2 valid) {
    const float2* d = p.d;
    float2 inv = p.inv;
    float2 wts = mul2(t.w, s.w);
    if (KIND == K_MASKED) {
        inv = make_float2(valid.x != 0.f ? inv.x : 0.f, valid.y != 0.f ? inv.y : 0.f);
        wts = mul2(wts, valid);
    }
    float2 a = mul2(t.n[0], d[0]);
    a = fma2(t.n[1], d[1], a);
    a = fma2(t.n[2], d[2], a);
    float2 b = mul2(s.n[0], d[0]);
    b = fma2(s.n[1], d[1], b);
    b = fma2(s.n[2], d[2], b);
    float2 al = mul2(a, inv), be = mul2(b, inv);
#if TP_PAIR_T
    // wi s6 = wi (al^q + be^q) = A5 al + B5 be: no al^q, be^q or s6 of their own;
    // the pair energy E = wts s6 = (wi s6) |d|^2 is fused into both energy sums
    float2 al5 = powm1<Q>(al), be5 = powm1<Q>(be);
    float2 wi = mul2(wts, inv);
    float2 A5 = mul2(wi, al5);
    float2 B5 = mul2(wi, be5);
    const float2 tt = fma2(A5, al, mul2(B5, be));
    float2 nk = mul2(tt, f2(-2.0f));  // -(p/q) wts inv s6, p = 2q
    const float2 ew = tt, ewm = p.r2;
#else
    float2 alq;
    float2 al5 = powq_m1<Q>(al, alq);
    float2 be5, s6;
    powq_m1_fma<Q>(be, alq, be5, s6);  // be^(q-1), and s6 = be^q + al^q with one fused op
    float2 wi = mul2(wts, inv);
    float2 A5 = mul2(wi, al5);
    float2 B5 = mul2(wi, be5);
    float2 nk = mul2(mul2(wi, s6), f2(-2.0f));  // -(p/q) wts inv s6, p = 2q
    const float2 ew = wts, ewm = s6;
#endif
    // target side (E = wts s6 is fused into both energy accumulations)
    at.v[0] = fma2(ew, ewm, at.v[0]);
    at.v[1] = add2(at.v[1], A5);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        at.v[2 + k] = fma2(A5, d[k], at.v[2 + k]);
        at.v[5 + k] = fma2(nk, d[k], fma2(B5, s.n[k], at.v[5 + k]));
    }
    // source side (slots 1 and 5..7 negated, see above)
    if (FIRST) {
        as.v[0] = mul2(ew, ewm);
        as.v[1] = B5;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            as.v[2 + k] = mul2(B5, d[k]);
            as.v[5 + k] = fma2(nk, d[k], mul2(A5, t.n[k]));
        }
    } else {
        as.v[0] = fma2(ew, ewm, as.v[0]);
        as.v[1] = add2(as.v[1], B5);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            as.v[2 + k] = fma2(B5, d[k], as.v[2 + k]);
            as.v[5 + k] = fma2(nk, d[k], fma2(A5, t.n[k], as.v[5 + k]));
        }
    }
}

template <int Q, int KIND, bool FIRST>
__device__ __forceinline__ void pair_grad(const TgtPair& t, const SrcRec& s, Acc8& at, Acc8& as, float2 valid) {
    PairPre p;
    pair_pre<KIND>(t, s, p);
    pair_post<Q, KIND, FIRST>(t, s, p, at, as, valid);
}

// Energy only: returns w~_S * s6 per half (the caller multiplies by w~_T at the end).
template <int Q, int KIND>
__device__ __forceinline__ float2 pair_energy(const TgtPair& t, const SrcRec& s, float2 valid) {
    float2 d[3];
    pair_diff<KIND != K_FAST>(t, s, d);
    float2 r2 = mul2(d[0], d[0]);
    r2 = fma2(d[1], d[1], r2);
    r2 = fma2(d[2], d[2], r2);
    float2 inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    float2 ws = s.w;
    if (KIND == K_MASKED) {
        inv = make_float2(valid.x != 0.f ? inv.x : 0.f, valid.y != 0.f ? inv.y : 0.f);
        ws = mul2(ws, valid);
    }
    float2 a = mul2(t.n[0], d[0]);
    a = fma2(t.n[1], d[1], a);
    a = fma2(t.n[2], d[2], a);
    float2 b = mul2(s.n[0], d[0]);
    b = fma2(s.n[1], d[1], b);
    b = fma2(s.n[2], d[2], b);
    float2 al = mul2(a, inv), be = mul2(b, inv);
    float2 alq, beq;
    powq_m1<Q>(al, alq);
    powq_m1<Q>(be, beq);
    return mul2(ws, add2(alq, beq));
}

// Butterfly transpose-reduction of 8 per-lane values over the warp.  On
// return every lane holds the warp total of component ((lane >> 2) & 7).
__device__ __forceinline__ float warp_transpose_reduce8(float v[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = b4 ? v[i] : v[i + 4];
        float keep = b4 ? v[i + 4] : v[i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = b3 ? u[i] : u[i + 2];
        float keep = b3 ? u[i + 2] : u[i];
        w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float send = b2 ? w2[0] : w2[1];
    float keep = b2 ? w2[1] : w2[0];
    float r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

__device__ __forceinline__ bool share_vertex(int3 a, int3 b, int edge_only) {
    int k = (a.x == b.x) + (a.x == b.y) + (a.x == b.z) + (a.y == b.x) + (a.y == b.y) + (a.y == b.z) +
            (a.z == b.x) + (a.z == b.y) + (a.z == b.z);
    return edge_only ? (k >= 2) : (k >= 1);
}

__device__ __forceinline__ int3 load_face(const int32_t* Fs, int64_t k) {
    return make_int3(Fs[3 * k], Fs[3 * k + 1], Fs[3 * k + 2]);
}

// Work item fetched from the dynamic queue: kind and super-tile pair.
struct Item {
    int kind, I, J, m;  // m: position in the masked list (masked items)
};

__device__ __forceinline__ Item decode_item(const DirectArgs& A, unsigned w) {
    Item it;
    int32_t e;
    if (w < (unsigned)A.nm) {
        it.kind = K_MASKED;
        e = A.mlist[w];
    } else if (w < (unsigned)(A.nm + A.np)) {
        it.kind = K_PRECISE;
        e = A.plist[w - A.nm];
    } else if (w < (unsigned)(A.nm + A.np + A.nf)) {
        it.kind = K_FAST;
        e = A.flist[w - A.nm - A.np];
    } else {
        it.kind = -1;
        e = 0;
    }
    it.I = e >> 16;
    it.J = e & 0xffff;
    it.m = (int)w;
#if TP_DEBUG
    // a listed item names an upper-triangle pair of existing super-tiles
    if (it.kind >= 0 && !tp_dbg_ok(it.I <= it.J && it.J < A.nsup, A.derr)) it.kind = -1;
#endif
    return it;
}

// Double-buffered TMA staging of the 12 source chunks of one item.
struct ChunkPipe {
    float* chunk;
    uint64_t* mbar;
    uint32_t phases;  // bit b: parity of the next completion of buffer b
    __device__ void issue(const DirectArgs& A, int J, int c, int buf) {
        const float* srcp = A.src + ((int64_t)J * TP_SUPER + (int64_t)c * TP_CHUNK) * TP_SRCW;
        mbar_expect_tx(&mbar[buf], CHUNK_BYTES);
        tma_load_1d(chunk + buf * TP_CHUNK * TP_SRCW, srcp, CHUNK_BYTES, &mbar[buf]);
    }
    // wait for chunk c (buffer c & 1), then queue chunk c + 1; false on timeout
    __device__ bool acquire(const DirectArgs& A, int J, int c, const float*& cb) {
        const int buf = c & 1;
        const bool ok = mbar_wait_bounded(&mbar[buf], (phases >> buf) & 1u);
        phases ^= 1u << buf;
        if (__syncthreads_or(!ok)) return false;
        if (threadIdx.x == 0 && c + 1 < NCHUNK) issue(A, J, c + 1, buf ^ 1);
        cb = chunk + buf * TP_CHUNK * TP_SRCW;
        return true;
    }
};

// block-wide fetch of the next item (thread 0 takes it from the queue); WITH_M
// also passes the item's position in the masked list
template <bool WITH_M>
__device__ __forceinline__ Item fetch_item(const DirectArgs& A, int* s_item) {
    if (threadIdx.x == 0) {
        const unsigned w = atomicAdd(A.work, 1u);
        const Item it = decode_item(A, w);
        s_item[0] = it.kind;
        s_item[1] = it.I;
        s_item[2] = it.J;
        if (WITH_M) s_item[3] = it.m;
    }
    __syncthreads();
    Item it;
    it.kind = s_item[0];
    it.I = s_item[1];
    it.J = s_item[2];
    it.m = WITH_M ? s_item[3] : 0;
    __syncthreads();  // s_item may be overwritten by the next fetch
    return it;
}

// Block shape of the gradient kernels: W warps, each lane NP packed target
// pairs, W * 32 * NP * 2 = TP_SUPER targets per block.  The masked items
// (per-pair exclusion test, face indices in registers) use 12 warps x 2
// pairs; the precise and fast items 8 warps x 3 pairs, whose larger
// register budget holds a prefetched source record and amortises the
// per-source warp reduction over 6 targets per lane.
#ifndef TP_GRAD_W
#define TP_GRAD_W 8  // warps of the precise/fast gradient kernel (8 or 12)
#endif
#ifndef TP_GRAD_PREFETCH
#define TP_GRAD_PREFETCH 1  // 1: prefetch the next source record; 2: also its geometry
#endif
#ifndef TP_EFOLD_SMEM
#define TP_EFOLD_SMEM 0  // compensated energy sums of the gradient kernels: 0 registers, 1 shared memory
#endif
#ifndef TP_FAST_ONLY
#define TP_FAST_ONLY 0  // 1: the precise/fast launch takes the fast items only; precise items run in the masked launch
#endif
#ifndef TP_GRAD_RED
#define TP_GRAD_RED 1  // per-source warp reduction: 0 shuffle butterfly, 1 transposed through shared memory
#endif
// Transposed reduction of the source partials (TP_GRAD_RED 1): per warp two
// slabs of 16 rows (row = component + 8 x source of a 2-source step) of 32
// lanes' values.  TP_SLAB_PAD 1: rows padded to 36 floats, so that row r's
// 16-byte groups fall on banks 4r + 4j (mod 32): the stores of one row by 32
// lanes and the 16-byte loads of 8 lanes reading rows r..r+7 are free of bank
// conflicts, and the store addresses are one base plus immediates.
// TP_SLAB_PAD 0: unpadded rows with the column XOR-swizzled by the row.
#ifndef TP_SLAB_PAD
#define TP_SLAB_PAD 0
#endif
constexpr int SLAB_ROW = TP_SLAB_PAD ? 36 : 32;
constexpr int SLAB_FLOATS = 16 * SLAB_ROW;
template <bool MASKQ>
struct GradShape {
    static constexpr int W = MASKQ ? 12 : TP_GRAD_W;
    static constexpr int NP = TP_SUPER / (64 * W);
    static constexpr int PF = MASKQ ? 1 : TP_GRAD_PREFETCH;  // source pipeline depth (register budget)
    static constexpr int RED = MASKQ ? 0 : TP_GRAD_RED;
    static constexpr int THREADS = 32 * W;
    static constexpr int SLAB_BYTES = RED == 1 ? W * 2 * SLAB_FLOATS * 4 : 0;
    static constexpr int EFOLD_BYTES = TP_EFOLD_SMEM ? W * NP * 32 * 16 : 0;
    static constexpr int SMEM = W * TP_CHUNK * TP_NACC * 4 + SLAB_BYTES + EFOLD_BYTES + 2 * CHUNK_BYTES + 64;
    static_assert(W * 32 * NP * 2 == TP_SUPER, "a block owns one super-tile of targets");
};

// One source of a precise/fast item: prefetch the next source record, the NP
// packed evaluations, then the warp reduction of the previous source (its
// shuffle chain overlaps this source's arithmetic).
template <int Q, int KIND, int NP>
__device__ __forceinline__ void src_step(const TgtPair (&tp)[NP], Acc8 (&at)[NP], const SrcRec& cur, SrcRec& nxt,
                                         const float* nrec, bool has_next, bool has_prev, float (&vprev)[8],
                                         float* sacc_prev, int lane) {
    constexpr bool LO = KIND != K_FAST;
    if (has_next) load_src<LO>(nrec, nxt);
    const float2 one = make_float2(1.f, 1.f);
    Acc8 as;
    pair_grad<Q, KIND, true>(tp[0], cur, at[0], as, one);
#pragma unroll
    for (int P = 1; P < NP; ++P) pair_grad<Q, KIND, false>(tp[P], cur, at[P], as, one);
    if (has_prev) {
        const float r = warp_transpose_reduce8(vprev, lane);
        if ((lane & 3) == 0) sacc_prev[(lane >> 2) & 7] = r;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) vprev[k] = as.v[k].x + as.v[k].y;
}

// One source of a precise/fast item with the transposed reduction: prefetch
// the next source record, the NP packed evaluations, then the lane's 8 source
// partials (both halves added) stored into rows row0..row0+7 of the slab.
// Row r, lane l is stored at r * 36 + l (padded rows) or r * 32 + (l ^ ((r & 7)
// << 2)) (swizzled rows): either way each store of a row covers the 32 banks
// once, and a load of 16 bytes by 8 lanes reading rows r..r+7 at one logical
// column covers them once as well.
template <int Q, int KIND, int NP>
__device__ __forceinline__ void src_step_slab(const TgtPair (&tp)[NP], Acc8 (&at)[NP], const SrcRec& cur,
                                              SrcRec& nxt, const float* nrec, bool has_next, float* slab_row0,
                                              int lane) {
    constexpr bool LO = KIND != K_FAST;
    if (has_next) load_src<LO>(nrec, nxt);
    const float2 one = make_float2(1.f, 1.f);
    Acc8 as;
    pair_grad<Q, KIND, true>(tp[0], cur, at[0], as, one);
#pragma unroll
    for (int P = 1; P < NP; ++P) pair_grad<Q, KIND, false>(tp[P], cur, at[P], as, one);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (TP_SLAB_PAD) slab_row0[k * SLAB_ROW + lane] = as.v[k].x + as.v[k].y;
        else slab_row0[k * 32 + (lane ^ (k << 2))] = as.v[k].x + as.v[k].y;
    }
}

// Column sums of one slab (16 rows: 8 components x 2 sources) over the 32
// lanes that stored them: lane l sums half a row (row l & 15, logical columns
// 16 (l >> 4) .. + 15) with four 16-byte loads, the two halves meet by one
// shuffle, and lanes 0..15 write the 16 totals (source-major, component-minor:
// the order of the warp's partial array) to out[0..15].
__device__ __forceinline__ void slab_reduce(const float* slab, float* out, int lane) {
    const int r = lane & 15, h = lane >> 4;
    const float* row = slab + r * SLAB_ROW;
    const int xr = TP_SLAB_PAD ? 0 : (r & 7) << 2;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = *reinterpret_cast<const float4*>(row + (((h << 4) | (k << 2)) ^ xr));
        v += (q.x + q.y) + (q.z + q.w);
    }
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    if (lane < 16) out[lane] = v;
}

// Pipelined variant of src_step: the normal-independent geometry of the next
// source (pn) is formed while the current source (geometry pc) is finished.
template <int Q, int KIND, int NP>
__device__ __forceinline__ void src_step_pp(const TgtPair (&tp)[NP], Acc8 (&at)[NP], const SrcRec& cur,
                                            const PairPre (&pc)[NP], SrcRec& nxt, PairPre (&pn)[NP],
                                            const float* nrec, bool has_next, bool has_prev, float (&vprev)[8],
                                            float* sacc_prev, int lane) {
    constexpr bool LO = KIND != K_FAST;
    if (has_next) {
        load_src<LO>(nrec, nxt);
#pragma unroll
        for (int P = 0; P < NP; ++P) pair_pre<KIND>(tp[P], nxt, pn[P]);
    }
    const float2 one = make_float2(1.f, 1.f);
    Acc8 as;
    pair_post<Q, KIND, true>(tp[0], cur, pc[0], at[0], as, one);
#pragma unroll
    for (int P = 1; P < NP; ++P) pair_post<Q, KIND, false>(tp[P], cur, pc[P], at[P], as, one);
    if (has_prev) {
        const float r = warp_transpose_reduce8(vprev, lane);
        if ((lane & 3) == 0) sacc_prev[(lane >> 2) & 7] = r;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) vprev[k] = as.v[k].x + as.v[k].y;
}

// Fold the FP32 energy partials of the targets into a compensated sum.  A
// target's energy terms can span many orders of magnitude (the nearest
// sources dominate), and a long FP32 running sum drops the small terms that
// follow a large one, so the plain FP32 partials cover at most 32 sources (or
// one chunk) and are then added to (s, c) with Kahan's compensated summation
// in FP32 (FP64 arithmetic is far slower on this part).
struct EFold {
    float2 s, c;  // running sum and its compensation, per packed target pair
};

// The same compensated sums kept in shared memory instead of registers: this
// lane's (s.x, s.y, c.x, c.y) per packed target pair at p[32 P].
struct EFoldSmem {
    float4* p;
};

template <int NP>
__device__ __forceinline__ void fold_energy(Acc8 (&at)[NP], EFoldSmem ef) {
    const float2 m1 = f2(-1.0f);
#pragma unroll
    for (int P = 0; P < NP; ++P) {
        const float4 q = ef.p[32 * P];
        const float2 s0 = make_float2(q.x, q.y), c0 = make_float2(q.z, q.w);
        const float2 y = fma2(c0, m1, at[P].v[0]);
        const float2 t = add2(s0, y);
        const float2 c = fma2(y, m1, fma2(s0, m1, t));
        ef.p[32 * P] = make_float4(t.x, t.y, c.x, c.y);
        at[P].v[0] = make_float2(0.f, 0.f);
    }
}

template <int NP>
__device__ __forceinline__ void fold_energy(Acc8 (&at)[NP], EFold (&ef)[NP]) {
    const float2 m1 = f2(-1.0f);
#pragma unroll
    for (int P = 0; P < NP; ++P) {
        const float2 y = fma2(ef[P].c, m1, at[P].v[0]);       // y = part - c
        const float2 t = add2(ef[P].s, y);                      // t = s + y
        ef[P].c = fma2(y, m1, fma2(ef[P].s, m1, t));            // c = (t - s) - y
        ef[P].s = t;
        at[P].v[0] = make_float2(0.f, 0.f);
    }
}

// The 12 chunks of one item for one item kind; target partials in `at`.
template <int Q, int KIND, int W, int NP, int PF, class EF>
__device__ __forceinline__ bool grad_item(const DirectArgs& A, ChunkPipe& pipe, float* sacc, int I, int J, int m,
                                          const TgtPair (&tp)[NP], Acc8 (&at)[NP], EF& e64, int warp,
                                          int lane, int pbase) {
    constexpr bool LO = KIND != K_FAST;
    constexpr bool SLABRED = KIND != K_MASKED && PF == 1 && TP_GRAD_RED == 1 && W == GradShape<false>::W &&
                             !(TP_FAST_ONLY && KIND == K_PRECISE);
    const int64_t ntp = A.ntp;
    int3 tf[NP][2];
    int tl[NP][2];  // target positions within the super-tile
    if (KIND == K_MASKED) {
#pragma unroll
        for (int P = 0; P < NP; ++P)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                tl[P][h] = 2 * (pbase + 32 * P) + h;
                tf[P][h] = load_face(A.Fs, (int64_t)I * TP_SUPER + tl[P][h]);
            }
    }
    for (int c = 0; c < NCHUNK; ++c) {
        const float* cb;
        if (!pipe.acquire(A, J, c, cb)) return false;
        const int64_t sbase = (int64_t)J * TP_SUPER + (int64_t)c * TP_CHUNK;
        // Masked items (one 128-target block per warp): on the diagonal, a chunk below
        // the warp's block has no admitted pair (admitted: source index > target index)
        // and the chunk level with it needs the per-pair test; elsewhere only blocks
        // that hold a vertex-sharing pair need it, the others take the unmasked path.
        static_assert(KIND != K_MASKED || 64 * NP == TP_CHUNK, "masked items need one 128-target block per warp");
        bool skip = false, masked = false;
        if (KIND == K_MASKED) {
            if (I == J && c < warp) {
                skip = true;
            } else if (I == J && c == warp) {
                masked = true;
            } else {
                const int blk = warp * TP_NBLK + c;
                const unsigned wd = __ldg(&A.bmask[((int64_t)I * A.nsup + J) * TP_BMASK_WORDS + (blk >> 5)]);
                masked = (wd >> (blk & 31)) & 1u;
            }
        }
        float* wacc = sacc + warp * TP_CHUNK * TP_NACC;
        if (masked && !A.edge_only) {
            // exclusion bits of this block: 128 bits per target of the lane, bit s set
            // where (target, source s) is not admitted
            const uint64_t* xp = reinterpret_cast<const uint64_t*>(A.partial);
            const uint32_t* xmask = reinterpret_cast<const uint32_t*>(xp[0]);
            const unsigned* e = reinterpret_cast<const unsigned*>(xp[1]) + (int64_t)m * TP_BMASK_WORDS;
            const int32_t* xbase = reinterpret_cast<const int32_t*>(xp[2]);
            const int blk = warp * TP_NBLK + c;
            int r = 0;
            for (int wd = 0; wd < (blk >> 5); ++wd) r += __popc(e[wd]);
            r += __popc(e[blk >> 5] & ((1u << (blk & 31)) - 1u));
            const int64_t slot = (int64_t)xbase[m] + r;
            uint4 xb[NP][2];
#pragma unroll
            for (int P = 0; P < NP; ++P)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    xb[P][h] = *reinterpret_cast<const uint4*>(
                        xmask + (slot * TP_CHUNK + (tl[P][h] - TP_CHUNK * warp)) * 4);
#pragma unroll
            for (int wd = 0; wd < 4; ++wd) {
                uint32_t xw[NP][2];
#pragma unroll
                for (int P = 0; P < NP; ++P)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        xw[P][h] = wd == 0 ? xb[P][h].x : wd == 1 ? xb[P][h].y : wd == 2 ? xb[P][h].z : xb[P][h].w;
#pragma unroll 1
                for (int i = 0; i < 32; ++i) {
                    const int s = 32 * wd + i;
                    SrcRec sr;
                    load_src<LO>(cb + s * TP_SRCW, sr);
                    Acc8 as;
                    float2 valid[NP];
#pragma unroll
                    for (int P = 0; P < NP; ++P)
                        valid[P] = make_float2((xw[P][0] >> i) & 1u ? 0.f : 1.f, (xw[P][1] >> i) & 1u ? 0.f : 1.f);
                    pair_grad<Q, KIND, true>(tp[0], sr, at[0], as, valid[0]);
#pragma unroll
                    for (int P = 1; P < NP; ++P) pair_grad<Q, KIND, false>(tp[P], sr, at[P], as, valid[P]);
                    float v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = as.v[k].x + as.v[k].y;
                    const float rr = warp_transpose_reduce8(v, lane);
                    if ((lane & 3) == 0) wacc[s * TP_NACC + ((lane >> 2) & 7)] = rr;
                }
            }
            fold_energy<NP>(at, e64);
        } else if (masked) {
            // exclusion by comparing vertex indices (edge-only exclusion)
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; ++s) {
                SrcRec sr;
                load_src<LO>(cb + s * TP_SRCW, sr);
                Acc8 as;
                float2 valid[NP];
                const int sl = c * TP_CHUNK + s;
                const int3 sf = load_face(A.Fs, sbase + s);
#pragma unroll
                for (int P = 0; P < NP; ++P) {
                    float v0 = ((I != J || sl > tl[P][0]) && !share_vertex(tf[P][0], sf, A.edge_only)) ? 1.f : 0.f;
                    float v1 = ((I != J || sl > tl[P][1]) && !share_vertex(tf[P][1], sf, A.edge_only)) ? 1.f : 0.f;
                    valid[P] = make_float2(v0, v1);
                }
                pair_grad<Q, KIND, true>(tp[0], sr, at[0], as, valid[0]);
#pragma unroll
                for (int P = 1; P < NP; ++P) pair_grad<Q, KIND, false>(tp[P], sr, at[P], as, valid[P]);
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = as.v[k].x + as.v[k].y;
                const float r = warp_transpose_reduce8(v, lane);
                if ((lane & 3) == 0) wacc[s * TP_NACC + ((lane >> 2) & 7)] = r;
            }
            fold_energy<NP>(at, e64);
        } else if (!skip) {
            // two sources per trip with alternating record registers: the next
            // source's record is loaded while the current one is evaluated
            constexpr int KU = KIND == K_MASKED ? K_PRECISE : KIND;  // unmasked blocks of masked items
            constexpr bool LOU = KU != K_FAST;
            float vprev[8];
            SrcRec ra, rb;
            if constexpr (PF == 2) {
            PairPre pa[NP], pb[NP];
            load_src<LOU>(cb, ra);
#pragma unroll
            for (int P = 0; P < NP; ++P) pair_pre<KU>(tp[P], ra, pa[P]);
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; s += 2) {
                src_step_pp<Q, KU, NP>(tp, at, ra, pa, rb, pb, cb + (s + 1) * TP_SRCW, true, s > 0, vprev,
                                         wacc + (s - 1) * TP_NACC, lane);
                src_step_pp<Q, KU, NP>(tp, at, rb, pb, ra, pa, cb + (s + 2) * TP_SRCW, s + 2 < TP_CHUNK, true,
                                         vprev, wacc + s * TP_NACC, lane);
                if ((s & 30) == 30) fold_energy<NP>(at, e64);
            }
            } else if constexpr (PF == 1 && KIND == K_MASKED) {
            // Unmasked blocks of masked items, with a branch-free loop body: the
            // first step reduces zeros into source 0's slots (overwritten by source
            // 0's own sums one step later, same lanes, program order), and the last
            // prefetch re-reads record TP_CHUNK - 1.  In the masked kernel this
            // form compiles without spills (161 registers against 168 and a spilled
            // stack frame) and takes about 0.25 ms less per evaluation at 327,680
            // triangles; in the precise/fast kernel the guarded form below is
            // faster (89.5 against 90.1 ms).
            load_src<LOU>(cb, ra);
#pragma unroll
            for (int k = 0; k < 8; ++k) vprev[k] = 0.f;
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; s += 2) {
                src_step<Q, KU, NP>(tp, at, ra, rb, cb + (s + 1) * TP_SRCW, true, true, vprev,
                                      wacc + (s > 0 ? s - 1 : 0) * TP_NACC, lane);
                src_step<Q, KU, NP>(tp, at, rb, ra, cb + min(s + 2, TP_CHUNK - 1) * TP_SRCW, true, true, vprev,
                                      wacc + s * TP_NACC, lane);
                if ((s & 30) == 30) fold_energy<NP>(at, e64);
            }
            } else if constexpr (PF == 1 && SLABRED) {
            // Two sources per trip; their 16 partials go to one slab, and the
            // previous trip's slab is summed first (its loads and adds overlap
            // this trip's arithmetic).  The __syncwarp at the end of a trip
            // orders a slab's stores before its loads one trip later, and those
            // loads before the stores into it two trips later.
            float* slab = sacc + W * TP_CHUNK * TP_NACC + warp * 2 * SLAB_FLOATS;
            load_src<LOU>(cb, ra);
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; s += 2) {
                float* sw = slab + ((s >> 1) & 1) * SLAB_FLOATS;
                if (s > 0) slab_reduce(slab + (((s >> 1) - 1) & 1) * SLAB_FLOATS, wacc + (s - 2) * TP_NACC, lane);
                src_step_slab<Q, KU, NP>(tp, at, ra, rb, cb + (s + 1) * TP_SRCW, true, sw, lane);
                src_step_slab<Q, KU, NP>(tp, at, rb, ra, cb + (s + 2) * TP_SRCW, s + 2 < TP_CHUNK,
                                         sw + 8 * SLAB_ROW, lane);
                if ((s & 30) == 30) fold_energy<NP>(at, e64);
                __syncwarp();
            }
            slab_reduce(slab + ((TP_CHUNK / 2 - 1) & 1) * SLAB_FLOATS, wacc + (TP_CHUNK - 2) * TP_NACC, lane);
            } else if constexpr (PF == 1) {
            load_src<LOU>(cb, ra);
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; s += 2) {
                src_step<Q, KU, NP>(tp, at, ra, rb, cb + (s + 1) * TP_SRCW, true, s > 0, vprev,
                                      wacc + (s - 1) * TP_NACC, lane);
                src_step<Q, KU, NP>(tp, at, rb, ra, cb + (s + 2) * TP_SRCW, s + 2 < TP_CHUNK, true, vprev,
                                      wacc + s * TP_NACC, lane);
                if ((s & 30) == 30) fold_energy<NP>(at, e64);
            }
            } else {
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; ++s) {
                load_src<LOU>(cb + s * TP_SRCW, ra);
                src_step<Q, KU, NP>(tp, at, ra, rb, nullptr, false, s > 0, vprev, wacc + (s - 1) * TP_NACC,
                                      lane);
                if ((s & 31) == 31) fold_energy<NP>(at, e64);
            }
            }
            if constexpr (!SLABRED) {
                const float r = warp_transpose_reduce8(vprev, lane);
                if ((lane & 3) == 0) wacc[(TP_CHUNK - 1) * TP_NACC + ((lane >> 2) & 7)] = r;
            }
        } else {
            for (int i = lane; i < TP_CHUNK * TP_NACC; i += 32) wacc[i] = 0.f;
        }
        __syncthreads();
        // sum the warps' source partials of this chunk, undo the sign convention of
        // slots 1 and 5..7 (see pair_grad) and promote to FP64
        for (int i = threadIdx.x; i < TP_CHUNK * TP_NACC; i += 32 * W) {
            float ssum = 0.f;
#pragma unroll
            for (int w = 0; w < W; ++w) ssum += sacc[w * TP_CHUNK * TP_NACC + i];
            const int s = i / TP_NACC, comp = i % TP_NACC;
            if (comp == 1 || comp >= 5) ssum = -ssum;
            if (ssum != 0.f) atomicAdd(&A.acc[comp * ntp + sbase + s], (double)ssum);
        }
        __syncthreads();
    }
    return true;
}

// ------------------------------------------------------------ gradient kernel
// Persistent: every block takes items from the queue until it is empty.  Two
// instantiations: MASKQ = true serves the masked items (per-pair exclusion
// test), MASKQ = false the precise and fast items (each has its own block
// shape and register budget, see GradShape).
template <int Q, bool MASKQ>
__global__ void __launch_bounds__(GradShape<MASKQ>::THREADS, 1) k_pairs_grad(DirectArgs A) {
    constexpr int W = GradShape<MASKQ>::W, NP = GradShape<MASKQ>::NP;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int SACC_BYTES =
        W * TP_CHUNK * TP_NACC * 4 + GradShape<MASKQ>::SLAB_BYTES + GradShape<MASKQ>::EFOLD_BYTES;
    float* sacc = reinterpret_cast<float*>(smem);  // [W][CHUNK][8], then slabs, then energy folds
    float* chunk = reinterpret_cast<float*>(smem + SACC_BYTES);                   // [2][CHUNK][SRCW]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + SACC_BYTES + 2 * CHUNK_BYTES);
    int* s_item = reinterpret_cast<int*>(smem + SACC_BYTES + 2 * CHUNK_BYTES + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntp = A.ntp;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    ChunkPipe pipe;
    pipe.chunk = chunk;
    pipe.mbar = mbar;
    pipe.phases = 0u;

    TgtPair tp[NP];
    int rowI = -1;
    const int pbase = warp * 32 * NP + lane;  // pair index within the super-tile: pbase + 32 P
    while (true) {
        const Item it = fetch_item<MASKQ>(A, s_item);
        if (it.kind < 0) break;
        if (tid == 0) pipe.issue(A, it.J, 0, 0);
        if (it.I != rowI) {
            rowI = it.I;
#pragma unroll
            for (int P = 0; P < NP; ++P)
                load_tgt<!(TP_FAST_ONLY && !MASKQ)>(A.soa, ntp, (int64_t)it.I * TP_SUPER + 2 * (pbase + 32 * P), tp[P]);
        }
        Acc8 at[NP];
#if TP_EFOLD_SMEM
        EFoldSmem e64;
        e64.p = reinterpret_cast<float4*>(smem + W * TP_CHUNK * TP_NACC * 4 + GradShape<MASKQ>::SLAB_BYTES) +
                warp * NP * 32 + lane;
#pragma unroll
        for (int P = 0; P < NP; ++P) e64.p[32 * P] = make_float4(0.f, 0.f, 0.f, 0.f);
#else
        EFold e64[NP];
#pragma unroll
        for (int P = 0; P < NP; ++P) e64[P].s = e64[P].c = make_float2(0.f, 0.f);
#endif
#pragma unroll
        for (int P = 0; P < NP; ++P) {
#pragma unroll
            for (int c = 0; c < TP_NACC; ++c) at[P].v[c] = make_float2(0.f, 0.f);
        }
        bool ok;
        if constexpr (MASKQ) {
            if (TP_FAST_ONLY && it.kind == K_PRECISE)
                ok = grad_item<Q, K_PRECISE, W, NP, GradShape<MASKQ>::PF>(A, pipe, sacc, it.I, it.J, it.m, tp, at, e64, warp, lane, pbase);
            else
                ok = grad_item<Q, K_MASKED, W, NP, GradShape<MASKQ>::PF>(A, pipe, sacc, it.I, it.J, it.m, tp, at, e64, warp, lane, pbase);
        } else if constexpr (TP_FAST_ONLY) {
            ok = grad_item<Q, K_FAST, W, NP, GradShape<MASKQ>::PF>(A, pipe, sacc, it.I, it.J, it.m, tp, at, e64, warp, lane, pbase);
        } else {
            if (it.kind == K_FAST) ok = grad_item<Q, K_FAST, W, NP, GradShape<MASKQ>::PF>(A, pipe, sacc, it.I, it.J, it.m, tp, at, e64, warp, lane, pbase);
            else ok = grad_item<Q, K_PRECISE, W, NP, GradShape<MASKQ>::PF>(A, pipe, sacc, it.I, it.J, it.m, tp, at, e64, warp, lane, pbase);
        }
        if (!ok) {
            if (tid == 0) tp_dev_error(A.derr, TP_DERR_TIMEOUT);
            return;
        }
        // promote the item's target partials to FP64 (the energy already folded)
        fold_energy<NP>(at, e64);
#pragma unroll
        for (int P = 0; P < NP; ++P) {
            const int64_t t0 = (int64_t)it.I * TP_SUPER + 2 * (pbase + 32 * P);
#if TP_EFOLD_SMEM
            const float4 q = e64.p[32 * P];
            const double ex = (double)q.x - (double)q.z, ey = (double)q.y - (double)q.w;
#else
            const double ex = (double)e64[P].s.x - (double)e64[P].c.x, ey = (double)e64[P].s.y - (double)e64[P].c.y;
#endif
            if (ex != 0.0) atomicAdd(&A.acc[t0], ex);
            if (ey != 0.0) atomicAdd(&A.acc[t0 + 1], ey);
#pragma unroll
            for (int k = 1; k < TP_NACC; ++k) {
                if (at[P].v[k].x != 0.f) atomicAdd(&A.acc[k * ntp + t0], (double)at[P].v[k].x);
                if (at[P].v[k].y != 0.f) atomicAdd(&A.acc[k * ntp + t0 + 1], (double)at[P].v[k].y);
            }
        }
    }
}

// ------------------------------------------------------------ energy kernel
template <int Q, int KIND>
__device__ __forceinline__ bool energy_item(const DirectArgs& A, ChunkPipe& pipe, int I, int J,
                                            const TgtPair (&tp)[2], float2 (&ea)[2], int warp, int pbase) {
    constexpr bool LO = KIND != K_FAST;
    int3 tf[2][2];
    int tl[2][2];
    if (KIND == K_MASKED) {
#pragma unroll
        for (int P = 0; P < 2; ++P)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                tl[P][h] = 2 * (pbase + 32 * P) + h;
                tf[P][h] = load_face(A.Fs, (int64_t)I * TP_SUPER + tl[P][h]);
            }
    }
    for (int c = 0; c < NCHUNK; ++c) {
        const float* cb;
        if (!pipe.acquire(A, J, c, cb)) return false;
        const int64_t sbase = (int64_t)J * TP_SUPER + (int64_t)c * TP_CHUNK;
        const bool skip = (KIND == K_MASKED) && (I == J) && (c < warp);
        // As in the gradient kernel, only the diagonal block and the 128 x 128
        // blocks that hold a vertex-sharing pair take the per-pair test; the
        // other blocks of a masked item run the unmasked arithmetic.
        bool masked = KIND == K_MASKED && !skip;
        if (KIND == K_MASKED && !skip && !(I == J && c == warp)) {
            const int blk = warp * TP_NBLK + c;
            const unsigned wd = __ldg(&A.bmask[((int64_t)I * A.nsup + J) * TP_BMASK_WORDS + (blk >> 5)]);
            masked = (wd >> (blk & 31)) & 1u;
        }
        if (KIND == K_MASKED && !skip && !masked) {
            const float2 one = make_float2(1.f, 1.f);
#pragma unroll 2
            for (int s = 0; s < TP_CHUNK; ++s) {
                SrcRec sr;
                load_src<true>(cb + s * TP_SRCW, sr);
#pragma unroll
                for (int P = 0; P < 2; ++P) ea[P] = add2(ea[P], pair_energy<Q, K_PRECISE>(tp[P], sr, one));
            }
        } else if (!skip) {
#pragma unroll 2
            for (int s = 0; s < TP_CHUNK; ++s) {
                SrcRec sr;
                load_src<LO>(cb + s * TP_SRCW, sr);
                float2 valid[2] = {make_float2(1.f, 1.f), make_float2(1.f, 1.f)};
                if (KIND == K_MASKED) {
                    const int sl = c * TP_CHUNK + s;
                    const int3 sf = load_face(A.Fs, sbase + s);
#pragma unroll
                    for (int P = 0; P < 2; ++P) {
                        float v0 = ((I != J || sl > tl[P][0]) && !share_vertex(tf[P][0], sf, A.edge_only)) ? 1.f : 0.f;
                        float v1 = ((I != J || sl > tl[P][1]) && !share_vertex(tf[P][1], sf, A.edge_only)) ? 1.f : 0.f;
                        valid[P] = make_float2(v0, v1);
                    }
                }
#pragma unroll
                for (int P = 0; P < 2; ++P) ea[P] = add2(ea[P], pair_energy<Q, KIND>(tp[P], sr, valid[P]));
            }
        }
        __syncthreads();
    }
    return true;
}

// Every lane accumulates sum_S w~_S s6 for its 4 targets in FP32 per item,
// promoted to FP64 per item; the block writes one FP64 partial, summed by a
// deterministic reduction.
template <int Q>
__global__ void __launch_bounds__(THREADS, 1) k_pairs_energy(DirectArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* chunk = reinterpret_cast<float*>(smem);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * CHUNK_BYTES);
    int* s_item = reinterpret_cast<int*>(smem + 2 * CHUNK_BYTES + 16);
    double* wsum = reinterpret_cast<double*>(smem + 2 * CHUNK_BYTES + 64);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntp = A.ntp;
    double esum = 0.0;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    ChunkPipe pipe;
    pipe.chunk = chunk;
    pipe.mbar = mbar;
    pipe.phases = 0u;
    const int pbase = warp * 64 + lane;
    TgtPair tp[2];
    int rowI = -1;
    while (true) {
        const Item it = fetch_item<false>(A, s_item);
        if (it.kind < 0) break;
        if (tid == 0) pipe.issue(A, it.J, 0, 0);
        if (it.I != rowI) {
            rowI = it.I;
#pragma unroll
            for (int P = 0; P < 2; ++P)
                load_tgt<true>(A.soa, ntp, (int64_t)it.I * TP_SUPER + 2 * (pbase + 32 * P), tp[P]);
        }
        float2 ea[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        bool ok;
        if (it.kind == K_FAST) ok = energy_item<Q, K_FAST>(A, pipe, it.I, it.J, tp, ea, warp, pbase);
        else if (it.kind == K_PRECISE) ok = energy_item<Q, K_PRECISE>(A, pipe, it.I, it.J, tp, ea, warp, pbase);
        else ok = energy_item<Q, K_MASKED>(A, pipe, it.I, it.J, tp, ea, warp, pbase);
        if (!ok) {
            if (tid == 0) tp_dev_error(A.derr, TP_DERR_TIMEOUT);
            break;
        }
#pragma unroll
        for (int P = 0; P < 2; ++P) esum += (double)(tp[P].w.x * ea[P].x) + (double)(tp[P].w.y * ea[P].y);
    }
    // deterministic block reduction (the block's item set itself depends on the queue order)
    for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
    if (lane == 0) wsum[warp] = esum;
    __syncthreads();
    if (tid == 0) {
        double b = 0.0;
        for (int w = 0; w < WARPS; ++w) b += wsum[w];
        A.partial[blockIdx.x] = b;
    }
}

// ------------------------------------------------------------ FP64 reference kernel (TP_F64)
// One thread per target, gather over every source (both orderings), FP64
// arithmetic throughout; writes the same accumulator convention.
template <int Q>
__global__ void k_pairs_f64(const double* x64, const double* nu64, const double* w64, const int32_t* F,
                            const int32_t* perm, int64_t nt, int64_t ntp, int edge_only, double* acc,
                            double* eper) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const double pq = 2.0;
    int64_t T = perm[k];
    double xt[3], nt3[3];
    for (int a = 0; a < 3; ++a) {
        xt[a] = x64[a * nt + T];
        nt3[a] = nu64[a * nt + T];
    }
    double wt = w64[T];
    int3 ft = make_int3(F[3 * T], F[3 * T + 1], F[3 * T + 2]);
    double Ew = 0, U = 0, Gn[3] = {0, 0, 0}, Gx[3] = {0, 0, 0}, es = 0;
    for (int64_t S = 0; S < nt; ++S) {
        if (S == T) continue;
        int3 fs = make_int3(F[3 * S], F[3 * S + 1], F[3 * S + 2]);
        if (share_vertex(ft, fs, edge_only)) continue;
        double d[3], r2 = 0, a = 0, b = 0;
        for (int c = 0; c < 3; ++c) {
            d[c] = xt[c] - x64[c * nt + S];
            r2 += d[c] * d[c];
        }
        for (int c = 0; c < 3; ++c) {
            a += nt3[c] * d[c];
            b += nu64[c * nt + S] * d[c];
        }
        double inv = 1.0 / r2, al = a * inv, be = b * inv;
        double al2 = al * al, be2 = be * be;
        double alq, beq, al5, be5;
        if (Q == 6) {
            alq = al2 * al2 * al2;
            beq = be2 * be2 * be2;
            al5 = al2 * al2 * al;
            be5 = be2 * be2 * be;
        } else {
            alq = al2 * al2 * al2 * al2;
            beq = be2 * be2 * be2 * be2;
            al5 = al2 * al2 * al2 * al;
            be5 = be2 * be2 * be2 * be;
        }
        double wts = pq * wt * w64[S];
        double s6 = alq + beq, E = wts * s6, wi = wts * inv, A5 = wi * al5, B5 = wi * be5, kk = pq * wi * s6;
        Ew += E;
        U += A5;
        es += wt * w64[S] * alq;
        for (int c = 0; c < 3; ++c) {
            Gn[c] += A5 * d[c];
            Gx[c] += B5 * nu64[c * nt + S] - kk * d[c];
        }
    }
    acc[0 * ntp + k] = Ew;
    acc[1 * ntp + k] = U;
    for (int c = 0; c < 3; ++c) {
        acc[(2 + c) * ntp + k] = Gn[c];
        acc[(5 + c) * ntp + k] = Gx[c];
    }
    eper[k] = es;
}

// ------------------------------------------------------------ compensated FP32 kernel (TP_F32_KAHAN)
// One thread per target (library order), gathering over every source: the
// pair terms in FP32 (centroid differences from hi + lo parts, as in the
// precise items of the symmetric kernel) and every one of the target's eight
// sums (Ew, U, Gn[3], Gx[3], both orderings) accumulated with Kahan's
// compensated summation in FP32, so that no sum is carried in FP64: FP64
// enters only when the finished sums are stored for the pull-back and the
// final energy reduction.  Each unordered pair is evaluated twice (once from
// each end), which the symmetric kernel avoids; this form trades that for
// sums whose error does not grow with the number of sources.
struct Kahan {
    float s, c;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

constexpr int KAHAN_TILE = 128;

template <int Q>
__global__ void __launch_bounds__(KAHAN_TILE) k_pairs_kahan(const float* __restrict__ soa, const int32_t* __restrict__ Fs,
                                                          int64_t nt, int64_t ntp, int edge_only,
                                                          double* __restrict__ acc) {
    __shared__ float sd[10][KAHAN_TILE];
    __shared__ int sf[3][KAHAN_TILE];
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = k < nt;
    float t[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) t[c] = active ? soa[c * ntp + k] : 0.f;
    const int3 ft = active ? make_int3(Fs[3 * k], Fs[3 * k + 1], Fs[3 * k + 2]) : make_int3(-1, -1, -1);
    Kahan K[TP_NACC];
#pragma unroll
    for (int c = 0; c < TP_NACC; ++c) K[c].s = K[c].c = 0.f;
    for (int64_t s0 = 0; s0 < nt; s0 += KAHAN_TILE) {
        __syncthreads();
        const int64_t S = s0 + threadIdx.x;
#pragma unroll
        for (int c = 0; c < 10; ++c) sd[c][threadIdx.x] = S < nt ? soa[c * ntp + S] : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) sf[c][threadIdx.x] = S < nt ? Fs[3 * S + c] : -1;
        __syncthreads();
        if (!active) continue;
        const int m = (nt - s0) < KAHAN_TILE ? (int)(nt - s0) : KAHAN_TILE;
        for (int j = 0; j < m; ++j) {
            if (s0 + j == k) continue;
            if (share_vertex(ft, make_int3(sf[0][j], sf[1][j], sf[2][j]), edge_only)) continue;
            float d[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) d[c] = (t[c] - sd[c][j]) + (t[3 + c] - sd[3 + c][j]);
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const float inv = rcp_approx(r2);
            const float a = t[6] * d[0] + t[7] * d[1] + t[8] * d[2];
            const float b = sd[6][j] * d[0] + sd[7][j] * d[1] + sd[8][j] * d[2];
            const float al = a * inv, be = b * inv;
            const float al2 = al * al, be2 = be * be, al4 = al2 * al2, be4 = be2 * be2;
            float al5, be5, alq, beq;
            if (Q == 6) {
                al5 = al4 * al;
                be5 = be4 * be;
                alq = al4 * al2;
                beq = be4 * be2;
            } else {
                al5 = al4 * al2 * al;
                be5 = be4 * be2 * be;
                alq = al4 * al4;
                beq = be4 * be4;
            }
            const float wts = t[9] * sd[9][j];  // w~_T w~_S = (p/q) w_T w_S
            const float s6 = alq + beq, wi = wts * inv;
            const float A5 = wi * al5, B5 = wi * be5, kk = 2.0f * wi * s6;  // p = 2q
            K[0].add(wts * s6);
            K[1].add(A5);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                K[2 + c].add(A5 * d[c]);
                K[5 + c].add(B5 * sd[6 + c][j] - kk * d[c]);
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int c = 0; c < TP_NACC; ++c) acc[c * ntp + k] = (double)K[c].s - (double)K[c].c;
}


template <int Q>
tp_status launch_grad_q(tp_ctx* ctx, DirectArgs A) {
    // the shared-memory limit is a per-device attribute: set it on the current device at every launch
    TP_CU(cudaFuncSetAttribute(k_pairs_grad<Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               GradShape<false>::SMEM));
    TP_CU(cudaFuncSetAttribute(k_pairs_grad<Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               GradShape<true>::SMEM));
    TP_CU(cudaMemsetAsync(ctx->work, 0, 2 * sizeof(unsigned), ctx->stream));
    // masked items first (their own queue), then the precise and fast items
    const int64_t nmq = ctx->n_masked + (TP_FAST_ONLY ? ctx->n_precise : 0);
    if (nmq > 0) {
        DirectArgs M = A;
        if (!TP_FAST_ONLY) M.np = 0;
        M.nf = 0;
        M.work = ctx->work + 1;
        M.partial = reinterpret_cast<double*>(ctx->xptrs);
        const int grid = (int)std::min<int64_t>(ctx->num_sms, nmq);
        k_pairs_grad<Q, true><<<grid, GradShape<true>::THREADS, GradShape<true>::SMEM, ctx->stream>>>(M);
        ++ctx->nlaunch;
    }
    const int64_t nrest = (TP_FAST_ONLY ? 0 : ctx->n_precise) + ctx->n_fast;
    cudaEventRecord(ctx->ev[0], ctx->stream);
    if (nrest > 0) {
        DirectArgs R = A;
        R.nm = 0;
        if (TP_FAST_ONLY) R.np = 0;
        const int grid = (int)std::min<int64_t>(ctx->num_sms, nrest);
        k_pairs_grad<Q, false><<<grid, GradShape<false>::THREADS, GradShape<false>::SMEM, ctx->stream>>>(R);
        ++ctx->nlaunch;
    }
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    return TP_OK;
}

template <int Q>
tp_status launch_energy_q(tp_ctx* ctx, DirectArgs A, int* nparts) {
    const int64_t nitems = ctx->n_masked + ctx->n_precise + ctx->n_fast;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms, nitems));
    TP_CU(cudaMemsetAsync(ctx->work, 0, sizeof(unsigned), ctx->stream));
    cudaEventRecord(ctx->ev[0], ctx->stream);
    k_pairs_energy<Q><<<grid, THREADS, SMEM_ENERGY, ctx->stream>>>(A);
    ++ctx->nlaunch;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    *nparts = grid;
    return TP_OK;
}

// ------------------------------------------------------------ confinement (Eq. TPConf)
// Phi_conf = c sum_{T in S} sum_{K in S_conf} w_T a_K |nu_T.(x_T - y_K)|^q / |x_T - y_K|^p
// (Sec. 2.2, Confinement): the target side of the pair kernel with only the
// al^q ordering, because the confining surface's normal never enters and it
// does not move.  With wts = w~_T w~_K (w~ = sqrt(p/q) area), inv = 1/|d|^2,
// al = nu_T.d inv:
//   Ew += wts al^q, U += A5 = wts inv al^(q-1), Gn += A5 d, Gx += -(p/q) wts inv al^q d,
// the direct kernel's accumulator convention, so the same adjoint gives the
// vertex gradient; Phi_conf = c sum_T Ew_T / (p/q).  No pair is excluded (the
// surfaces share no vertex); d always takes the hi/lo parts.

// FP64 centroid and area of each confining triangle (its normal is not needed)
__global__ void k_conf_tri(const double* __restrict__ V, const int32_t* __restrict__ F, int64_t nt, int64_t nv,
                           double* __restrict__ y64, double* __restrict__ a64, unsigned* derr) {
    const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K >= nt) return;
    const int32_t i0 = F[3 * K], i1 = F[3 * K + 1], i2 = F[3 * K + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        tp_dev_error(derr, TP_DERR_INDEX);
        for (int a = 0; a < 3; ++a) y64[a * nt + K] = 0.0;
        a64[K] = 0.0;
        return;
    }
    const double *pa = V + 3 * (int64_t)i0, *pb = V + 3 * (int64_t)i1, *pc = V + 3 * (int64_t)i2;
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        y64[k * nt + K] = __ddiv_rn(__dadd_rn(__dadd_rn(pa[k], pb[k]), pc[k]), 3.0);
        e1[k] = __dsub_rn(pb[k], pa[k]);
        e2[k] = __dsub_rn(pc[k], pa[k]);
    }
    const double N0 = e1[1] * e2[2] - e1[2] * e2[1], N1 = e1[2] * e2[0] - e1[0] * e2[2],
                 N2 = e1[0] * e2[1] - e1[1] * e2[0];
    const double area = 0.5 * sqrt(N0 * N0 + N1 * N1 + N2 * N2);
    if (!isfinite(area) || !isfinite(y64[K]) || !isfinite(y64[nt + K]) || !isfinite(y64[2 * nt + K]))
        tp_dev_error(derr, TP_DERR_NONFINITE);
    a64[K] = area;
}

// staged source records (the direct kernel's layout, normal zero) relative to
// the evolving mesh's centre; padding: zero area, far away
__global__ void k_conf_records(const double* __restrict__ y64, const double* __restrict__ a64,
                               const double* __restrict__ center, int64_t nt, int64_t ntp, float* __restrict__ src) {
    const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (K >= ntp) return;
    float v[10];
    if (K < nt) {
        for (int a = 0; a < 3; ++a) {
            const double yc = y64[a * nt + K] - center[a];
            const float hi = (float)yc;
            v[a] = hi;
            v[3 + a] = (float)(yc - (double)hi);
            v[6 + a] = 0.f;
        }
        v[9] = (float)(1.4142135623730951 * a64[K]);  // sqrt(p/q) a, p = 2q
    } else {
        v[0] = 8192.0f + 8.0f * (float)(K - nt);
        v[1] = v[2] = 8192.0f;
        for (int a = 3; a < 10; ++a) v[a] = 0.f;
    }
    for (int a = 0; a < 10; ++a) {
        src[K * TP_SRCW + 2 * a] = v[a];
        src[K * TP_SRCW + 2 * a + 1] = v[a];
    }
}

// centroid hi/lo and weight of a staged record (the normal is not read)
__device__ __forceinline__ void load_src_pos(const float* rec, SrcRec& s) {
    const float4* r = reinterpret_cast<const float4*>(rec);
    const float4 a = r[0], b = r[1], c = r[2], e = r[4];
    s.h[0] = make_float2(a.x, a.y);
    s.h[1] = make_float2(a.z, a.w);
    s.h[2] = make_float2(b.x, b.y);
    s.l[0] = make_float2(b.z, b.w);
    s.l[1] = make_float2(c.x, c.y);
    s.l[2] = make_float2(c.z, c.w);
    s.w = make_float2(e.z, e.w);
}

template <int Q>
__device__ __forceinline__ void conf_pair(const TgtPair& t, const SrcRec& s, Acc8& at) {
    float2 d[3];
    pair_diff<true>(t, s, d);
    float2 r2 = mul2(d[0], d[0]);
    r2 = fma2(d[1], d[1], r2);
    r2 = fma2(d[2], d[2], r2);
    const float2 inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    const float2 wts = mul2(t.w, s.w);
    float2 a = mul2(t.n[0], d[0]);
    a = fma2(t.n[1], d[1], a);
    a = fma2(t.n[2], d[2], a);
    const float2 al = mul2(a, inv);
#if TP_PAIR_T
    // wi al^q = A5 al; the pair energy wts al^q = (wi al^q) |d|^2; Gx collects
    // (wi al^q) d, and its factor -(p/q) = -2 is applied once per item
    const float2 al5 = powm1<Q>(al);
    const float2 wi = mul2(wts, inv);
    const float2 A5 = mul2(wi, al5);
    const float2 tt = mul2(A5, al);
    at.v[0] = fma2(tt, r2, at.v[0]);
    at.v[1] = add2(at.v[1], A5);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        at.v[2 + k] = fma2(A5, d[k], at.v[2 + k]);
        at.v[5 + k] = fma2(tt, d[k], at.v[5 + k]);
    }
#else
    float2 alq;
    const float2 al5 = powq_m1<Q>(al, alq);
    const float2 wi = mul2(wts, inv);
    const float2 A5 = mul2(wi, al5);
    const float2 nk = mul2(mul2(wi, alq), f2(-2.0f));  // -(p/q) wts inv al^q, p = 2q
    at.v[0] = fma2(wts, alq, at.v[0]);
    at.v[1] = add2(at.v[1], A5);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        at.v[2 + k] = fma2(A5, d[k], at.v[2 + k]);
        at.v[5 + k] = fma2(nk, d[k], at.v[5 + k]);
    }
#endif
}
// factor of the Gx partials of conf_pair at the end of an item
constexpr float CONF_GX_SCALE = TP_PAIR_T ? -2.0f : 1.0f;

// Persistent: items (target super-tile I, confining super-tile J) for all I, J,
// from a dynamic queue; block shape of the precise/fast gradient kernel.
template <int Q>
__global__ void __launch_bounds__(GradShape<false>::THREADS, 1) k_conf_grad(DirectArgs A) {
    constexpr int NP = GradShape<false>::NP;
    extern __shared__ __align__(128) unsigned char smem[];
    float* chunk = reinterpret_cast<float*>(smem);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * CHUNK_BYTES);
    int* s_item = reinterpret_cast<int*>(smem + 2 * CHUNK_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntp = A.ntp;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    ChunkPipe pipe;
    pipe.chunk = chunk;
    pipe.mbar = mbar;
    pipe.phases = 0u;
    TgtPair tp[NP];
    int rowI = -1;
    const int pbase = warp * 32 * NP + lane;
    const unsigned nitems = (unsigned)A.nf;  // nsup x nsup_conf
    while (true) {
        if (tid == 0) {
            const unsigned w = atomicAdd(A.work, 1u);
            s_item[0] = w < nitems ? (int)(w / (unsigned)A.np) : -1;
            s_item[1] = w < nitems ? (int)(w % (unsigned)A.np) : 0;
        }
        __syncthreads();
        const int I = s_item[0], J = s_item[1];
        __syncthreads();
        if (I < 0) break;
        if (tid == 0) pipe.issue(A, J, 0, 0);
        if (I != rowI) {
            rowI = I;
#pragma unroll
            for (int P = 0; P < NP; ++P) load_tgt<true>(A.soa, ntp, (int64_t)I * TP_SUPER + 2 * (pbase + 32 * P), tp[P]);
        }
        Acc8 at[NP];
        EFold e64[NP];
#pragma unroll
        for (int P = 0; P < NP; ++P) {
            e64[P].s = e64[P].c = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < TP_NACC; ++k) at[P].v[k] = make_float2(0.f, 0.f);
        }
        for (int c = 0; c < NCHUNK; ++c) {
            const float* cb;
            if (!pipe.acquire(A, J, c, cb)) {
                if (tid == 0) tp_dev_error(A.derr, TP_DERR_TIMEOUT);
                return;
            }
            SrcRec ra, rb;
            load_src_pos(cb, ra);
#pragma unroll 1
            for (int s = 0; s < TP_CHUNK; s += 2) {
                load_src_pos(cb + (s + 1) * TP_SRCW, rb);
#pragma unroll
                for (int P = 0; P < NP; ++P) conf_pair<Q>(tp[P], ra, at[P]);
                // unconditional prefetch (the last one re-reads record TP_CHUNK - 1): no
                // branch in the loop body, 1.4 % faster than a guarded load
                load_src_pos(cb + min(s + 2, TP_CHUNK - 1) * TP_SRCW, ra);
#pragma unroll
                for (int P = 0; P < NP; ++P) conf_pair<Q>(tp[P], rb, at[P]);
                if ((s & 30) == 30) fold_energy<NP>(at, e64);
            }
        }
#pragma unroll
        for (int P = 0; P < NP; ++P) {
            const int64_t t0 = (int64_t)I * TP_SUPER + 2 * (pbase + 32 * P);
            const double ex = (double)e64[P].s.x - (double)e64[P].c.x, ey = (double)e64[P].s.y - (double)e64[P].c.y;
            if (ex != 0.0) atomicAdd(&A.acc[t0], ex);
            if (ey != 0.0) atomicAdd(&A.acc[t0 + 1], ey);
#pragma unroll
            for (int k = 1; k < TP_NACC; ++k) {
                const float sc = k >= 5 ? CONF_GX_SCALE : 1.0f;
                if (at[P].v[k].x != 0.f) atomicAdd(&A.acc[k * ntp + t0], (double)(sc * at[P].v[k].x));
                if (at[P].v[k].y != 0.f) atomicAdd(&A.acc[k * ntp + t0 + 1], (double)(sc * at[P].v[k].y));
            }
        }
    }
}

// FP64 reference form: one thread per target (library order), every confining
// triangle, FP64 arithmetic; same accumulator convention.
template <int Q>
__global__ void k_conf_f64(const double* __restrict__ x64, const double* __restrict__ nu64,
                           const double* __restrict__ w64, const int32_t* __restrict__ perm,
                           const double* __restrict__ y64, const double* __restrict__ a64, int64_t nt, int64_t nk,
                           int64_t ntp, double* __restrict__ acc) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int64_t T = perm[k];
    double xt[3], nt3[3];
    for (int a = 0; a < 3; ++a) {
        xt[a] = x64[a * nt + T];
        nt3[a] = nu64[a * nt + T];
    }
    const double wt = w64[T];
    double Ew = 0, U = 0, Gn[3] = {0, 0, 0}, Gx[3] = {0, 0, 0};
    for (int64_t K = 0; K < nk; ++K) {
        double d[3], r2 = 0, a = 0;
        for (int c = 0; c < 3; ++c) {
            d[c] = xt[c] - y64[c * nk + K];
            r2 += d[c] * d[c];
            a += nt3[c] * d[c];
        }
        const double inv = 1.0 / r2, al = a * inv, al2 = al * al;
        const double alq = Q == 6 ? al2 * al2 * al2 : al2 * al2 * al2 * al2;
        const double al5 = Q == 6 ? al2 * al2 * al : al2 * al2 * al2 * al;
        const double wts = 2.0 * wt * a64[K];  // (p/q) w_T a_K
        const double wi = wts * inv, A5 = wi * al5, kk = 2.0 * wi * alq;
        Ew += wts * alq;
        U += A5;
        for (int c = 0; c < 3; ++c) {
            Gn[c] += A5 * d[c];
            Gx[c] -= kk * d[c];
        }
    }
    acc[0 * ntp + k] = Ew;
    acc[1 * ntp + k] = U;
    for (int c = 0; c < 3; ++c) {
        acc[(2 + c) * ntp + k] = Gn[c];
        acc[(5 + c) * ntp + k] = Gx[c];
    }
}

DirectArgs make_args(tp_ctx* ctx, const tp_params* prm) {
    DirectArgs A;
    A.soa = ctx->soa;
    A.src = ctx->src;
    A.Fs = ctx->Fs;
    A.acc = ctx->acc;
    A.mlist = ctx->mlist;
    A.plist = ctx->plist;
    A.flist = ctx->flist;
    A.bmask = ctx->bmask;
    A.nsup = (int)ctx->nsup;
    A.nm = (int)ctx->n_masked;
    A.np = (int)ctx->n_precise;
    A.nf = (int)ctx->n_fast;
    A.work = ctx->work;
    A.ntp = ctx->ntp;
    A.edge_only = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    A.derr = ctx->derr;
    A.partial = ctx->red;
    return A;
}

}  // namespace

tp_status tp_launch_direct_grad(tp_ctx* ctx, const tp_params* prm) {
    TpRange nvtx_range("tp_launch_direct_grad");
    TP_TRY(tp_ensure_flagged(ctx));
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    DirectArgs A = make_args(ctx, prm);
    if (prm->q == 6) return launch_grad_q<6>(ctx, A);
    return launch_grad_q<8>(ctx, A);
}

tp_status tp_launch_conf_tri(tp_ctx* ctx) {
    k_conf_tri<<<(unsigned)((ctx->conf_nt + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->conf_V64, ctx->conf_F, ctx->conf_nt, ctx->conf_nv, ctx->conf_y64, ctx->conf_a64, ctx->derr);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

// Confinement accumulators of the evolving mesh's triangles (library order)
// into ctx->acc; the pair launch is bracketed by ev[0] / ev[1].
tp_status tp_launch_conf(tp_ctx* ctx, const tp_params* prm) {
    TpRange nvtx_range("tp_launch_conf");
    TP_TRY(tp_ensure_sorted(ctx));
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    if (prm->prec == TP_F64) {
        cudaEventRecord(ctx->ev[0], ctx->stream);
        const unsigned b = (unsigned)((ctx->nt + 127) / 128);
        if (prm->q == 6)
            k_conf_f64<6><<<b, 128, 0, ctx->stream>>>(ctx->x64, ctx->nu64, ctx->w64, ctx->perm, ctx->conf_y64,
                                                       ctx->conf_a64, ctx->nt, ctx->conf_nt, ctx->ntp, ctx->acc);
        else
            k_conf_f64<8><<<b, 128, 0, ctx->stream>>>(ctx->x64, ctx->nu64, ctx->w64, ctx->perm, ctx->conf_y64,
                                                       ctx->conf_a64, ctx->nt, ctx->conf_nt, ctx->ntp, ctx->acc);
        ++ctx->nlaunch;
        cudaEventRecord(ctx->ev[1], ctx->stream);
        TP_CU(cudaGetLastError());
        return TP_OK;
    }
    k_conf_records<<<(unsigned)((ctx->conf_ntp + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->conf_y64, ctx->conf_a64, ctx->center, ctx->conf_nt, ctx->conf_ntp, ctx->conf_src);
    ++ctx->nlaunch;
    constexpr int SMEM = 2 * CHUNK_BYTES + 64;
    // per-device attribute: set on the current device at every launch
    TP_CU(cudaFuncSetAttribute(k_conf_grad<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    TP_CU(cudaFuncSetAttribute(k_conf_grad<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    DirectArgs A = make_args(ctx, prm);
    A.src = ctx->conf_src;
    const int64_t nsupc = ctx->conf_ntp / TP_SUPER;
    A.np = (int)nsupc;
    A.nf = (int)(ctx->nsup * nsupc);
    TP_CU(cudaMemsetAsync(ctx->work, 0, sizeof(unsigned), ctx->stream));
    const int grid = (int)std::min<int64_t>(ctx->num_sms, ctx->nsup * nsupc);
    cudaEventRecord(ctx->ev[0], ctx->stream);
    if (prm->q == 6)
        k_conf_grad<6><<<grid, GradShape<false>::THREADS, SMEM, ctx->stream>>>(A);
    else
        k_conf_grad<8><<<grid, GradShape<false>::THREADS, SMEM, ctx->stream>>>(A);
    ++ctx->nlaunch;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_direct_energy(tp_ctx* ctx, const tp_params* prm, double* partials, int* nparts) {
    TpRange nvtx_range("tp_launch_direct_energy");
    TP_TRY(tp_ensure_flagged(ctx));
    DirectArgs A = make_args(ctx, prm);
    A.partial = partials;
    if (prm->q == 6) return launch_energy_q<6>(ctx, A, nparts);
    return launch_energy_q<8>(ctx, A, nparts);
}

// unordered pairs of the launch that ev[0] / ev[1] bracket in the direct gradient
int64_t tp_direct_timed_pairs(const tp_ctx* ctx) {
    return ctx->pairs_fast + (TP_FAST_ONLY ? 0 : ctx->pairs_precise);
}

tp_status tp_launch_direct_kahan(tp_ctx* ctx, const tp_params* prm) {
    TpRange nvtx_range("tp_launch_direct_kahan");
    TP_TRY(tp_ensure_sorted(ctx));
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    const int edge = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    const unsigned blocks = (unsigned)((ctx->nt + KAHAN_TILE - 1) / KAHAN_TILE);
    cudaEventRecord(ctx->ev[0], ctx->stream);
    if (prm->q == 6)
        k_pairs_kahan<6><<<blocks, KAHAN_TILE, 0, ctx->stream>>>(ctx->soa, ctx->Fs, ctx->nt, ctx->ntp, edge, ctx->acc);
    else
        k_pairs_kahan<8><<<blocks, KAHAN_TILE, 0, ctx->stream>>>(ctx->soa, ctx->Fs, ctx->nt, ctx->ntp, edge, ctx->acc);
    ++ctx->nlaunch;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_direct_f64(tp_ctx* ctx, const tp_params* prm, bool grad) {
    TpRange nvtx_range("tp_launch_direct_f64");
    (void)grad;
    TP_CU(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * TP_NACC * ctx->ntp, ctx->stream));
    const int edge = (prm->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    int blocks = (int)((ctx->nt + 127) / 128);
    cudaEventRecord(ctx->ev[0], ctx->stream);
    if (prm->q == 6)
        k_pairs_f64<6><<<blocks, 128, 0, ctx->stream>>>(ctx->x64, ctx->nu64, ctx->w64, ctx->F, ctx->perm, ctx->nt,
                                                        ctx->ntp, edge, ctx->acc, ctx->red);
    else
        k_pairs_f64<8><<<blocks, 128, 0, ctx->stream>>>(ctx->x64, ctx->nu64, ctx->w64, ctx->F, ctx->perm, ctx->nt,
                                                        ctx->ntp, edge, ctx->acc, ctx->red);
    ++ctx->nlaunch;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    TP_CU(cudaGetLastError());
    return TP_OK;
}
