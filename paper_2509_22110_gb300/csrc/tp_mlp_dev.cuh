// tp_mlp_dev.cuh - device pieces of the learned far-field correction shared
// by the training kernels (tp_mlp.cu) and the Barnes-Hut traversal
// (tp_bh.cu): network layout, BF16 tensor-core layers (mma.sync m16n8k16,
// FP32 accumulation), the tanh form of GELU and the pair features.
//
// Network: 24 -> 64 -> 64 -> 64 -> 7, y = W4 g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4,
// g(z) = z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2.  The FP32 master
// parameters use the packed layout W1[64][24] b1 W2[64][64] b2 W3[64][64] b3
// W4[7][64] b4; the BF16 copy used by the tensor cores pads W1 to [64][32]
// and W4 to [16][64] with zeros.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#define MLP_NI 24
#define MLP_NIP 32
#define MLP_NH 64
#define MLP_NO 7
#define MLP_NOP 8
#define MLP_OFF_W1 0
#define MLP_OFF_B1 (MLP_OFF_W1 + MLP_NH * MLP_NI)
#define MLP_OFF_W2 (MLP_OFF_B1 + MLP_NH)
#define MLP_OFF_B2 (MLP_OFF_W2 + MLP_NH * MLP_NH)
#define MLP_OFF_W3 (MLP_OFF_B2 + MLP_NH)
#define MLP_OFF_B3 (MLP_OFF_W3 + MLP_NH * MLP_NH)
#define MLP_OFF_W4 (MLP_OFF_B3 + MLP_NH)
#define MLP_OFF_B4 (MLP_OFF_W4 + MLP_NO * MLP_NH)
#define MLP_NPARAM (MLP_OFF_B4 + MLP_NO)
// BF16 weight block: W1p[64][32] W2[64][64] W3[64][64] W4p[16][64] (W4 rows 7..15
// zero: the backward pass reads W4 as a K = 16 operand)
#define MLPB_W1 0
#define MLPB_W2 (MLPB_W1 + MLP_NH * MLP_NIP)
#define MLPB_W3 (MLPB_W2 + MLP_NH * MLP_NH)
#define MLPB_W4 (MLPB_W3 + MLP_NH * MLP_NH)
#define MLPB_N (MLPB_W4 + 16 * MLP_NH)
// FP32 bias block: b1[64] b2[64] b3[64] b4p[8]
#define MLPF_B1 0
#define MLPF_B2 64
#define MLPF_B3 128
#define MLPF_B4 192
#define MLPF_N 200

// f32 node record for the features: A, X[3], nubar[3], M2/A (6), diag, pad
#define FEAT_REC 16

__device__ __forceinline__ float mlp_gelu(float z, float* dg) {
    const float c = 0.7978845608028654f, a = 0.044715f;
    const float u = c * (z + a * z * z * z);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    if (dg) *dg = 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * a * z * z);
    return 0.5f * z * (1.0f + t);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_bf16_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t*>(&v);
}

// D = A B + D for one m16n8k16 tile (A row-major 16x16, B column-major 16x8)
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Generic fragment loaders: element (r, c) of a matrix at base[r * rs + c * cs]
// (BF16 in shared memory).  A: rows m0..m0+15, cols k0..k0+15.
__device__ __forceinline__ void load_a(const __nv_bfloat16* base, int rs, int cs, int m0, int k0, uint32_t a[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = (lane & 3) * 2;
    const int r0 = m0 + g, r1 = m0 + g + 8, c0 = k0 + t, c1 = k0 + t + 8;
    a[0] = pack_bf16_raw(base[r0 * rs + c0 * cs], base[r0 * rs + (c0 + 1) * cs]);
    a[1] = pack_bf16_raw(base[r1 * rs + c0 * cs], base[r1 * rs + (c0 + 1) * cs]);
    a[2] = pack_bf16_raw(base[r0 * rs + c1 * cs], base[r0 * rs + (c1 + 1) * cs]);
    a[3] = pack_bf16_raw(base[r1 * rs + c1 * cs], base[r1 * rs + (c1 + 1) * cs]);
}
// B (k x n): element (k, n) at base[k * ks + n * ns]; k0..k0+15, n0..n0+7
__device__ __forceinline__ void load_b(const __nv_bfloat16* base, int ks, int ns, int k0, int n0, uint32_t b[2]) {
    const int lane = threadIdx.x & 31, n = n0 + (lane >> 2), k = k0 + (lane & 3) * 2;
    b[0] = pack_bf16_raw(base[k * ks + n * ns], base[(k + 1) * ks + n * ns]);
    b[1] = pack_bf16_raw(base[(k + 8) * ks + n * ns], base[(k + 9) * ks + n * ns]);
}
// C fragment coordinates of value v (0..3) of this lane: row, col within the 16x8 tile
__device__ __forceinline__ int frag_row(int v) { return ((threadIdx.x & 31) >> 2) + (v >= 2 ? 8 : 0); }
__device__ __forceinline__ int frag_col(int v) { return ((threadIdx.x & 31) & 3) * 2 + (v & 1); }

// Contiguous-layout fragment loads (32-bit shared-memory reads): A row-major
// with leading dimension lda (k contiguous), B stored as W[n][K] (k contiguous).
__device__ __forceinline__ void load_a_rm(const __nv_bfloat16* base, int lda, int m0, int k0, uint32_t a[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = (lane & 3) * 2;
    const __nv_bfloat16* p0 = base + (m0 + g) * lda + k0 + t;
    const __nv_bfloat16* p1 = p0 + 8 * lda;
    a[0] = *reinterpret_cast<const uint32_t*>(p0);
    a[1] = *reinterpret_cast<const uint32_t*>(p1);
    a[2] = *reinterpret_cast<const uint32_t*>(p0 + 8);
    a[3] = *reinterpret_cast<const uint32_t*>(p1 + 8);
}
__device__ __forceinline__ void load_b_nk(const __nv_bfloat16* W, int K, int k0, int n0, uint32_t b[2]) {
    const int lane = threadIdx.x & 31;
    const __nv_bfloat16* p = W + (n0 + (lane >> 2)) * K + k0 + (lane & 3) * 2;
    b[0] = *reinterpret_cast<const uint32_t*>(p);
    b[1] = *reinterpret_cast<const uint32_t*>(p + 8);
}

// One dense layer for a warp: out[16 x N] = in[16 x K] W^T + b over rows m0..m0+15.
// in: BF16 [rows][ld_in]; W: BF16 row-major [N][K] (element (k, n) = W[n * K + k]);
// the raw FP32 result z goes to zout[r * ld_z + c] (may be null) and act(z) as BF16
// to hout[r * ld_h + c] (may be null); act = 0 identity, 1 GELU.
template <int K, int N>
__device__ __forceinline__ void warp_dense(const __nv_bfloat16* in, int ld_in, const __nv_bfloat16* W,
                                           const float* bias, int m0, float* zout, int ld_z, __nv_bfloat16* hout,
                                           int ld_h, int act) {
    uint32_t af[K / 16][4];
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) load_a_rm(in, ld_in, m0, k0, af[k0 / 16]);
#pragma unroll
    for (int n0 = 0; n0 < N; n0 += 8) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += 16) {
            uint32_t b[2];
            load_b_nk(W, K, k0, n0, b);
            mma_bf16(d, af[k0 / 16], b);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = m0 + frag_row(v), c = n0 + frag_col(v);
            const float z = d[v] + bias[c];
            if (zout) zout[r * ld_z + c] = z;
            if (hout) hout[r * ld_h + c] = __float2bfloat16_rn(act ? mlp_gelu(z, nullptr) : z);
        }
    }
}

// Network forward for 16 rows (m0..m0+15) of X (BF16 [rows][32], normalised
// features, zero-padded).  ha/hb: BF16 scratch [rows][64] (ping-pong);
// z1..z3: optional FP32 pre-activations [rows][64]; y: FP32 [rows][8].
__device__ __forceinline__ void warp_mlp_forward(const __nv_bfloat16* wb, const float* bias, const __nv_bfloat16* X,
                                                 __nv_bfloat16* ha, __nv_bfloat16* hb, __nv_bfloat16* hc, float* z1,
                                                 float* z2, float* z3, float* y, int m0) {
    warp_dense<MLP_NIP, MLP_NH>(X, MLP_NIP, wb + MLPB_W1, bias + MLPF_B1, m0, z1, MLP_NH, ha, MLP_NH, 1);
    __syncwarp();
    warp_dense<MLP_NH, MLP_NH>(ha, MLP_NH, wb + MLPB_W2, bias + MLPF_B2, m0, z2, MLP_NH, hb, MLP_NH, 1);
    __syncwarp();
    warp_dense<MLP_NH, MLP_NH>(hb, MLP_NH, wb + MLPB_W3, bias + MLPF_B3, m0, z3, MLP_NH, hc, MLP_NH, 1);
    __syncwarp();
    warp_dense<MLP_NH, MLP_NOP>(hc, MLP_NH, wb + MLPB_W4, bias + MLPF_B4, m0, y, MLP_NOP, nullptr, 0, 0);
    __syncwarp();
}

// Inference keeps the hidden activations in registers: the accumulator
// fragment of a 16 x 8 output tile holds (row g, cols 2t, 2t+1) and (row g+8,
// same cols) per lane (g = lane/4, t = lane%4), exactly the halves of the A
// fragment of the next layer's 16 x 16 k-tile, so GELU and the BF16 packing
// happen in registers and only the input X and the output y touch memory.
// Fragment-ordered copy of the BF16 weights for the inference kernels: for
// each layer, n-tile j and k-tile kk, lane l holds the two 32-bit B-fragment
// registers of mma.m16n8k16 (W[n][k..k+1] and W[n][k+8..k+9], n = 8j + l/4,
// k = 16kk + 2(l%4)) side by side, so a fragment is one conflict-free 64-bit
// shared-memory load (the row-major copy puts the 32 lanes in 4 banks).
#define MLPW_W1 0                       // [8 j][2 kk][32] uint2 (K = 32, padded)
#define MLPW_W2 (MLPW_W1 + 8 * 2 * 32)  // [8][4][32]
#define MLPW_W3 (MLPW_W2 + 8 * 4 * 32)  // [8][4][32]
#define MLPW_W4 (MLPW_W3 + 8 * 4 * 32)  // [1][4][32]
#define MLPW_N (MLPW_W4 + 1 * 4 * 32)   // 2688 uint2 = 21 KB

// Build the fragment-ordered copy wf[MLPW_N] from the row-major BF16 block wb
// (threads t of n cooperate).
__device__ __forceinline__ void mlp_frag_weights(const __nv_bfloat16* wb, uint2* wf, int t, int n) {
    for (int i = t; i < MLPW_N; i += n) {
        int base, K, r;
        const __nv_bfloat16* W;
        if (i < MLPW_W2) {
            base = MLPW_W1; K = MLP_NIP; W = wb + MLPB_W1;
        } else if (i < MLPW_W3) {
            base = MLPW_W2; K = MLP_NH; W = wb + MLPB_W2;
        } else if (i < MLPW_W4) {
            base = MLPW_W3; K = MLP_NH; W = wb + MLPB_W3;
        } else {
            base = MLPW_W4; K = MLP_NH; W = wb + MLPB_W4;
        }
        r = i - base;
        const int lane = r & 31, kk = (r >> 5) % (K / 16), j = (r >> 5) / (K / 16);
        const int n0 = 8 * j + (lane >> 2), k = 16 * kk + 2 * (lane & 3);
        const __nv_bfloat16* p = W + n0 * K + k;
        wf[i] = make_uint2(pack_bf16_raw(p[0], p[1]), pack_bf16_raw(p[8], p[9]));
    }
}

// One layer for M 16-row tiles with activations in registers: the B fragment
// of each (n-tile, k-tile) is loaded once and used by every row tile.
template <int KT, int NT, int M>
__device__ __forceinline__ void dense_frag(const uint32_t (&a)[M][KT][4], const uint2* wf, const float* bias,
                                           uint32_t (&h)[M][NT / 2][4]) {
    const int lane = threadIdx.x & 31, t2 = (lane & 3) * 2;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        uint32_t b[KT][2];
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            const uint2 v = wf[(j * KT + kk) * 32 + lane];
            b[kk][0] = v.x;
            b[kk][1] = v.y;
        }
        const float b0 = bias[8 * j + t2], b1 = bias[8 * j + t2 + 1];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) mma_bf16(d, a[m][kk], b[kk]);
            h[m][j >> 1][(j & 1) * 2 + 0] = pack_bf16(mlp_gelu(d[0] + b0, nullptr), mlp_gelu(d[1] + b1, nullptr));
            h[m][j >> 1][(j & 1) * 2 + 1] = pack_bf16(mlp_gelu(d[2] + b0, nullptr), mlp_gelu(d[3] + b1, nullptr));
        }
    }
}

// Network forward for 32 rows (two 16-row tiles) of X (BF16, row-major with
// leading dimension 32, any memory space; rows row0..row0+31 must exist):
// y (FP32 [32][8] in shared memory, row 0 = row0, column 7 unused).  Same
// arithmetic as warp_mlp_forward (BF16 operands and activations, FP32
// accumulation).
__device__ __forceinline__ void warp_mlp_rows32(const uint2* wf, const float* bias, const __nv_bfloat16* X,
                                                int64_t row0, float* y) {
    uint32_t a1[2][2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        load_a_rm(X + row0 * MLP_NIP, MLP_NIP, 16 * m, 0, a1[m][0]);
        load_a_rm(X + row0 * MLP_NIP, MLP_NIP, 16 * m, 16, a1[m][1]);
    }
    uint32_t h1[2][4][4], h2[2][4][4];
    dense_frag<2, 8, 2>(a1, wf + MLPW_W1, bias + MLPF_B1, h1);
    dense_frag<4, 8, 2>(h1, wf + MLPW_W2, bias + MLPF_B2, h2);
    dense_frag<4, 8, 2>(h2, wf + MLPW_W3, bias + MLPF_B3, h1);
    const int lane = threadIdx.x & 31;
    uint32_t b[4][2];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint2 v = wf[MLPW_W4 + kk * 32 + lane];
        b[kk][0] = v.x;
        b[kk][1] = v.y;
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma_bf16(d, h1[m][kk], b[kk]);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = 16 * m + frag_row(v), c = frag_col(v);
            y[r * MLP_NOP + c] = d[v] + bias[MLPF_B4 + c];
        }
    }
}

// ---------------------------------------------------------------- features
// 24 rotation-invariant features of (leaf L, cluster C) from their f32 node
// records (A, X[3], nubar[3], M2/A[6], diag):
//   0 log(r/sqrt(A_C)), 1 log(r/sqrt(A_L)), 2 diag_C/r, 3 diag_L/r,
//   4-6 nubar_L in the pair frame, 7-8 nubar_C . e1, e2,
//   9-14 M2_C/A_C in the frame, 15-20 M2_L/A_L in the frame,
//   21 |nubar_L|, 22 |nubar_C|, 23 log(A_C/A_L);
// frame: e1 = (X_C - X_L)/r, e2 along the part of nubar_C orthogonal to e1
// (or of the coordinate axis least aligned with e1), e3 = e1 x e2.
// Single-precision intrinsics throughout (reciprocal square roots, fast
// logarithms): the features are rounded to BF16 after normalisation, far
// coarser than their error.
__device__ __forceinline__ void moment_frame(const float* m6, const float e[3][3], float* out) {
    const float M[3][3] = {{m6[0], m6[1], m6[2]}, {m6[1], m6[3], m6[4]}, {m6[2], m6[4], m6[5]}};
    float Me[3][3];  // Me[j] = M e_j
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) Me[j][a] = M[a][0] * e[j][0] + M[a][1] * e[j][1] + M[a][2] * e[j][2];
    int o = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) out[o++] = e[i][0] * Me[j][0] + e[i][1] * Me[j][1] + e[i][2] * Me[j][2];
}

__device__ __forceinline__ void far_features(const float* L, const float* C, float* f) {
    float D[3], e[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) D[a] = C[1 + a] - L[1 + a];
    const float r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const float rinv = rsqrtf(r2), r = r2 * rinv;
#pragma unroll
    for (int a = 0; a < 3; ++a) e[0][a] = D[a] * rinv;
    float u[3] = {C[4], C[5], C[6]};
    float p = u[0] * e[0][0] + u[1] * e[0][1] + u[2] * e[0][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] -= p * e[0][a];
    float un2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (un2 < 1e-12f) {  // |u| < 1e-6: use the coordinate axis least aligned with e1
        int k = 0;
        float ek = e[0][0];  // selected without indexing, so e stays in registers
        if (fabsf(e[0][1]) < fabsf(ek)) {
            k = 1;
            ek = e[0][1];
        }
        if (fabsf(e[0][2]) < fabsf(ek)) {
            k = 2;
            ek = e[0][2];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = (a == k ? 1.f : 0.f) - ek * e[0][a];
        un2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    }
    const float uinv = rsqrtf(un2);
#pragma unroll
    for (int a = 0; a < 3; ++a) e[1][a] = u[a] * uinv;
    e[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    e[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    e[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    const float lr = __logf(r), lc = __logf(C[0]), ll = __logf(L[0]);
    f[0] = lr - 0.5f * lc;
    f[1] = lr - 0.5f * ll;
    f[2] = C[13] * rinv;
    f[3] = L[13] * rinv;
#pragma unroll
    for (int i = 0; i < 3; ++i) f[4 + i] = L[4] * e[i][0] + L[5] * e[i][1] + L[6] * e[i][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) f[7 + i] = C[4] * e[i][0] + C[5] * e[i][1] + C[6] * e[i][2];
    moment_frame(C + 7, e, f + 9);
    moment_frame(L + 7, e, f + 15);
    f[21] = sqrtf(L[4] * L[4] + L[5] * L[5] + L[6] * L[6]);
    f[22] = sqrtf(C[4] * C[4] + C[5] * C[5] + C[6] * C[6]);
    f[23] = lc - ll;
}

// Network input row of one listed (leaf, cluster) pair: the 24 features of
// far_features normalised with the fitted mean and 1/std (norm[0..23],
// norm[24..47]) and rounded to BF16 pairs in pk[0..11], pk[12..14] zero, and
// in the high half of pk[15] (column 31) 1 when every raw feature lies in the
// admitted range [norm[48 + i], norm[72 + i]], else 0 (a zero-weight column).
__device__ __forceinline__ void feature_row_bf16(const float* fl, const float* cr, const float* norm,
                                                 uint32_t (&pk)[16]) {
    float f[MLP_NI];
    far_features(fl, cr, f);
    int in_dist = 1;
#pragma unroll
    for (int c = 0; c < MLP_NI; c += 2) {
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(f[c + h] >= norm[2 * MLP_NI + c + h] && f[c + h] <= norm[3 * MLP_NI + c + h])) in_dist = 0;
            v[h] = (f[c + h] - norm[c + h]) * norm[MLP_NI + c + h];
        }
        pk[c / 2] = pack_bf16(v[0], v[1]);
    }
#pragma unroll
    for (int c = MLP_NI / 2; c < 15; ++c) pk[c] = 0u;
    pk[15] = pack_bf16(0.f, in_dist ? 1.f : 0.f);
}
