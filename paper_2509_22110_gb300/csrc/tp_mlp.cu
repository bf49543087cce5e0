// tp_mlp.cu - learned correction of the Barnes-Hut far field: training
// data, training (forward, backward, AdamW) and model files.
//
// The paper clusters the inner integral with averages over a patch
// (Sec. 3.2); the monopole far term of this library (area, area-weighted
// centroid, area-averaged normal) is exact for a single-triangle cluster and
// otherwise biased.  A small network corrects it per (target leaf L,
// cluster C) pair: from 24 rotation-invariant features of the two clusters'
// moments it predicts 7 log-factors, one per channel of the far term
//   0 e_TC energy (al^q part), 1 e_CT energy (be^q part), 2 U (own-normal
//   force coefficient), 3 Gn (normal derivative), 4 the nubar_C force term,
//   5 and 6 the al^q and be^q parts of the d force term,
// each the log of (exact member sum) / (monopole) summed over the targets of
// L.  Training data come from the direct sums over the members of sampled
// admissible pairs (the direct sum generates its own labels).  Weights are
// BF16 on the tensor cores (mma.sync m16n8k16) with FP32 accumulation and
// FP32 master copies updated by AdamW.  Pairs whose features fall outside
// the training ranges keep the plain monopole (the Barnes-Hut fallback).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "tp_internal.cuh"
#include "tp_mlp_dev.cuh"

struct tp_mlp_model {
    float* master = nullptr;  // [MLP_NPARAM] FP32 parameters
    float* am = nullptr;      // AdamW first moments
    float* av = nullptr;      // AdamW second moments
    float* grad = nullptr;    // [MLP_NPARAM]
    __nv_bfloat16* wb = nullptr;  // [MLPB_N] BF16 weights (padded)
    float* bias = nullptr;    // [MLPF_N]
    float* norm = nullptr;    // [4][24]: mean, std, lo, hi of the raw features
    double* red = nullptr;    // [4] loss / mask-sum scratch
    int step = 0;
    bool have_norm = false;
    float theta = 0.25f;
    // dataset (raw features, labels, masks) and sampled pairs
    float* dfeat = nullptr;   // [cap][24]
    float* dlab = nullptr;    // [cap][8]
    float* dmask = nullptr;   // [cap][8]
    int2* dpairs = nullptr;   // [cap] (leaf index, node) of the last sampling pass
    int32_t* dcount_d = nullptr;
    int64_t dcount = 0, dcap = 0;
};

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// FP32 feature record of every node the traversal can reach: A, X[3],
// nubar[3], M2/A (6), diag
__global__ void __launch_bounds__(TP_NODE_THREADS) k_node_feat(const double* __restrict__ mom,
                                                               const double* __restrict__ box,
                                                               const int32_t* __restrict__ parent,
                                                               const int32_t* __restrict__ first,
                                                               const int32_t* __restrict__ last, int leaf_size,
                                                               int64_t nn, float* __restrict__ rec) {
    __shared__ int32_t list[TP_NODE_BLK];
    __shared__ int cnt;
    const int n = tp_reachable_list(parent, first, last, leaf_size, blockIdx.x * (int64_t)TP_NODE_BLK, nn, list,
                                    &cnt);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t v = list[i];
        const double* m = mom + 13 * v;
        const double* b = box + 6 * v;
        float* r = rec + FEAT_REC * v;
        const double A = m[0];
        r[0] = (float)A;
        for (int a = 0; a < 3; ++a) {
            r[1 + a] = (float)(m[1 + a] / A);
            r[4 + a] = (float)(m[4 + a] / A);
        }
        for (int c = 0; c < 6; ++c) r[7 + c] = (float)(m[7 + c] / A);
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) d2 += (b[3 + a] - b[a]) * (b[3 + a] - b[a]);
        r[13] = (float)sqrt(d2);
        r[14] = r[15] = 0.f;
    }
}

// Features and labels of sampled (leaf, cluster) pairs; one block per pair.
// Channel sums follow the oracle's or_far_channels: the monopole in FP64
// from the cluster moments, the exact member sums with FP32 pair terms and
// FP64 accumulation.
__global__ void __launch_bounds__(128) k_far_label(const int2* __restrict__ pairs, int64_t n0, int64_t npairs,
                                                   const int32_t* __restrict__ leaves, const int32_t* __restrict__ first,
                                                   const int32_t* __restrict__ last, const double* __restrict__ mom,
                                                   const float* __restrict__ frec, const float* __restrict__ soa,
                                                   int64_t ntp, const double* __restrict__ center, int q,
                                                   float* __restrict__ feat, float* __restrict__ lab,
                                                   float* __restrict__ mask) {
    const int64_t i = blockIdx.x;
    if (i >= npairs) return;
    const int2 pr = pairs[i];
    const int64_t L = leaves[pr.x], C = pr.y;
    const int64_t fL = first[L], nl = last[L] - first[L] + 1;
    const int64_t fC = first[C], nc = last[C] - first[C] + 1;
    __shared__ float s_t[32][12];    // per target: x hi[3], lo[3], nu[3], w~, |d| to X_C, pad
    __shared__ float s_dh[32][3];    // unit d_TC
    __shared__ double s_red[7][128];
    __shared__ double s_mono[7];
    const double* mc = mom + 13 * C;
    const double A = mc[0];
    double XC[3], nb[3];
    for (int a = 0; a < 3; ++a) {
        XC[a] = mc[1 + a] / A - center[a];
        nb[a] = mc[4 + a] / A;
    }
    const double nbn = sqrt(nb[0] * nb[0] + nb[1] * nb[1] + nb[2] * nb[2]);
    const int t = threadIdx.x;
    if (t < 7) s_mono[t] = 0.0;
    __syncthreads();
    if (t < nl) {
        const int64_t k = fL + t;
        for (int a = 0; a < 3; ++a) {
            s_t[t][a] = soa[a * ntp + k];
            s_t[t][3 + a] = soa[(3 + a) * ntp + k];
            s_t[t][6 + a] = soa[(6 + a) * ntp + k];
        }
        s_t[t][9] = soa[9 * ntp + k];
        // monopole channels (FP64)
        double d[3], r2 = 0.0, al = 0.0, be = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = ((double)s_t[t][a] + (double)s_t[t][3 + a]) - XC[a];
            r2 += d[a] * d[a];
        }
        for (int a = 0; a < 3; ++a) {
            al += (double)s_t[t][6 + a] * d[a];
            be += nb[a] * d[a];
        }
        const double inv = 1.0 / r2, rn = sqrt(r2);
        al *= inv;
        be *= inv;
        const double wts = (double)s_t[t][9] * 1.4142135623730951 * A;  // (p/q) w_T A_C, p = 2q
        double al5 = 1.0, be5 = 1.0;
        for (int e = 0; e < q - 1; ++e) {
            al5 *= al;
            be5 *= be;
        }
        const double alq = al5 * al, beq = be5 * be;
        const double lam = 2.0;
        atomicAdd(&s_mono[0], wts * alq);
        atomicAdd(&s_mono[1], wts * beq);
        atomicAdd(&s_mono[2], wts * inv * al5);
        atomicAdd(&s_mono[3], wts * inv * al5 * rn);
        atomicAdd(&s_mono[4], wts * inv * be5 * nbn);
        atomicAdd(&s_mono[5], lam * wts * inv * alq * rn);
        atomicAdd(&s_mono[6], lam * wts * inv * beq * rn);
        for (int a = 0; a < 3; ++a) s_dh[t][a] = (float)(d[a] / rn);
    }
    __syncthreads();
    // exact member sums
    float acc[7] = {0, 0, 0, 0, 0, 0, 0};
    double accd[7] = {0, 0, 0, 0, 0, 0, 0};
    const float nbu[3] = {(float)(nb[0] / nbn), (float)(nb[1] / nbn), (float)(nb[2] / nbn)};
    int cnt = 0;
    for (int64_t j = t; j < nc; j += blockDim.x) {
        const int64_t s = fC + j;
        float sh[3], sl[3], sn[3];
        for (int a = 0; a < 3; ++a) {
            sh[a] = soa[a * ntp + s];
            sl[a] = soa[(3 + a) * ntp + s];
            sn[a] = soa[(6 + a) * ntp + s];
        }
        const float sw = soa[9 * ntp + s];
        const float pn = sn[0] * nbu[0] + sn[1] * nbu[1] + sn[2] * nbu[2];
        for (int64_t i2 = 0; i2 < nl; ++i2) {
            float d[3];
            for (int a = 0; a < 3; ++a) d[a] = (s_t[i2][a] - sh[a]) + (s_t[i2][3 + a] - sl[a]);
            const float inv = 1.0f / (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const float al = (s_t[i2][6] * d[0] + s_t[i2][7] * d[1] + s_t[i2][8] * d[2]) * inv;
            const float be = (sn[0] * d[0] + sn[1] * d[1] + sn[2] * d[2]) * inv;
            const float wt = s_t[i2][9] * sw;
            float al5 = 1.f, be5 = 1.f;
            for (int e = 0; e < q - 1; ++e) {
                al5 *= al;
                be5 *= be;
            }
            const float alq = al5 * al, beq = be5 * be;
            const float pd = d[0] * s_dh[i2][0] + d[1] * s_dh[i2][1] + d[2] * s_dh[i2][2];
            acc[0] += wt * alq;
            acc[1] += wt * beq;
            acc[2] += wt * inv * al5;
            acc[3] += wt * inv * al5 * pd;
            acc[4] += wt * inv * be5 * pn;
            acc[5] += 2.0f * wt * inv * alq * pd;
            acc[6] += 2.0f * wt * inv * beq * pd;
        }
        if (++cnt == 16) {
            for (int c = 0; c < 7; ++c) {
                accd[c] += acc[c];
                acc[c] = 0.f;
            }
            cnt = 0;
        }
    }
    for (int c = 0; c < 7; ++c) s_red[c][t] = accd[c] + acc[c];
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (t < o)
            for (int c = 0; c < 7; ++c) s_red[c][t] += s_red[c][t + o];
        __syncthreads();
    }
    if (t < 8) {
        float lv = 0.f, mv = 0.f;
        if (t < 7) {
            const double ex = s_red[t][0], mo = s_mono[t];
            const double ratio = ex / mo;
            if (mo != 0.0 && ratio > 0.0 && isfinite(ratio)) {
                lv = (float)fmin(4.0, fmax(-4.0, log(ratio)));
                mv = 1.f;
            }
        }
        lab[(n0 + i) * 8 + t] = lv;
        mask[(n0 + i) * 8 + t] = mv;
    }
    if (t == 0) far_features(frec + FEAT_REC * L, frec + FEAT_REC * C, feat + (n0 + i) * MLP_NI);
}

// per-feature mean, std, min, max over the dataset (one block per feature)
__global__ void k_feat_stats(const float* __restrict__ feat, int64_t n, float* __restrict__ norm) {
    __shared__ double s1[256], s2[256];
    __shared__ float smin[256], smax[256];
    const int f = blockIdx.x;
    double a = 0.0, b = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float v = feat[i * MLP_NI + f];
        a += v;
        b += (double)v * v;
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double var = fmax(s2[0] / (double)n - mean * mean, 0.0);
        norm[f] = (float)mean;
        norm[MLP_NI + f] = (float)fmax(sqrt(var), 1e-6);
        norm[2 * MLP_NI + f] = smin[0];
        norm[3 * MLP_NI + f] = smax[0];
    }
}

// BF16 weights and FP32 biases from the master parameters
__global__ void k_pack_weights(const float* __restrict__ P, __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float v = P[i];
    if (i < MLP_OFF_B1) {
        const int o = i / MLP_NI, c = i % MLP_NI;
        wb[MLPB_W1 + o * MLP_NIP + c] = __float2bfloat16_rn(v);
    } else if (i < MLP_OFF_W2) {
        bias[MLPF_B1 + (i - MLP_OFF_B1)] = v;
    } else if (i < MLP_OFF_B2) {
        wb[MLPB_W2 + (i - MLP_OFF_W2)] = __float2bfloat16_rn(v);
    } else if (i < MLP_OFF_W3) {
        bias[MLPF_B2 + (i - MLP_OFF_B2)] = v;
    } else if (i < MLP_OFF_B3) {
        wb[MLPB_W3 + (i - MLP_OFF_W3)] = __float2bfloat16_rn(v);
    } else if (i < MLP_OFF_W4) {
        bias[MLPF_B3 + (i - MLP_OFF_B3)] = v;
    } else if (i < MLP_OFF_B4) {
        wb[MLPB_W4 + (i - MLP_OFF_W4)] = __float2bfloat16_rn(v);
    } else {
        bias[MLPF_B4 + (i - MLP_OFF_B4)] = v;
    }
}

__global__ void k_adamw(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[i] = w[i] - lr * (mh / (sqrtf(vh) + eps)) - lr * wd * w[i];
}

// Batch of 64 samples per block (4 warps x 16 rows): forward, masked
// mean-square loss, backward, parameter gradients summed into `grad`.
// Rows are either dataset indices drawn by a counter-based hash or, with
// `rows` non-null, given explicitly (tests); X may also be given directly.
constexpr int TB = 64;
struct TrainSmem {
    __nv_bfloat16 wb[MLPB_N];
    float bias[MLPF_N];
    __nv_bfloat16 X[TB][MLP_NIP];
    float z1[TB][MLP_NH], z2[TB][MLP_NH], z3[TB][MLP_NH];  // pre-activations, then their gradients
    __nv_bfloat16 h1[TB][MLP_NH], h2[TB][MLP_NH], h3[TB][MLP_NH];
    __nv_bfloat16 dz[TB][MLP_NH];  // BF16 copy of the current layer gradient
    float y[TB][MLP_NOP];
    __nv_bfloat16 dy[TB][16];
    float tgt[TB][MLP_NOP], msk[TB][MLP_NOP];
    float g[MLP_NPARAM];
    double lsum[4];
};

// dst[o][c] += sum over the warp's 16 rows of A[r][o] * B[r][c] (outer-product
// accumulation on the tensor cores: M = o, N = c, K = rows), A and B BF16
// [rows][lda]/[rows][ldb]; dst FP32 row-major with leading dimension ldd.
template <int MO, int NC>
__device__ __forceinline__ void warp_wgrad(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int r0,
                                           float* dst, int ldd, int mvalid, int nvalid) {
#pragma unroll
    for (int m0 = 0; m0 < MO; m0 += 16)
#pragma unroll
        for (int n0 = 0; n0 < NC; n0 += 8) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t a[4], b[2];
            load_a(A, 1, lda, m0, r0, a);  // element (m = o, k = r) at A[r * lda + o]
            load_b(B, ldb, 1, r0, n0, b);  // element (k = r, n = c) at B[r * ldb + c]
            mma_bf16(d, a, b);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int o = m0 + frag_row(v), c = n0 + frag_col(v);
                if (o < mvalid && c < nvalid) atomicAdd(&dst[o * ldd + c], d[v]);
            }
        }
}

// dh[r][c] = sum_o G[r][o] W[o][c] for the warp's rows; G BF16 [rows][ldg] (K = KO),
// W BF16 row-major [KO][NC]; then the gradient through GELU: dz = dh g'(z),
// written over z (FP32) and as BF16 to dzb.
template <int KO, int NC>
__device__ __forceinline__ void warp_back(const __nv_bfloat16* G, int ldg, const __nv_bfloat16* W, int r0, float* z,
                                          __nv_bfloat16* dzb) {
#pragma unroll
    for (int n0 = 0; n0 < NC; n0 += 8) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k0 = 0; k0 < KO; k0 += 16) {
            uint32_t a[4], b[2];
            load_a(G, ldg, 1, r0, k0, a);
            load_b(W, NC, 1, k0, n0, b);  // element (k = o, n = c) at W[o * NC + c]
            mma_bf16(d, a, b);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + frag_row(v), c = n0 + frag_col(v);
            float dg;
            mlp_gelu(z[r * MLP_NH + c], &dg);
            const float dzv = d[v] * dg;
            z[r * MLP_NH + c] = dzv;
            dzb[r * MLP_NH + c] = __float2bfloat16_rn(dzv);
        }
    }
}

__global__ void __launch_bounds__(128) k_mlp_train(const __nv_bfloat16* __restrict__ wb_g,
                                                   const float* __restrict__ bias_g, const float* __restrict__ norm,
                                                   const float* __restrict__ feat, const float* __restrict__ lab,
                                                   const float* __restrict__ mask, int64_t ndata, int64_t batch,
                                                   uint64_t seed, const float* __restrict__ Xin, int xin_normalised,
                                                   float inv_msum, float* __restrict__ grad, double* __restrict__ loss,
                                                   float* __restrict__ yout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < MLPB_N; i += blockDim.x) S.wb[i] = wb_g[i];
    for (int i = tid; i < MLPF_N; i += blockDim.x) S.bias[i] = bias_g[i];
    for (int i = tid; i < MLP_NPARAM; i += blockDim.x) S.g[i] = 0.f;
    if (tid < 4) S.lsum[tid] = 0.0;
    // rows of this block
    for (int e = tid; e < TB * MLP_NIP; e += blockDim.x) {
        const int r = e / MLP_NIP, c = e % MLP_NIP;
        const int64_t gi = (int64_t)blockIdx.x * TB + r;
        float v = 0.f;
        if (gi < batch && c < MLP_NI) {
            if (Xin) {
                v = Xin[gi * MLP_NI + c];
                if (!xin_normalised) v = (v - norm[c]) / norm[MLP_NI + c];
            } else {
                const int64_t di = (int64_t)(splitmix64(seed ^ (uint64_t)gi * 0x9e3779b97f4a7c15ull) % (uint64_t)ndata);
                v = (feat[di * MLP_NI + c] - norm[c]) / norm[MLP_NI + c];
            }
        }
        S.X[r][c] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < TB * MLP_NOP; e += blockDim.x) {
        const int r = e / MLP_NOP, c = e % MLP_NOP;
        const int64_t gi = (int64_t)blockIdx.x * TB + r;
        float tv = 0.f, mv = 0.f;
        if (gi < batch && c < MLP_NO) {
            const int64_t di = Xin ? gi : (int64_t)(splitmix64(seed ^ (uint64_t)gi * 0x9e3779b97f4a7c15ull) % (uint64_t)ndata);
            tv = lab[di * 8 + c];
            mv = mask[di * 8 + c];
        }
        S.tgt[r][c] = tv;
        S.msk[r][c] = mv;
    }
    __syncthreads();
    const int r0 = warp * 16;
    warp_mlp_forward(S.wb, S.bias, &S.X[0][0], &S.h1[0][0], &S.h2[0][0], &S.h3[0][0], &S.z1[0][0], &S.z2[0][0],
                     &S.z3[0][0], &S.y[0][0], r0);
    // loss and dL/dy (BF16, K padded to 16)
    {
        const int lane = tid & 31;
        double lw = 0.0;
        for (int e = lane; e < 16 * 16; e += 32) {
            const int r = r0 + e / 16, c = e % 16;
            float g = 0.f;
            if (c < MLP_NOP) {
                const float res = S.y[r][c] - S.tgt[r][c];
                g = 2.f * S.msk[r][c] * res * inv_msum;
                lw += (double)(S.msk[r][c] * res * res);
                if (yout) {
                    const int64_t gi = (int64_t)blockIdx.x * TB + r;
                    if (gi < batch && c < MLP_NO) yout[gi * MLP_NO + c] = S.y[r][c];
                }
            }
            S.dy[r][c] = __float2bfloat16_rn(g);
        }
        for (int o = 16; o > 0; o >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, o);
        if (lane == 0) atomicAdd(&S.lsum[0], lw);
    }
    __syncwarp();
    // output layer: dW4 = dy^T h3, db4 = sum dy, then dz3 = (dy W4) g'(z3)
    warp_wgrad<16, 64>(&S.dy[0][0], 16, &S.h3[0][0], MLP_NH, r0, S.g + MLP_OFF_W4, MLP_NH, MLP_NO, MLP_NH);
    if ((tid & 31) < MLP_NO) {
        float s = 0.f;
        for (int r = r0; r < r0 + 16; ++r) s += __bfloat162float(S.dy[r][tid & 31]);
        atomicAdd(&S.g[MLP_OFF_B4 + (tid & 31)], s);
    }
    warp_back<16, 64>(&S.dy[0][0], 16, S.wb + MLPB_W4, r0, &S.z3[0][0], &S.dz[0][0]);
    __syncwarp();
    // layer 3
    warp_wgrad<64, 64>(&S.dz[0][0], MLP_NH, &S.h2[0][0], MLP_NH, r0, S.g + MLP_OFF_W3, MLP_NH, MLP_NH, MLP_NH);
    for (int c = tid & 31; c < MLP_NH; c += 32) {
        float s = 0.f;
        for (int r = r0; r < r0 + 16; ++r) s += S.z3[r][c];
        atomicAdd(&S.g[MLP_OFF_B3 + c], s);
    }
    __syncwarp();
    warp_back<64, 64>(&S.dz[0][0], MLP_NH, S.wb + MLPB_W3, r0, &S.z2[0][0], &S.h3[0][0]);  // dz2 -> h3 buffer
    __syncwarp();
    // layer 2
    warp_wgrad<64, 64>(&S.h3[0][0], MLP_NH, &S.h1[0][0], MLP_NH, r0, S.g + MLP_OFF_W2, MLP_NH, MLP_NH, MLP_NH);
    for (int c = tid & 31; c < MLP_NH; c += 32) {
        float s = 0.f;
        for (int r = r0; r < r0 + 16; ++r) s += S.z2[r][c];
        atomicAdd(&S.g[MLP_OFF_B2 + c], s);
    }
    __syncwarp();
    warp_back<64, 64>(&S.h3[0][0], MLP_NH, S.wb + MLPB_W2, r0, &S.z1[0][0], &S.dz[0][0]);  // dz1 -> dz
    __syncwarp();
    // layer 1
    warp_wgrad<64, 32>(&S.dz[0][0], MLP_NH, &S.X[0][0], MLP_NIP, r0, S.g + MLP_OFF_W1, MLP_NI, MLP_NH, MLP_NI);
    for (int c = tid & 31; c < MLP_NH; c += 32) {
        float s = 0.f;
        for (int r = r0; r < r0 + 16; ++r) s += S.z1[r][c];
        atomicAdd(&S.g[MLP_OFF_B1 + c], s);
    }
    __syncthreads();
    for (int i = tid; i < MLP_NPARAM; i += blockDim.x)
        if (S.g[i] != 0.f) atomicAdd(&grad[i], S.g[i]);
    if (tid == 0) atomicAdd(&loss[0], S.lsum[0]);
}

// BF16 network rows [n][32] from host features [n][24] (normalised here
// unless already normalised); column 31 (the training-range flag) set to 1.
__global__ void k_rows_bf16(const float* __restrict__ X, int64_t n, int normalised, const float* __restrict__ norm,
                            __nv_bfloat16* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * MLP_NIP) return;
    const int64_t r = i / MLP_NIP;
    const int c = (int)(i % MLP_NIP);
    float v = 0.f;
    if (c < MLP_NI) {
        v = X[r * MLP_NI + c];
        if (!normalised) v = (v - norm[c]) / norm[MLP_NI + c];
    } else if (c == MLP_NIP - 1) {
        v = 1.f;
    }
    out[i] = __float2bfloat16_rn(v);
}

// Forward pass only, with the arithmetic of the learned Barnes-Hut
// correction's register-resident mma.sync path (warp_mlp_rows32): 4 warps x
// 32 rows per block.
__global__ void __launch_bounds__(128) k_mlp_infer(const __nv_bfloat16* __restrict__ wb_g,
                                                   const float* __restrict__ bias_g, const float* __restrict__ norm,
                                                   const float* __restrict__ X, int64_t n, int normalised,
                                                   float* __restrict__ Y) {
    __shared__ __align__(16) uint2 s_wf[MLPW_N];
    __shared__ float s_bias[MLPF_N];
    __shared__ __align__(16) __nv_bfloat16 s_x[4][32 * MLP_NIP];
    __shared__ float s_y[4][32 * MLP_NOP];
    mlp_frag_weights(wb_g, s_wf, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < MLPF_N; i += blockDim.x) s_bias[i] = bias_g[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * 4 + warp) * 32 + lane;
    __nv_bfloat16* x = s_x[warp] + lane * MLP_NIP;
#pragma unroll
    for (int c = 0; c < MLP_NIP; ++c) {
        float v = 0.f;
        if (row < n && c < MLP_NI) {
            v = X[row * MLP_NI + c];
            if (!normalised) v = (v - norm[c]) / norm[MLP_NI + c];
        }
        x[c] = __float2bfloat16_rn(v);
    }
    __syncwarp();
    warp_mlp_rows32(s_wf, s_bias, s_x[warp], 0, s_y[warp]);
    __syncwarp();
    if (row < n)
        for (int c = 0; c < MLP_NO; ++c) Y[row * MLP_NO + c] = s_y[warp][lane * MLP_NOP + c];
}

// sum of the masks of a batch (the loss normaliser)
__global__ void k_mask_sum(const float* __restrict__ mask, int64_t ndata, int64_t batch, uint64_t seed,
                           const float* __restrict__ mask_direct, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < batch; i += (int64_t)gridDim.x * blockDim.x) {
        const float* m;
        if (mask_direct) m = mask_direct + i * 8;
        else m = mask + (int64_t)(splitmix64(seed ^ (uint64_t)i * 0x9e3779b97f4a7c15ull) % (uint64_t)ndata) * 8;
        for (int c = 0; c < MLP_NO; ++c) s += m[c];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

tp_status model_alloc(tp_ctx* ctx) {
    if (ctx->mlp) return TP_OK;
    tp_mlp_model* m = new tp_mlp_model();
    ctx->mlp = m;
    TP_TRY(tp_alloc_t(ctx, &m->master, MLP_NPARAM));
    TP_TRY(tp_alloc_t(ctx, &m->am, MLP_NPARAM));
    TP_TRY(tp_alloc_t(ctx, &m->av, MLP_NPARAM));
    TP_TRY(tp_alloc_t(ctx, &m->grad, MLP_NPARAM));
    TP_TRY(tp_alloc_t(ctx, &m->wb, MLPB_N));
    TP_TRY(tp_alloc_t(ctx, &m->bias, MLPF_N));
    TP_TRY(tp_alloc_t(ctx, &m->norm, 4 * MLP_NI));
    TP_TRY(tp_alloc_t(ctx, &m->red, 4));
    TP_TRY(tp_alloc_t(ctx, &m->dcount_d, 4));
    TP_CU(cudaMemsetAsync(m->wb, 0, sizeof(__nv_bfloat16) * MLPB_N, ctx->stream));
    TP_CU(cudaMemsetAsync(m->bias, 0, sizeof(float) * MLPF_N, ctx->stream));
    TP_CU(cudaMemsetAsync(m->am, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
    TP_CU(cudaMemsetAsync(m->av, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
    return TP_OK;
}

tp_status pack(tp_ctx* ctx) {
    k_pack_weights<<<(MLP_NPARAM + 255) / 256, 256, 0, ctx->stream>>>(ctx->mlp->master, ctx->mlp->wb, ctx->mlp->bias);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

struct ModelHeader {
    char magic[4];
    uint32_t version, ni, nh, no, nparam;
    float theta;
    uint32_t q, p, step, reserved[4];
};

tp_status ensure_dataset(tp_ctx* ctx, int64_t need) {
    tp_mlp_model* m = ctx->mlp;
    if (need <= m->dcap) return TP_OK;
    int64_t cap = std::max<int64_t>(need, 2 * m->dcap);
    float *f = nullptr, *l = nullptr, *k = nullptr;
    TP_TRY(tp_alloc_t(ctx, &f, cap * MLP_NI));
    TP_TRY(tp_alloc_t(ctx, &l, cap * 8));
    TP_TRY(tp_alloc_t(ctx, &k, cap * 8));
    if (m->dcount > 0) {
        TP_CU(cudaMemcpyAsync(f, m->dfeat, sizeof(float) * MLP_NI * m->dcount, cudaMemcpyDeviceToDevice, ctx->stream));
        TP_CU(cudaMemcpyAsync(l, m->dlab, sizeof(float) * 8 * m->dcount, cudaMemcpyDeviceToDevice, ctx->stream));
        TP_CU(cudaMemcpyAsync(k, m->dmask, sizeof(float) * 8 * m->dcount, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    TP_CU(cudaStreamSynchronize(ctx->stream));
    tp_free(ctx, m->dfeat);
    tp_free(ctx, m->dlab);
    tp_free(ctx, m->dmask);
    m->dfeat = f;
    m->dlab = l;
    m->dmask = k;
    m->dcap = cap;
    return TP_OK;
}

}  // namespace

// ---------------------------------------------------------------- library-internal
void tp_mlp_release(tp_ctx* ctx) {
    if (!ctx->mlp) return;
    tp_mlp_model* m = ctx->mlp;
    tp_free(ctx, m->master);
    tp_free(ctx, m->am);
    tp_free(ctx, m->av);
    tp_free(ctx, m->grad);
    tp_free(ctx, m->wb);
    tp_free(ctx, m->bias);
    tp_free(ctx, m->norm);
    tp_free(ctx, m->red);
    tp_free(ctx, m->dcount_d);
    tp_free(ctx, m->dfeat);
    tp_free(ctx, m->dlab);
    tp_free(ctx, m->dmask);
    tp_free(ctx, m->dpairs);
    delete m;
    ctx->mlp = nullptr;
}

tp_status tp_mlp_node_features(tp_ctx* ctx) {
    tp_tree& t = ctx->tree;
    const int64_t nn = 2 * ctx->nt - 1;
    k_node_feat<<<(unsigned)((nn + TP_NODE_BLK - 1) / TP_NODE_BLK), TP_NODE_THREADS, 0, ctx->stream>>>(
        t.mom, t.box, t.parent, t.first, t.last, t.leaf_size, nn, t.nodeft);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_ensure_node_features(tp_ctx* ctx) {
    TpRange nvtx_range("tp_ensure_node_features");
    if (!ctx->tree.feat_stale) return TP_OK;
    TP_TRY(tp_mlp_node_features(ctx));
    ctx->tree.feat_stale = false;
    return TP_OK;
}

const void* tp_mlp_weights(const tp_ctx* ctx) { return ctx->mlp ? ctx->mlp->wb : nullptr; }
const float* tp_mlp_bias(const tp_ctx* ctx) { return ctx->mlp ? ctx->mlp->bias : nullptr; }
const float* tp_mlp_norm(const tp_ctx* ctx) { return ctx->mlp ? ctx->mlp->norm : nullptr; }
bool tp_mlp_ready(const tp_ctx* ctx) { return ctx->mlp && ctx->mlp->have_norm; }

// ---------------------------------------------------------------- C ABI
extern "C" {

tp_status tp_far_model_init(tp_ctx* ctx, uint64_t seed) {
    if (!ctx) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    TP_TRY(model_alloc(ctx));
    // Xavier-uniform weights, zero biases (host RNG: splitmix64 of (seed, index))
    std::vector<float> P(MLP_NPARAM, 0.f);
    auto fill = [&](int off, int nout, int nin) {
        const double a = std::sqrt(6.0 / (nin + nout));
        for (int i = 0; i < nout * nin; ++i) {
            uint64_t x = seed * 0x9e3779b97f4a7c15ull + (uint64_t)(off + i) + 1;
            x += 0x9e3779b97f4a7c15ull;
            x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
            x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
            x ^= x >> 31;
            const double u = (double)(x >> 11) / 9007199254740992.0;
            P[off + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    fill(MLP_OFF_W1, MLP_NH, MLP_NI);
    fill(MLP_OFF_W2, MLP_NH, MLP_NH);
    fill(MLP_OFF_W3, MLP_NH, MLP_NH);
    fill(MLP_OFF_W4, MLP_NO, MLP_NH);
    // small output layer: the untrained network predicts factors near 1
    for (int i = 0; i < MLP_NO * MLP_NH; ++i) P[MLP_OFF_W4 + i] *= 0.01f;
    TP_CU(cudaMemcpyAsync(ctx->mlp->master, P.data(), sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice,
                          ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->mlp->am, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->mlp->av, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
    ctx->mlp->step = 0;
    TP_TRY(pack(ctx));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    return TP_OK;
}

tp_status tp_far_set_params(tp_ctx* ctx, const float* params, const float* norm) {
    if (!ctx || !params) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    TP_TRY(model_alloc(ctx));
    TP_CU(cudaMemcpyAsync(ctx->mlp->master, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, ctx->stream));
    if (norm) {
        TP_CU(cudaMemcpyAsync(ctx->mlp->norm, norm, sizeof(float) * 4 * MLP_NI, cudaMemcpyHostToDevice, ctx->stream));
        ctx->mlp->have_norm = true;
    }
    TP_TRY(pack(ctx));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    return TP_OK;
}

tp_status tp_far_get_params(tp_ctx* ctx, float* params, float* norm) {
    if (!ctx || !ctx->mlp) return TP_E_STATE;
    cudaSetDevice(ctx->device);
    if (params)
        TP_CU(cudaMemcpyAsync(params, ctx->mlp->master, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost,
                              ctx->stream));
    if (norm)
        TP_CU(cudaMemcpyAsync(norm, ctx->mlp->norm, sizeof(float) * 4 * MLP_NI, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    return TP_OK;
}

tp_status tp_far_dataset_reset(tp_ctx* ctx) {
    if (!ctx) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    TP_TRY(model_alloc(ctx));
    ctx->mlp->dcount = 0;
    return TP_OK;
}

tp_status tp_far_dataset_size(tp_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return TP_E_ARG;
    *n = ctx->mlp ? ctx->mlp->dcount : 0;
    return TP_OK;
}

// Sample admissible (leaf, cluster) pairs of the current tree at opening
// angle theta, each kept with probability keep (counter-based hash of the
// pair and seed), up to max_pairs; append their features and labels.
tp_status tp_far_sample_pairs(tp_ctx* ctx, double theta, double keep, uint64_t seed, int64_t max_pairs,
                              int64_t* n_added) {
    TpRange nvtx_range("tp_far_sample_pairs");
    if (!ctx) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    ctx->err.clear();
    if (!ctx->tree.valid || ctx->nt < 2) return tp_set_err(ctx, TP_E_STATE, "tp_far_sample_pairs needs a tree");
    if (!(keep > 0.0 && keep <= 1.0) || max_pairs < 0 || !(theta > 0.0))
        return tp_set_err(ctx, TP_E_ARG, "bad sampling arguments");
    TP_TRY(model_alloc(ctx));
    tp_mlp_model* m = ctx->mlp;
    if (m->dpairs) tp_free(ctx, m->dpairs);
    m->dpairs = nullptr;
    TP_TRY(tp_alloc_t(ctx, &m->dpairs, std::max<int64_t>(1, max_pairs)));
    TP_CU(cudaMemsetAsync(m->dcount_d, 0, sizeof(int32_t), ctx->stream));
    const uint32_t keep_u = keep >= 1.0 ? 0xffffffffu : (uint32_t)(keep * 4294967296.0);
    TP_TRY(tp_launch_bh_sample(ctx, theta, keep_u, seed, m->dpairs, max_pairs, m->dcount_d));
    int32_t h = 0;
    TP_CU(cudaMemcpyAsync(&h, m->dcount_d, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    if (max_pairs == 0) {  // count only
        if (n_added) *n_added = h;
        return TP_OK;
    }
    const int64_t np = std::min<int64_t>(h, max_pairs);
    TP_TRY(ensure_dataset(ctx, m->dcount + np));
    if (np > 0) {
        TP_TRY(tp_ensure_node_features(ctx));
        tp_tree& t = ctx->tree;
        k_far_label<<<(unsigned)np, 128, 0, ctx->stream>>>(m->dpairs, m->dcount, np, t.leaves, t.first, t.last, t.mom,
                                                           t.nodeft, ctx->soa, ctx->ntp, ctx->center, 6, m->dfeat,
                                                           m->dlab, m->dmask);
        ++ctx->nlaunch;
        TP_CU(cudaGetLastError());
    }
    TP_CU(cudaStreamSynchronize(ctx->stream));
    m->dcount += np;
    m->theta = (float)theta;
    if (n_added) *n_added = np;
    return TP_OK;
}

// Copy dataset rows [i0, i0 + n) to the host (features [n][24], labels and masks [n][8]).
tp_status tp_far_dataset_get(tp_ctx* ctx, int64_t i0, int64_t n, float* feat, float* lab, float* mask,
                             int32_t* pairs) {
    if (!ctx || !ctx->mlp) return TP_E_STATE;
    cudaSetDevice(ctx->device);
    tp_mlp_model* m = ctx->mlp;
    if (i0 < 0 || n < 0 || i0 + n > m->dcount) return tp_set_err(ctx, TP_E_ARG, "rows outside the dataset");
    if (feat) TP_CU(cudaMemcpyAsync(feat, m->dfeat + i0 * MLP_NI, 4 * MLP_NI * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (lab) TP_CU(cudaMemcpyAsync(lab, m->dlab + i0 * 8, 32 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (mask) TP_CU(cudaMemcpyAsync(mask, m->dmask + i0 * 8, 32 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (pairs && m->dpairs) TP_CU(cudaMemcpyAsync(pairs, m->dpairs, 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    return TP_OK;
}

// Feature normalisation (mean, std) and in-distribution ranges from the dataset.
tp_status tp_far_fit_normalisation(tp_ctx* ctx) {
    TpRange nvtx_range("tp_far_fit_normalisation");
    if (!ctx || !ctx->mlp || ctx->mlp->dcount < 2) return TP_E_STATE;
    cudaSetDevice(ctx->device);
    k_feat_stats<<<MLP_NI, 256, 0, ctx->stream>>>(ctx->mlp->dfeat, ctx->mlp->dcount, ctx->mlp->norm);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->mlp->have_norm = true;
    return TP_OK;
}

// `steps` AdamW steps on batches of `batch` rows drawn from the dataset;
// *mean_loss receives the mean batch loss of the last step.
tp_status tp_far_train(tp_ctx* ctx, int64_t steps, int64_t batch, double lr, double wd, uint64_t seed,
                       double* last_loss) {
    TpRange nvtx_range("tp_far_train");
    if (!ctx || !ctx->mlp) return TP_E_STATE;
    cudaSetDevice(ctx->device);
    tp_mlp_model* m = ctx->mlp;
    if (m->dcount < 1 || !m->have_norm) return tp_set_err(ctx, TP_E_STATE, "empty dataset or no normalisation");
    if (steps < 1 || batch < 1) return tp_set_err(ctx, TP_E_ARG, "steps and batch must be positive");
    // per-device attribute: set on the current device at every call
    TP_CU(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
    const unsigned blocks = (unsigned)((batch + TB - 1) / TB);
    double hl[2] = {0, 0};
    for (int64_t s = 0; s < steps; ++s) {
        const uint64_t sd = seed * 0x2545f4914f6cdd1dull + (uint64_t)m->step * 0x9e3779b97f4a7c15ull + 17;
        TP_CU(cudaMemsetAsync(m->red, 0, 2 * sizeof(double), ctx->stream));
        TP_CU(cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
        k_mask_sum<<<64, 256, 0, ctx->stream>>>(m->dmask, m->dcount, batch, sd, nullptr, m->red + 1);
        TP_CU(cudaMemcpyAsync(hl + 1, m->red + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        TP_CU(cudaStreamSynchronize(ctx->stream));
        const float inv_msum = hl[1] > 0.0 ? (float)(1.0 / hl[1]) : 0.f;
        k_mlp_train<<<blocks, 128, sizeof(TrainSmem), ctx->stream>>>(m->wb, m->bias, m->norm, m->dfeat, m->dlab,
                                                                    m->dmask, m->dcount, batch, sd, nullptr, 0,
                                                                    inv_msum, m->grad, m->red, nullptr);
        m->step += 1;
        const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
        k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, ctx->stream>>>(m->master, m->am, m->av, m->grad, (float)lr, 0.9f,
                                                                   0.999f, 1e-8f, (float)wd, c1, c2);
        TP_TRY(pack(ctx));
        TP_CU(cudaGetLastError());
        if (s == steps - 1) {
            TP_CU(cudaMemcpyAsync(hl, m->red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            TP_CU(cudaStreamSynchronize(ctx->stream));
            if (last_loss) *last_loss = hl[1] > 0.0 ? hl[0] / hl[1] : 0.0;
        }
    }
    return TP_OK;
}

// Forward pass (and, with tgt/mask, the loss and parameter gradient) of the
// current network on given rows: X [n][24] (raw features unless normalised
// != 0), Y [n][7] out; grad [MLP_NPARAM] out (may be null).  For tests.
tp_status tp_far_eval(tp_ctx* ctx, const float* X, int64_t n, int normalised, const float* tgt, const float* mask,
                      float* Y, float* grad, double* loss) {
    TpRange nvtx_range("tp_far_eval");
    if (!ctx || !ctx->mlp || !X || n < 1) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    tp_mlp_model* m = ctx->mlp;
    if (!(normalised & 1) && !m->have_norm) return tp_set_err(ctx, TP_E_STATE, "no normalisation");
    // per-device attribute: set on the current device at every call
    TP_CU(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
    float *dX = nullptr, *dT = nullptr, *dM = nullptr, *dY = nullptr;
    if (!tgt && !mask) {
        // forward only: the inference kernels of the learned correction, the
        // tensor-core (tcgen05) network, or with normalised = 2 or 3 (bit 1 set)
        // the register-resident mma.sync one
        const bool sync_path = normalised >= 2;
        const int norm_in = normalised & 1;
        TP_TRY(tp_alloc_t(ctx, &dX, n * MLP_NI));
        TP_TRY(tp_alloc_t(ctx, &dY, n * 8));
        TP_CU(cudaMemcpyAsync(dX, X, 4 * MLP_NI * n, cudaMemcpyHostToDevice, ctx->stream));
        if (sync_path) {
            k_mlp_infer<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(m->wb, m->bias, m->norm, dX, n,
                                                                              norm_in, dY);
            TP_CU(cudaGetLastError());
            if (Y) TP_CU(cudaMemcpyAsync(Y, dY, 4 * MLP_NO * n, cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            __nv_bfloat16* dR = nullptr;
            TP_TRY(tp_alloc_t(ctx, &dR, n * MLP_NIP));
            k_rows_bf16<<<(unsigned)((n * MLP_NIP + 255) / 256), 256, 0, ctx->stream>>>(dX, n, norm_in, m->norm, dR);
            TP_TRY(tp_launch_mlp_tc(ctx, m->wb, m->bias, dR, n, dY, 1));
            std::vector<float> y8(8 * n);
            TP_CU(cudaMemcpyAsync(y8.data(), dY, 32 * n, cudaMemcpyDeviceToHost, ctx->stream));
            TP_CU(cudaStreamSynchronize(ctx->stream));
            if (Y)
                for (int64_t r = 0; r < n; ++r)
                    for (int c = 0; c < MLP_NO; ++c) Y[r * MLP_NO + c] = y8[r * 8 + c];
            tp_free(ctx, dR);
        }
        TP_CU(cudaStreamSynchronize(ctx->stream));
        TP_TRY(take_device_error(ctx, "tp_far_eval"));
        if (grad) memset(grad, 0, 4 * MLP_NPARAM);
        if (loss) *loss = 0.0;
        tp_free(ctx, dX);
        tp_free(ctx, dY);
        return TP_OK;
    }
    TP_TRY(tp_alloc_t(ctx, &dX, n * MLP_NI));
    TP_TRY(tp_alloc_t(ctx, &dT, n * 8));
    TP_TRY(tp_alloc_t(ctx, &dM, n * 8));
    TP_TRY(tp_alloc_t(ctx, &dY, n * MLP_NO));
    TP_CU(cudaMemcpyAsync(dX, X, 4 * MLP_NI * n, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<float> z(8 * n, 0.f);
    TP_CU(cudaMemcpyAsync(dT, tgt ? tgt : z.data(), 32 * n, cudaMemcpyHostToDevice, ctx->stream));
    TP_CU(cudaMemcpyAsync(dM, mask ? mask : z.data(), 32 * n, cudaMemcpyHostToDevice, ctx->stream));
    TP_CU(cudaMemsetAsync(m->red, 0, 2 * sizeof(double), ctx->stream));
    TP_CU(cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NPARAM, ctx->stream));
    k_mask_sum<<<64, 256, 0, ctx->stream>>>(nullptr, 1, n, 0, dM, m->red + 1);
    double hl[2] = {0, 0};
    TP_CU(cudaMemcpyAsync(hl + 1, m->red + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    const float inv_msum = hl[1] > 0.0 ? (float)(1.0 / hl[1]) : 0.f;
    const unsigned blocks = (unsigned)((n + TB - 1) / TB);
    k_mlp_train<<<blocks, 128, sizeof(TrainSmem), ctx->stream>>>(m->wb, m->bias, m->norm, nullptr, dT, dM, n, n, 0,
                                                                dX, normalised & 1, inv_msum, m->grad, m->red, dY);
    TP_CU(cudaGetLastError());
    if (Y) TP_CU(cudaMemcpyAsync(Y, dY, 4 * MLP_NO * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (grad) TP_CU(cudaMemcpyAsync(grad, m->grad, 4 * MLP_NPARAM, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hl, m->red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = hl[1] > 0.0 ? hl[0] / hl[1] : 0.0;
    tp_free(ctx, dX);
    tp_free(ctx, dT);
    tp_free(ctx, dM);
    tp_free(ctx, dY);
    return TP_OK;
}

// One AdamW step with a given gradient (host, [MLP_NPARAM]); for tests.
tp_status tp_far_adamw_step(tp_ctx* ctx, const float* grad, double lr, double wd) {
    TpRange nvtx_range("tp_far_adamw_step");
    if (!ctx || !ctx->mlp || !grad) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    tp_mlp_model* m = ctx->mlp;
    TP_CU(cudaMemcpyAsync(m->grad, grad, 4 * MLP_NPARAM, cudaMemcpyHostToDevice, ctx->stream));
    m->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
    k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, ctx->stream>>>(m->master, m->am, m->av, m->grad, (float)lr, 0.9f,
                                                               0.999f, 1e-8f, (float)wd, c1, c2);
    TP_TRY(pack(ctx));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    return TP_OK;
}

tp_status tp_far_model_save(tp_ctx* ctx, const char* path) {
    if (!ctx || !path) return TP_E_ARG;
    if (!ctx->mlp || !ctx->mlp->have_norm) return tp_set_err(ctx, TP_E_STATE, "no trained model to save");
    std::vector<float> P(MLP_NPARAM), N(4 * MLP_NI);
    TP_TRY(tp_far_get_params(ctx, P.data(), N.data()));
    FILE* f = fopen(path, "wb");
    if (!f) return tp_set_err(ctx, TP_E_ARG, "cannot open %s for writing", path);
    ModelHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "TPFM", 4);
    h.version = 1;
    h.ni = MLP_NI;
    h.nh = MLP_NH;
    h.no = MLP_NO;
    h.nparam = MLP_NPARAM;
    h.theta = ctx->mlp->theta;
    h.q = 6;
    h.p = 12;
    h.step = (uint32_t)ctx->mlp->step;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(N.data(), 4, N.size(), f) == N.size() &&
              fwrite(P.data(), 4, P.size(), f) == P.size();
    fclose(f);
    return ok ? TP_OK : tp_set_err(ctx, TP_E_ARG, "write to %s failed", path);
}

tp_status tp_far_model_load(tp_ctx* ctx, const char* path) {
    TpRange nvtx_range("tp_far_model_load");
    if (!ctx || !path) return TP_E_ARG;
    cudaSetDevice(ctx->device);
    FILE* f = fopen(path, "rb");
    if (!f) return tp_set_err(ctx, TP_E_MODEL, "cannot open %s", path);
    ModelHeader h;
    std::vector<float> P(MLP_NPARAM), N(4 * MLP_NI);
    bool ok = fread(&h, sizeof(h), 1, f) == 1;
    ok = ok && memcmp(h.magic, "TPFM", 4) == 0 && h.version == 1 && h.ni == MLP_NI && h.nh == MLP_NH &&
         h.no == MLP_NO && h.nparam == MLP_NPARAM;
    ok = ok && fread(N.data(), 4, N.size(), f) == N.size() && fread(P.data(), 4, P.size(), f) == P.size();
    fclose(f);
    if (!ok) return tp_set_err(ctx, TP_E_MODEL, "%s is not a version-1 far-field model", path);
    for (float v : P)
        if (!std::isfinite(v)) return tp_set_err(ctx, TP_E_MODEL, "%s holds non-finite weights", path);
    TP_TRY(tp_far_set_params(ctx, P.data(), N.data()));
    ctx->mlp->theta = h.theta;
    ctx->mlp->step = (int)h.step;
    return TP_OK;
}

}  // extern "C"
