// tp_tri.cu - per-triangle data (centroid, unit normal, area), Morton order,
// the library-order SoA staged by the pair kernels, vertex->triangle
// incidence and the masks of super-tile pairs.
//
// Sec. 3.2 caches positions, area elements and normals at every quadrature
// point contiguously and iterates them in memory order; here the cache is a
// structure of arrays in Morton order (one point per triangle).
//
// The FP64 triangle data is computed with separately rounded operations in
// a fixed association order - x = ((v0 + v1) + v2) / 3, N = e1 x e2 with
// products then differences, |N| = sqrt((Nx^2 + Ny^2) + Nz^2), w = |N|/2,
// nu = N/|N| - so the Morton codes and cluster moments built from it are
// reproducible bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "tp_internal.cuh"

namespace {

// Per element: position, unit normal and weight.  With the centroid rule the
// element is the triangle, x = ((v0 + v1) + v2) / 3 and w = |N| / 2; with a
// k-point rule element i is point q = i % k of its triangle (whose vertices
// F[i] carries), x = (l0 v0 + l1 v1) + l2 v2 and w = om_q |N| / 2; every
// operation separately rounded (the oracle's order).
__global__ void k_tri_data(const double* __restrict__ V, const int32_t* __restrict__ F, int64_t nt, int64_t nv,
                           double* __restrict__ x64, double* __restrict__ nu64, double* __restrict__ w64,
                           unsigned* derr, tp_quad_rule rule) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    int32_t i0 = F[3 * T], i1 = F[3 * T + 1], i2 = F[3 * T + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        tp_dev_error(derr, TP_DERR_INDEX);
        for (int a = 0; a < 3; ++a) {
            x64[a * nt + T] = 0.0;
            nu64[a * nt + T] = 0.0;
        }
        w64[T] = 0.0;
        return;
    }
    const double* a = V + 3 * (int64_t)i0;
    const double* b = V + 3 * (int64_t)i1;
    const double* c = V + 3 * (int64_t)i2;
    double e1[3], e2[3];
    const int q = rule.k > 1 ? (int)(T % rule.k) : 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (rule.k == 1)
            x64[k * nt + T] = __ddiv_rn(__dadd_rn(__dadd_rn(a[k], b[k]), c[k]), 3.0);
        else
            x64[k * nt + T] = __dadd_rn(__dadd_rn(__dmul_rn(rule.bary[q][0], a[k]), __dmul_rn(rule.bary[q][1], b[k])),
                                        __dmul_rn(rule.bary[q][2], c[k]));
        e1[k] = __dsub_rn(b[k], a[k]);
        e2[k] = __dsub_rn(c[k], a[k]);
    }
    double N0 = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    double N1 = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    double N2 = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
    double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(N0, N0), __dmul_rn(N1, N1)), __dmul_rn(N2, N2)));
    if (!(len > 0.0) || !isfinite(len)) tp_dev_error(derr, TP_DERR_NONFINITE);
    w64[T] = rule.k == 1 ? __dmul_rn(0.5, len) : __dmul_rn(rule.w[q], __dmul_rn(0.5, len));
    nu64[0 * nt + T] = __ddiv_rn(N0, len);
    nu64[1 * nt + T] = __ddiv_rn(N1, len);
    nu64[2 * nt + T] = __ddiv_rn(N2, len);
}

// faces of the elements: every quadrature point carries its triangle's vertices
__global__ void k_expand_faces(const int32_t* __restrict__ Ft, int64_t nt_tri, int k, int32_t* __restrict__ F) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt_tri * k) return;
    const int64_t T = i / k;
    F[3 * i] = Ft[3 * T];
    F[3 * i + 1] = Ft[3 * T + 1];
    F[3 * i + 2] = Ft[3 * T + 2];
}

// per-block min/max of the centroids (6 values), then a final single-block pass
__global__ void k_bounds_partial(const double* __restrict__ x64, int64_t nt, double* __restrict__ part) {
    __shared__ double smin[3][256], smax[3][256];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; T < nt; T += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            double v = x64[a * nt + T];
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = mn[a];
        smax[a][threadIdx.x] = mx[a];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + s]);
                smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            part[6 * blockIdx.x + a] = smin[a][0];
            part[6 * blockIdx.x + 3 + a] = smax[a][0];
        }
}

__global__ void k_bounds_final(const double* __restrict__ part, int nb, double* __restrict__ bounds,
                               double* __restrict__ center) {
    __shared__ double smin[3][256], smax[3][256];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin(mn[a], part[6 * b + a]);
            mx[a] = fmax(mx[a], part[6 * b + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = mn[a];
        smax[a][threadIdx.x] = mx[a];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + o]);
                smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            bounds[a] = smin[a][0];
            bounds[3 + a] = smax[a][0];
            center[a] = 0.5 * (smin[a][0] + smax[a][0]);
        }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

// Morton code: q_a = min(2^b - 1, floor((x_a - lo_a) * (2^b / (hi_a - lo_a)))), FP64 RN,
// interleaved with x the most significant bit of each triplet.
__global__ void k_morton(const double* __restrict__ x64, int64_t nt, const double* __restrict__ bounds, int bits,
                         uint32_t* __restrict__ codes, int32_t* __restrict__ idx) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    const uint32_t Q = 1u << bits;
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double lo = bounds[a], hi = bounds[3 + a];
        double s = hi > lo ? __ddiv_rn((double)Q, __dsub_rn(hi, lo)) : 0.0;
        double t = __dmul_rn(__dsub_rn(x64[a * nt + T], lo), s);
        double f = floor(t);
        q[a] = f >= (double)(Q - 1) ? Q - 1 : (uint32_t)f;
    }
    codes[T] = (spread3(q[0], bits) << 2) | (spread3(q[1], bits) << 1) | spread3(q[2], bits);
    idx[T] = (int32_t)T;
}

// library-order SoA, staged source records and sorted faces
__global__ void k_sorted_soa(const double* __restrict__ x64, const double* __restrict__ nu64,
                             const double* __restrict__ w64, const int32_t* __restrict__ F,
                             const int32_t* __restrict__ perm, const double* __restrict__ center, int64_t nt,
                             int64_t ntp, int32_t* __restrict__ iperm, float* __restrict__ soa,
                             float* __restrict__ src, int32_t* __restrict__ Fs) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ntp) return;
    float v[10];
    int3 f;
    if (k < nt) {
        int64_t T = perm[k];
        iperm[T] = (int32_t)k;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double xc = x64[a * nt + T] - center[a];
            float hi = (float)xc;
            float lo = (float)(xc - (double)hi);
            v[a] = hi;
            v[3 + a] = lo;
            v[6 + a] = (float)nu64[a * nt + T];
        }
        v[9] = (float)(1.4142135623730951 * w64[T]);  // sqrt(p/q) w with p = 2q
        f = make_int3(F[3 * T], F[3 * T + 1], F[3 * T + 2]);
    } else {
        // zero-area padding placed far apart so no padding pair coincides
        v[0] = 4096.0f + 8.0f * (float)(k - nt);
        v[1] = 4096.0f;
        v[2] = 4096.0f;
        for (int a = 3; a < 10; ++a) v[a] = 0.0f;
        f = make_int3(-1, -1, -1);
    }
#pragma unroll
    for (int a = 0; a < 10; ++a) {
        soa[a * ntp + k] = v[a];
        src[k * TP_SRCW + 2 * a] = v[a];
        src[k * TP_SRCW + 2 * a + 1] = v[a];
    }
    Fs[3 * k] = f.x;
    Fs[3 * k + 1] = f.y;
    Fs[3 * k + 2] = f.z;
}

// vertex -> triangle incidence (CSR), entries triangle*4 + corner
__global__ void k_v2t_count(const int32_t* __restrict__ F, int64_t nt, int64_t nv, int32_t* __restrict__ cnt,
                            unsigned* derr) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * nt) return;
    int32_t v = F[i];
    if (v < 0 || v >= nv) {
        tp_dev_error(derr, TP_DERR_INDEX);
        return;
    }
    atomicAdd(&cnt[v], 1);
}

__global__ void k_v2t_fill(const int32_t* __restrict__ F, int64_t nt, int64_t nv, const int32_t* __restrict__ off,
                           int32_t* __restrict__ fillc, int32_t* __restrict__ v2t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * nt) return;
    int32_t v = F[i];
    if (v < 0 || v >= nv) return;
    int32_t slot = atomicAdd(&fillc[v], 1);
    v2t[off[v] + slot] = (int32_t)((i / 3) * 4 + (i % 3));
}

// sort each vertex's short list so later sums over it are deterministic
__global__ void k_v2t_sort(const int32_t* __restrict__ off, int64_t nv, int32_t* __restrict__ v2t) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int32_t b = off[v], e = off[v + 1];
    for (int32_t i = b + 1; i < e; ++i) {
        int32_t key = v2t[i];
        int32_t j = i - 1;
        while (j >= b && v2t[j] > key) {
            v2t[j + 1] = v2t[j];
            --j;
        }
        v2t[j + 1] = key;
    }
}

// super-tile pairs containing a pair of triangles that share a vertex, and
// within each such pair the 128 x 128 blocks holding one.  The pair {T, S}
// is evaluated as target = the one earlier in Morton order and source = the
// later one (the item is (I, J) with I <= J), which fixes its block.
__global__ void k_flag_pairs(const int32_t* __restrict__ F, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ iperm, const int32_t* __restrict__ off,
                             const int32_t* __restrict__ v2t, int64_t nt, int nsup, unsigned* __restrict__ bm,
                             unsigned* __restrict__ bmask) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    int64_t T = perm[k];
    for (int c = 0; c < 3; ++c) {
        int32_t v = F[3 * T + c];
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            int64_t S = v2t[e] >> 2;
            const int64_t ks = iperm[S];
            const int64_t kt = k < ks ? k : ks, kss = k < ks ? ks : k;  // target, source positions
            const int a = (int)(kt / TP_SUPER), b = (int)(kss / TP_SUPER);
            const int64_t bit = (int64_t)a * nsup + b;
            atomicOr(&bm[bit >> 5], 1u << (bit & 31));
            const int blk = (int)((kt % TP_SUPER) / TP_CHUNK) * TP_NBLK + (int)((kss % TP_SUPER) / TP_CHUNK);
            atomicOr(&bmask[bit * TP_BMASK_WORDS + (blk >> 5)], 1u << (blk & 31));
        }
    }
}

__global__ void k_flag_diag(int nsup, unsigned* __restrict__ bm) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nsup) return;
    int64_t bit = (int64_t)I * nsup + I;
    atomicOr(&bm[bit >> 5], 1u << (bit & 31));
}

// centroid box of every super-tile (f32 hi parts, library order)
__global__ void k_tile_boxes(const float* __restrict__ soa, int64_t ntp, int64_t nt, float* __restrict__ tbox) {
    __shared__ float red[6][256];
    const int64_t I = blockIdx.x;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int t = threadIdx.x; t < TP_SUPER; t += blockDim.x) {
        const int64_t k = I * TP_SUPER + t;
        if (k >= nt) break;
        for (int a = 0; a < 3; ++a) {
            const float v = soa[a * ntp + k];
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = mn[a];
        red[3 + a][threadIdx.x] = mx[a];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fminf(red[a][threadIdx.x], red[a][threadIdx.x + o]);
                red[3 + a][threadIdx.x] = fmaxf(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) tbox[6 * I + threadIdx.x] = red[threadIdx.x][0];
}

// Sort the super-tile pairs (I <= J) into: masked (a vertex-sharing pair
// inside, or I == J), precise (unmasked but the two centroid boxes lie
// closer than delta: centroid differences there need the hi/lo split), and
// fast (everything else; the bitmap bit stays clear).
__global__ void k_flag_classify(const unsigned* __restrict__ adj, unsigned* __restrict__ bm, int nsup, int64_t nt,
                                const float* __restrict__ tbox,
                                const double* __restrict__ bounds, float delta_rel, int32_t* __restrict__ mlist,
                                int32_t* __restrict__ plist, int32_t* __restrict__ flist, int32_t* __restrict__ count,
                                unsigned long long* __restrict__ npairs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)nsup * nsup;
    if (i >= n) return;
    const int I = (int)(i / nsup), J = (int)(i % nsup);
    if (J < I) return;
    // unordered pairs of real (non-padding) triangles in this item
    const int64_t rI = (nt - (int64_t)I * TP_SUPER) < TP_SUPER ? nt - (int64_t)I * TP_SUPER : TP_SUPER;
    const int64_t rJ = (nt - (int64_t)J * TP_SUPER) < TP_SUPER ? nt - (int64_t)J * TP_SUPER : TP_SUPER;
    const unsigned long long pairs = (unsigned long long)(I == J ? rI * (rI - 1) / 2 : rI * rJ);
    if ((adj[i >> 5] >> (i & 31)) & 1u) {
        mlist[atomicAdd(&count[0], 1)] = (I << 16) | J;
        atomicOr(&bm[i >> 5], 1u << (i & 31));
        atomicAdd(&npairs[2], pairs);
        return;
    }
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = bounds[3 + a] - bounds[a];
        d2 += e * e;
    }
    const float delta = delta_rel * (float)sqrt(d2);
    float g2 = 0.f;
    for (int a = 0; a < 3; ++a) {
        const float gap = fmaxf(0.f, fmaxf(tbox[6 * J + a] - tbox[6 * I + 3 + a], tbox[6 * I + a] - tbox[6 * J + 3 + a]));
        g2 += gap * gap;
    }
    if (g2 < delta * delta) {
        plist[atomicAdd(&count[1], 1)] = (I << 16) | J;
        atomicOr(&bm[i >> 5], 1u << (i & 31));
        atomicAdd(&npairs[1], pairs);
    } else {
        flist[atomicAdd(&count[8], 1)] = (I << 16) | J;
        atomicAdd(&npairs[0], pairs);
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

tp_status tp_launch_expand_faces(tp_ctx* ctx) {
    TpRange nvtx_range("tp_launch_expand_faces");
    const int64_t n = ctx->nt_tri * ctx->quad.k;
    k_expand_faces<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(ctx->F_tri, ctx->nt_tri, ctx->quad.k, ctx->F);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_tri_data(tp_ctx* ctx) {
    TpRange nvtx_range("tp_launch_tri_data");
    const int64_t nt = ctx->nt;
    k_tri_data<<<blocks_for(nt, 256), 256, 0, ctx->stream>>>(ctx->V64, ctx->F, nt, ctx->nv, ctx->x64, ctx->nu64,
                                                             ctx->w64, ctx->derr, ctx->quad);
    ++ctx->nlaunch;
    int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (nt + 255) / 256));
    k_bounds_partial<<<nb, 256, 0, ctx->stream>>>(ctx->x64, nt, ctx->red);
    ++ctx->nlaunch;
    k_bounds_final<<<1, 256, 0, ctx->stream>>>(ctx->red, nb, ctx->bounds, ctx->center);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_morton_order(tp_ctx* ctx, int morton_bits) {
    TpRange nvtx_range("tp_launch_morton_order");
    const int64_t nt = ctx->nt;
    k_morton<<<blocks_for(nt, 256), 256, 0, ctx->stream>>>(ctx->x64, nt, ctx->bounds, morton_bits / 3, ctx->codes,
                                                           ctx->idx_tmp);
    ++ctx->nlaunch;
    // stable sort of (code, T) by code: ties keep ascending T, i.e. the order of key = code << 32 | T
    TP_TRY(tp_sort_pairs_u32(ctx, ctx->codes, ctx->idx_tmp, ctx->codes_sorted, ctx->perm, nt, morton_bits));
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_sorted_soa(tp_ctx* ctx) {
    TpRange nvtx_range("tp_launch_sorted_soa");
    k_sorted_soa<<<blocks_for(ctx->ntp, 256), 256, 0, ctx->stream>>>(
        ctx->x64, ctx->nu64, ctx->w64, ctx->F, ctx->perm, ctx->center, ctx->nt, ctx->ntp, ctx->iperm, ctx->soa,
        ctx->src, ctx->Fs);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    ctx->soa_stale = false;
    return TP_OK;
}

tp_status tp_ensure_sorted(tp_ctx* ctx) {
    return ctx->soa_stale ? tp_launch_sorted_soa(ctx) : TP_OK;
}

tp_status tp_build_v2t(tp_ctx* ctx) {
    TpRange nvtx_range("tp_build_v2t");
    const int64_t nt = ctx->nt, nv = ctx->nv;
    int32_t* cnt = ctx->idx_tmp;  // reuse as counter scratch (nt >= nv/2 for closed meshes; sized max)
    TP_CU(cudaMemsetAsync(ctx->v2t_off, 0, sizeof(int32_t) * (nv + 1), ctx->stream));
    k_v2t_count<<<blocks_for(3 * nt, 256), 256, 0, ctx->stream>>>(ctx->F, nt, nv, ctx->v2t_off + 1, ctx->derr);
    ++ctx->nlaunch;
    uint32_t* off = reinterpret_cast<uint32_t*>(ctx->v2t_off + 1);
    TP_TRY(tp_scan_u32(ctx, off, off, nv, true, nullptr));
    TP_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nv, ctx->stream));
    k_v2t_fill<<<blocks_for(3 * nt, 256), 256, 0, ctx->stream>>>(ctx->F, nt, nv, ctx->v2t_off, cnt, ctx->v2t);
    ++ctx->nlaunch;
    k_v2t_sort<<<blocks_for(nv, 256), 256, 0, ctx->stream>>>(ctx->v2t_off, nv, ctx->v2t);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

// ------------------------------------------------------------ exclusion bits of masked blocks
__global__ void k_item_index(const int32_t* __restrict__ mlist, int n_masked, int nsup, int32_t* __restrict__ idx) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_masked) return;
    const int I = mlist[m] >> 16, J = mlist[m] & 0xffff;
    idx[(int64_t)I * nsup + J] = m;
}

// blocks of masked item m that take the per-pair test: on a diagonal item the
// blocks level with the diagonal and those above it holding a vertex-sharing
// pair (blocks below are skipped), elsewhere the blocks holding one
__global__ void k_xeff(const int32_t* __restrict__ mlist, int n_masked, int nsup, const unsigned* __restrict__ bmask,
                       unsigned* __restrict__ xeff, int32_t* __restrict__ xcount) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > n_masked) return;
    if (m == n_masked) {
        xcount[m] = 0;
        return;
    }
    const int I = mlist[m] >> 16, J = mlist[m] & 0xffff;
    const unsigned* bm = bmask + ((int64_t)I * nsup + J) * TP_BMASK_WORDS;
    int cnt = 0;
    for (int wd = 0; wd < TP_BMASK_WORDS; ++wd) {
        unsigned v = 0;
        for (int bit = 0; bit < 32; ++bit) {
            const int blk = 32 * wd + bit;
            if (blk >= TP_NBLK * TP_NBLK) break;
            const int w = blk / TP_NBLK, c = blk % TP_NBLK;
            const bool set = (bm[wd] >> bit) & 1u;
            const bool use = I == J ? (c == w || (c > w && set)) : set;
            if (use) v |= 1u << bit;
        }
        xeff[(int64_t)m * TP_BMASK_WORDS + wd] = v;
        cnt += __popc(v);
    }
    xcount[m] = cnt;
}

// slot of block blk of masked item m: its first slot plus the used blocks before blk
__device__ __forceinline__ int64_t x_slot(const unsigned* xeff, const int32_t* xbase, int m, int blk) {
    const unsigned* e = xeff + (int64_t)m * TP_BMASK_WORDS;
    int r = 0;
    for (int wd = 0; wd < blk >> 5; ++wd) r += __popc(e[wd]);
    r += __popc(e[blk >> 5] & ((1u << (blk & 31)) - 1u));
    return (int64_t)xbase[m] + r;
}

// the vertex-sharing pairs: every element and each element touching one of its
// vertices (target = the earlier in Morton order)
__global__ void k_xmask_pairs(const int32_t* __restrict__ F, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ iperm, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ v2t, int64_t nt, int nsup,
                              const int32_t* __restrict__ item_index, const unsigned* __restrict__ xeff,
                              const int32_t* __restrict__ xbase, uint32_t* __restrict__ xmask) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const int64_t T = perm[k];
    for (int c = 0; c < 3; ++c) {
        const int32_t v = F[3 * T + c];
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            const int64_t ks = iperm[v2t[e] >> 2];
            const int64_t kt = k < ks ? k : ks, kss = k < ks ? ks : k;
            const int a = (int)(kt / TP_SUPER), b = (int)(kss / TP_SUPER);
            const int m = item_index[(int64_t)a * nsup + b];
            if (m < 0) continue;  // cannot happen: the pair makes the item masked
            const int tl = (int)(kt % TP_SUPER), sl = (int)(kss % TP_SUPER);
            const int blk = (tl / TP_CHUNK) * TP_NBLK + sl / TP_CHUNK;
            const int64_t slot = x_slot(xeff, xbase, m, blk);
            const int t = tl % TP_CHUNK, s = sl % TP_CHUNK;
            atomicOr(&xmask[(slot * TP_CHUNK + t) * 4 + (s >> 5)], 1u << (s & 31));
        }
    }
}

// diagonal blocks of diagonal items: source <= target is not a pair of the item
__global__ void k_xmask_diag(const int32_t* __restrict__ mlist, int n_masked, const unsigned* __restrict__ xeff,
                             const int32_t* __restrict__ xbase, uint32_t* __restrict__ xmask) {
    const int m = blockIdx.x;
    if (m >= n_masked) return;
    const int I = mlist[m] >> 16, J = mlist[m] & 0xffff;
    if (I != J) return;
    for (int i = threadIdx.x; i < TP_NBLK * TP_CHUNK; i += blockDim.x) {
        const int w = i / TP_CHUNK, t = i % TP_CHUNK;
        const int64_t slot = x_slot(xeff, xbase, m, w * TP_NBLK + w);
        for (int wd = 0; wd < 4; ++wd) {
            const int lo = 32 * wd;
            unsigned bits;
            if (t >= lo + 31) bits = 0xffffffffu;  // every source of this word <= t
            else if (t < lo) bits = 0u;
            else bits = (t - lo == 31) ? 0xffffffffu : ((1u << (t - lo + 1)) - 1u);
            atomicOr(&xmask[(slot * TP_CHUNK + t) * 4 + wd], bits);
        }
    }
}

tp_status tp_build_exclusion_bits(tp_ctx* ctx) {
    TpRange nvtx_range("tp_build_exclusion_bits");
    const int nsup = (int)ctx->nsup;
    const int nm = (int)ctx->n_masked;
    const int64_t nbits = (int64_t)nsup * nsup;
    if (nbits > ctx->x_item_cap || !ctx->item_index) {
        tp_free(ctx, ctx->item_index);
        ctx->item_index = nullptr;
        TP_TRY(tp_alloc_t(ctx, &ctx->item_index, nbits));
    }
    if (nm + 1 > ctx->x_item_cap || !ctx->xeff) {
        tp_free(ctx, ctx->xeff);
        tp_free(ctx, ctx->xbase);
        tp_free(ctx, ctx->xcount);
        ctx->xeff = nullptr;
        ctx->xbase = nullptr;
        ctx->xcount = nullptr;
        const int64_t cap = std::max<int64_t>(nbits, nm + 1);
        TP_TRY(tp_alloc_t(ctx, &ctx->xeff, cap * TP_BMASK_WORDS));
        TP_TRY(tp_alloc_t(ctx, &ctx->xbase, cap + 1));
        TP_TRY(tp_alloc_t(ctx, &ctx->xcount, cap + 1));
        ctx->x_item_cap = cap;
    }
    TP_CU(cudaMemsetAsync(ctx->item_index, 0xff, sizeof(int32_t) * nbits, ctx->stream));
    if (nm == 0) {
        ctx->x_slots = 0;
        return TP_OK;
    }
    k_item_index<<<blocks_for(nm, 256), 256, 0, ctx->stream>>>(ctx->mlist, nm, nsup, ctx->item_index);
    int32_t* xcount = ctx->xcount;
    k_xeff<<<blocks_for(nm + 1, 256), 256, 0, ctx->stream>>>(ctx->mlist, nm, nsup, ctx->bmask, ctx->xeff, xcount);
    ctx->nlaunch += 2;
    TP_TRY(tp_scan_u32(ctx, reinterpret_cast<const uint32_t*>(xcount), reinterpret_cast<uint32_t*>(ctx->xbase),
                       nm + 1, false, nullptr));
    int32_t total = 0;
    TP_CU(cudaMemcpyAsync(&total, ctx->xbase + nm, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->x_slots = total;
    if (total > ctx->x_cap || !ctx->xmask) {
        tp_free(ctx, ctx->xmask);
        ctx->xmask = nullptr;
        TP_TRY(tp_alloc_t(ctx, &ctx->xmask, std::max<int64_t>(total, 1) * TP_CHUNK * 4));
        ctx->x_cap = std::max<int64_t>(total, 1);
    }
    TP_CU(cudaMemsetAsync(ctx->xmask, 0, sizeof(uint32_t) * (size_t)total * TP_CHUNK * 4, ctx->stream));
    k_xmask_pairs<<<blocks_for(ctx->nt, 256), 256, 0, ctx->stream>>>(ctx->F, ctx->perm, ctx->iperm, ctx->v2t_off,
                                                                     ctx->v2t, ctx->nt, nsup, ctx->item_index,
                                                                     ctx->xeff, ctx->xbase, ctx->xmask);
    k_xmask_diag<<<nm, 256, 0, ctx->stream>>>(ctx->mlist, nm, ctx->xeff, ctx->xbase, ctx->xmask);
    ctx->nlaunch += 2;
    if (!ctx->xptrs) TP_TRY(tp_alloc_t(ctx, &ctx->xptrs, 3));
    const uint64_t hp[3] = {(uint64_t)(uintptr_t)ctx->xmask, (uint64_t)(uintptr_t)ctx->xeff,
                            (uint64_t)(uintptr_t)ctx->xbase};
    TP_CU(cudaMemcpyAsync(ctx->xptrs, hp, sizeof(hp), cudaMemcpyHostToDevice, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));  // hp is a host stack array
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_flagged(tp_ctx* ctx, bool topology) {
    TpRange nvtx_range("tp_launch_flagged");
    const int nsup = (int)ctx->nsup;
    const int64_t nbits = (int64_t)nsup * nsup;
    if (topology) {
        TP_CU(cudaMemsetAsync(ctx->adjbm, 0, sizeof(unsigned) * ((nbits + 31) / 32), ctx->stream));
        TP_CU(cudaMemsetAsync(ctx->bmask, 0, sizeof(unsigned) * nbits * TP_BMASK_WORDS, ctx->stream));
        k_flag_pairs<<<blocks_for(ctx->nt, 256), 256, 0, ctx->stream>>>(ctx->F, ctx->perm, ctx->iperm, ctx->v2t_off,
                                                                        ctx->v2t, ctx->nt, nsup, ctx->adjbm,
                                                                        ctx->bmask);
        ++ctx->nlaunch;
        k_flag_diag<<<blocks_for(nsup, 256), 256, 0, ctx->stream>>>(nsup, ctx->adjbm);
        ++ctx->nlaunch;
    }
    TP_CU(cudaMemsetAsync(ctx->flagged, 0, sizeof(unsigned) * ((nbits + 31) / 32), ctx->stream));
    TP_CU(cudaMemsetAsync(ctx->mcount, 0, 10 * sizeof(int32_t), ctx->stream));
    k_tile_boxes<<<nsup, 256, 0, ctx->stream>>>(ctx->soa, ctx->ntp, ctx->nt, ctx->tbox);
    ++ctx->nlaunch;
    unsigned long long* npairs = reinterpret_cast<unsigned long long*>(ctx->mcount + 2);
    k_flag_classify<<<blocks_for(nbits, 256), 256, 0, ctx->stream>>>(ctx->adjbm, ctx->flagged, nsup, ctx->nt, ctx->tbox,
                                                                     ctx->bounds, TP_PRECISE_GAP_REL, ctx->mlist,
                                                                     ctx->plist, ctx->flist, ctx->mcount, npairs);
    ++ctx->nlaunch;
    int32_t h[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    TP_CU(cudaMemcpyAsync(h, ctx->mcount, 10 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->n_masked = h[0];
    ctx->n_precise = h[1];
    ctx->n_fast = h[8];
    unsigned long long p3[3];
    memcpy(p3, h + 2, sizeof(p3));
    ctx->pairs_fast = (int64_t)p3[0];
    ctx->pairs_precise = (int64_t)p3[1];
    ctx->pairs_masked_items = (int64_t)p3[2];
    if (ctx->n_masked > 1) {
        // a fixed order of the masked items (the exclusion bits are indexed by it)
        const int nm = (int)ctx->n_masked;
        int32_t* tmp = ctx->idx_tmp;  // nm <= nt
        // entries are I << 16 | J with I, J < 2^15: non-negative, so their unsigned order is theirs
        TP_TRY(tp_sort_pairs_u32(ctx, reinterpret_cast<const uint32_t*>(ctx->mlist), nullptr,
                                 reinterpret_cast<uint32_t*>(tmp), nullptr, nm, 31));
        TP_CU(cudaMemcpyAsync(ctx->mlist, tmp, sizeof(int32_t) * nm, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (topology) TP_TRY(tp_build_exclusion_bits(ctx));
    return TP_OK;
}

tp_status tp_ensure_flagged(tp_ctx* ctx) {
    TP_TRY(tp_ensure_sorted(ctx));
    if (ctx->flags_stale == 0) return TP_OK;
    TP_TRY(tp_launch_flagged(ctx, ctx->flags_stale >= 2));
    ctx->flags_stale = 0;
    return TP_OK;
}

namespace {
// Ordered excluded pairs: out[0] counts the distinct S != T sharing a vertex
// with T, out[1] those sharing an edge (two or more vertices), summed over T.
__global__ void k_count_excluded(const int32_t* __restrict__ F, const int32_t* __restrict__ off,
                                 const int32_t* __restrict__ v2t, int64_t nt, unsigned long long* __restrict__ out) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long cnt = 0, cnt_edge = 0;
    if (T < nt) {
        for (int c = 0; c < 3; ++c) {
            int32_t v = F[3 * T + c];
            for (int32_t e = off[v]; e < off[v + 1]; ++e) {
                int64_t S = v2t[e] >> 2;
                if (S == T) continue;
                // count S once: only at the first corner of T whose vertex S touches
                bool seen = false;
                for (int c2 = 0; c2 < c && !seen; ++c2) {
                    int32_t v2 = F[3 * T + c2];
                    seen = (F[3 * S] == v2) || (F[3 * S + 1] == v2) || (F[3 * S + 2] == v2);
                }
                if (seen) continue;
                ++cnt;
                int k = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) k += F[3 * T + i] == F[3 * S + j];
                if (k >= 2) ++cnt_edge;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        cnt_edge += __shfl_xor_sync(0xffffffffu, cnt_edge, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(out, cnt);
        if (cnt_edge) atomicAdd(out + 1, cnt_edge);
    }
}
}  // namespace

tp_status tp_count_excluded(tp_ctx* ctx) {
    TpRange nvtx_range("tp_count_excluded");
    unsigned long long* d = reinterpret_cast<unsigned long long*>(ctx->scalar + 8);
    TP_CU(cudaMemsetAsync(d, 0, 16, ctx->stream));
    k_count_excluded<<<blocks_for(ctx->nt, 256), 256, 0, ctx->stream>>>(ctx->F, ctx->v2t_off, ctx->v2t, ctx->nt, d);
    ++ctx->nlaunch;
    unsigned long long h[2] = {0, 0};
    TP_CU(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    ctx->n_excluded_ordered = (int64_t)h[0];
    ctx->n_excluded_edge_ordered = (int64_t)h[1];
    return TP_OK;
}
