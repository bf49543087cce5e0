// tp_adjoint.cu - pull-back of the per-triangle derivatives to the vertices
// and the FP64 reductions.
//
// The pair kernels leave, per triangle (library order), the accumulators
// Ew, U, Gn[3], Gx[3] (each carrying the factor p/q) from which
//     dPhi/dw_T  = Ew / ((p/q) w_T)
//     dPhi/dnu_T = q Gn / (p/q)
//     dPhi/dx_T  = q (Gx + U nu_T) / (p/q)
// (without the prefactor c).  The map (v0, v1, v2) -> (x_T, nu_T, w_T) has
//     x_T = (v0+v1+v2)/3,  N = e1 x e2 (e1 = v1-v0, e2 = v2-v0),
//     w_T = |N|/2,  nu_T = N/|N|,
// so with G = dPhi/dN = dPhi/dw nu/2 + (I - nu nu^T) dPhi/dnu / |N|:
//     dPhi/dv1 = e2 x G + dPhi/dx/3,  dPhi/dv2 = G x e1 + dPhi/dx/3,
//     dPhi/dv0 = -(e2 x G + G x e1) + dPhi/dx/3.
// This is the discrete counterpart of Eq. (dTP), Sec. 3.2 (the variation
// of the area element and of the normal under a vertex displacement).
// One thread per vertex gathers its incident triangles from the CSR list
// in a fixed order: deterministic, no atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"

namespace {

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// The chain rule of one element: its three corner contributions to dPhi/dV
// (corner c of element T at adjc[9 T + 3 c + a]), computed once per element.
__global__ void k_adjoint_tri(const double* __restrict__ V, const int32_t* __restrict__ F,
                              const int32_t* __restrict__ iperm, const double* __restrict__ nu64,
                              const double* __restrict__ w64, const double* __restrict__ acc, int64_t nt,
                              int64_t ntp, double qp, double ipq, double* __restrict__ adjc, tp_quad_rule rule) {
    const int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    const int64_t k = iperm[T];
    const double w = w64[T];
    double nu[3], gn[3], gx[3];
    for (int a = 0; a < 3; ++a) nu[a] = nu64[a * nt + T];
    // one division per element: the FP64 pipe is narrow, and reciprocals
    // change the result only in the last bits
    const double iw = 1.0 / w;
    const double Ew = acc[0 * ntp + k], U = acc[1 * ntp + k];
    const double gw = Ew * iw * ipq;  // Ew / (pq w)
    for (int a = 0; a < 3; ++a) {
        gn[a] = qp * acc[(2 + a) * ntp + k];
        gx[a] = qp * (acc[(5 + a) * ntp + k] + U * nu[a]);
    }
    const double* a0 = V + 3 * (int64_t)F[3 * T];
    const double* a1 = V + 3 * (int64_t)F[3 * T + 1];
    const double* a2 = V + 3 * (int64_t)F[3 * T + 2];
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = a1[a] - a0[a];
        e2[a] = a2[a] - a0[a];
    }
    // element weight w = om_q |N| / 2: dPhi/dN gets om_q dPhi/dw nu / 2 (om = 1 for the centroid rule)
    const int qi = rule.k > 1 ? (int)(T % rule.k) : 0;
    const double om = rule.k > 1 ? rule.w[qi] : 1.0;
    const double ilen = 0.5 * om * iw;  // 1 / |N|, |N| = 2 w / om
    const double ndg = nu[0] * gn[0] + nu[1] * gn[1] + nu[2] * gn[2];
    double G[3];
    for (int a = 0; a < 3; ++a) G[a] = 0.5 * om * gw * nu[a] + (gn[a] - nu[a] * ndg) * ilen;
    double c1[3], c2[3];
    cross3(e2, G, c1);  // dPhi/de1
    cross3(G, e1, c2);  // dPhi/de2
    double* out = adjc + 9 * T;
    for (int corner = 0; corner < 3; ++corner)
        for (int a = 0; a < 3; ++a) {
            // position x = sum_i l_i v_i: dPhi/dv_corner gets l_corner dPhi/dx (1/3 for the centroid)
            double t = rule.k > 1 ? rule.bary[qi][corner] * gx[a] : gx[a] * (1.0 / 3.0);
            if (corner == 0) t -= c1[a] + c2[a];
            else if (corner == 1) t += c1[a];
            else t += c2[a];
            out[3 * corner + a] = t;
        }
}

// dPhi/dV: per vertex, the corner contributions of its elements in the fixed
// order of the vertex -> element CSR (deterministic).
template <typename OutT>
__global__ void k_adjoint_gather(const int32_t* __restrict__ off, const int32_t* __restrict__ v2t,
                                 const double* __restrict__ adjc, int64_t nv, double scale,
                                 OutT* __restrict__ grad, int64_t nt, unsigned* __restrict__ derr) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double g[3] = {0.0, 0.0, 0.0};
    for (int32_t e = off[v]; e < off[v + 1]; ++e) {
        const int32_t ent = v2t[e];
        if (!tp_dbg_ok(ent >= 0 && (ent >> 2) < nt && (ent & 3) < 3, derr)) continue;
        const double* c = adjc + 9 * (int64_t)(ent >> 2) + 3 * (ent & 3);
        for (int a = 0; a < 3; ++a) g[a] += c[a];
    }
    for (int a = 0; a < 3; ++a) grad[3 * v + a] = (OutT)(scale * g[a]);
}

// Per-triangle derivatives in the caller's order, with w, nu and x taken as
// independent variables (the one-point counterparts of f_K, f_nu and f of
// Eq. (dTP_reordered), Sec. 3.2): fw [nt], fnu [nt][3], fx [nt][3].
__global__ void k_fields(const int32_t* __restrict__ iperm, const double* __restrict__ nu64,
                         const double* __restrict__ w64, const double* __restrict__ acc, int64_t nt, int64_t ntp,
                         double q, double pq, double scale, double* __restrict__ fw, double* __restrict__ fnu,
                         double* __restrict__ fx) {
    const int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    const int64_t k = iperm[T];
    const double U = acc[1 * ntp + k];
    if (fw) fw[T] = scale * acc[0 * ntp + k] / (pq * w64[T]);
    for (int a = 0; a < 3; ++a) {
        if (fnu) fnu[3 * T + a] = scale * q * acc[(2 + a) * ntp + k] / pq;
        if (fx) fx[3 * T + a] = scale * q * (acc[(5 + a) * ntp + k] + U * nu64[a * nt + T]) / pq;
    }
}

// deterministic two-pass sum of n doubles: fixed per-thread strides, fixed tree
__global__ void k_sum_partial(const double* __restrict__ in, int64_t n, int64_t stride, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += in[i * stride];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out = mul * (sum of the partials + *add), add may be null
__global__ void k_sum_final(const double* __restrict__ part, int nb, double mul, const double* __restrict__ add,
                            double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = mul * (sh[0] + (add ? *add : 0.0));
}

}  // namespace

tp_status tp_launch_adjoint(tp_ctx* ctx, const tp_params* prm, void* grad, int g_dtype) {
    TpRange nvtx_range("tp_launch_adjoint");
    const int64_t nv = ctx->nv, nt = ctx->nt;
    const double q = prm->q, pq = (double)prm->p / prm->q;
    if (nt > 0) {
        k_adjoint_tri<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->V64, ctx->F, ctx->iperm, ctx->nu64, ctx->w64, ctx->acc, nt, ctx->ntp, q / pq, 1.0 / pq, ctx->adjc,
            ctx->quad);
        ++ctx->nlaunch;
    }
    const unsigned blocks = (unsigned)((nv + 255) / 256);
    if (g_dtype == TP_DTYPE_F64)
        k_adjoint_gather<double><<<blocks, 256, 0, ctx->stream>>>(ctx->v2t_off, ctx->v2t, ctx->adjc, nv, prm->scale,
                                                                  static_cast<double*>(grad), nt, ctx->derr);
    else
        k_adjoint_gather<float><<<blocks, 256, 0, ctx->stream>>>(ctx->v2t_off, ctx->v2t, ctx->adjc, nv, prm->scale,
                                                                 static_cast<float*>(grad), nt, ctx->derr);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_fields(tp_ctx* ctx, const tp_params* prm, double* fw, double* fnu, double* fx) {
    TpRange nvtx_range("tp_launch_fields");
    const int64_t nt = ctx->nt;
    const double q = prm->q, pq = (double)prm->p / prm->q;
    k_fields<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(ctx->iperm, ctx->nu64, ctx->w64, ctx->acc, nt,
                                                                    ctx->ntp, q, pq, prm->scale, fw, fnu, fx);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

static tp_status reduce_strided(tp_ctx* ctx, const double* in, int64_t n, int64_t stride, double mul, double* d_out,
                                const double* add = nullptr) {
    const int nb = 512;
    double* part = ctx->red + (ctx->red_cap - nb);
    k_sum_partial<<<nb, 256, 0, ctx->stream>>>(in, n, stride, part);
    ++ctx->nlaunch;
    k_sum_final<<<1, 256, 0, ctx->stream>>>(part, nb, mul, add, d_out);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

// Phi = c * sum_T Ew_T / (2 p/q): every unordered pair adds (p/q)(e_TS + e_ST) to both ends.
// The learned form's energy-only correction (TP_LEARNED_ENERGY) is added to the sum.
tp_status tp_launch_energy_from_acc(tp_ctx* ctx, const tp_params* prm, double* d_out) {
    const double pq = (double)prm->p / prm->q;
    const bool eo = prm->mode == TP_LEARNED && (prm->flags & TP_LEARNED_ENERGY);
    return reduce_strided(ctx, ctx->acc, ctx->ntp, 1, prm->scale / (2.0 * pq), d_out, eo ? ctx->scalar + 6 : nullptr);
}

// mul * sum over triangles of the accumulator Ew
tp_status tp_launch_energy_scaled(tp_ctx* ctx, double mul, double* d_out) {
    return reduce_strided(ctx, ctx->acc, ctx->ntp, 1, mul, d_out);
}

tp_status tp_launch_reduce_sum(tp_ctx* ctx, const double* in, int64_t n, double* d_out) {
    return reduce_strided(ctx, in, n, 1, 1.0, d_out);
}

tp_status tp_launch_check_finite(tp_ctx* ctx) {
    (void)ctx;
    return TP_OK;
}
