// tp_noalloc.cu - direct energy and gradient that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// energy: code that records a CUDA graph (allocation calls are not allowed
// while a stream is being captured), plug-ins living inside a host
// application that hands out all device memory through its own pool, and
// control loops that forbid allocation once they are running.  For them
// tp_gradient_direct_noalloc takes device inputs and device outputs and
// keeps its scratch in one file-scope __device__ array of fixed size,
// TP_NOALLOC_MAX_TRIS triangles (about 7 MB, held by every GPU that loads
// the library until the process exits).
//
// The scratch address is looked up once per device with
// cudaGetSymbolAddress, on the first call made with that device current;
// make that first call before any stream capture starts.  The address is
// kept for the life of the process, which assumes the device's primary
// context is never reset (cudaDeviceReset) and is the context in use.
// Every call uses the same array: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it and give wrong
// results.
// Every scratch entry a call reads is written by that call first, so the
// contents left by an earlier call do not matter.
//
// Method: the same discrete energy and exact gradient as tp_gradient in
// TP_DIRECT mode (FP32 pair terms, FP64 accumulation), organised as a
// gather (one thread per target triangle, both orderings of every pair)
// instead of the symmetric tiled kernel, followed by a per-triangle
// pull-back to the vertices with FP64 atomic adds into the caller's output.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "tp_internal.cuh"

#define TP_NOALLOC_MAX_TRIS 65536
#define TP_NOALLOC_MAX_DEVICES 64
#define TP_NOALLOC_TILE 128
#define TP_NOALLOC_NPART 256

namespace {

// scratch: 10 f32 planes (x_hi[3], x_lo[3], nu[3], w) + 8 f64 accumulator
// planes per triangle + the energy partials
constexpr size_t NA_SOA_BYTES = (size_t)10 * TP_NOALLOC_MAX_TRIS * sizeof(float);
constexpr size_t NA_ACC_BYTES = (size_t)8 * TP_NOALLOC_MAX_TRIS * sizeof(double);
constexpr size_t NA_PART_BYTES = (size_t)TP_NOALLOC_NPART * sizeof(double);
constexpr size_t NA_BYTES = NA_SOA_BYTES + NA_ACC_BYTES + NA_PART_BYTES;

__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mutex;
void* g_na_ptr[TP_NOALLOC_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ float na_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int na_shared(int a0, int a1, int a2, int b0, int b1, int b2) {
    return (a0 == b0) + (a0 == b1) + (a0 == b2) + (a1 == b0) + (a1 == b1) + (a1 == b2) + (a2 == b0) + (a2 == b1) +
           (a2 == b2);
}

// per-triangle data: centroid split into f32 hi + lo, unit normal, area
__global__ void k_na_tri(const double* __restrict__ V, const int32_t* __restrict__ F, int64_t nt, int64_t nv,
                         float* __restrict__ soa) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    if (F[3 * T] < 0 || F[3 * T] >= nv || F[3 * T + 1] < 0 || F[3 * T + 1] >= nv || F[3 * T + 2] < 0 ||
        F[3 * T + 2] >= nv) {
        // an index outside [0, nv): poison this triangle so the energy comes out NaN
        for (int k = 0; k < 10; ++k) soa[k * TP_NOALLOC_MAX_TRIS + T] = __int_as_float(0x7fc00000);
        return;
    }
    const double* a = V + 3 * (int64_t)F[3 * T];
    const double* b = V + 3 * (int64_t)F[3 * T + 1];
    const double* c = V + 3 * (int64_t)F[3 * T + 2];
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        double x = ((a[k] + b[k]) + c[k]) / 3.0;
        float hi = (float)x;
        soa[k * TP_NOALLOC_MAX_TRIS + T] = hi;
        soa[(3 + k) * TP_NOALLOC_MAX_TRIS + T] = (float)(x - (double)hi);
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
    double N0 = e1[1] * e2[2] - e1[2] * e2[1];
    double N1 = e1[2] * e2[0] - e1[0] * e2[2];
    double N2 = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(N0 * N0 + N1 * N1 + N2 * N2);
    soa[6 * TP_NOALLOC_MAX_TRIS + T] = (float)(N0 / len);
    soa[7 * TP_NOALLOC_MAX_TRIS + T] = (float)(N1 / len);
    soa[8 * TP_NOALLOC_MAX_TRIS + T] = (float)(N2 / len);
    soa[9 * TP_NOALLOC_MAX_TRIS + T] = (float)(0.5 * len);
}

// gather: target T against every admitted S, both orderings, T-side derivatives
template <int Q>
__global__ void __launch_bounds__(TP_NOALLOC_TILE) k_na_pairs(const float* __restrict__ soa,
                                                               const int32_t* __restrict__ F, int64_t nt,
                                                               int edge_only, double* __restrict__ acc) {
    __shared__ float sd[10][TP_NOALLOC_TILE];
    __shared__ int sf[3][TP_NOALLOC_TILE];
    const int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = T < nt;
    float t[10];
    int f0 = -1, f1 = -1, f2 = -1;
    for (int k = 0; k < 10; ++k) t[k] = active ? soa[k * TP_NOALLOC_MAX_TRIS + T] : 0.f;
    if (active) {
        f0 = F[3 * T];
        f1 = F[3 * T + 1];
        f2 = F[3 * T + 2];
    }
    const float lam = 2.0f;  // p / q with p = 2q
    double Ew = 0, U = 0, Gn[3] = {0, 0, 0}, Gx[3] = {0, 0, 0};
    for (int64_t s0 = 0; s0 < nt; s0 += TP_NOALLOC_TILE) {
        __syncthreads();
        const int64_t S = s0 + threadIdx.x;
        for (int k = 0; k < 10; ++k) sd[k][threadIdx.x] = S < nt ? soa[k * TP_NOALLOC_MAX_TRIS + S] : 0.f;
        sf[0][threadIdx.x] = S < nt ? F[3 * S] : -1;
        sf[1][threadIdx.x] = S < nt ? F[3 * S + 1] : -1;
        sf[2][threadIdx.x] = S < nt ? F[3 * S + 2] : -1;
        __syncthreads();
        if (!active) continue;
        const int m = (nt - s0) < TP_NOALLOC_TILE ? (int)(nt - s0) : TP_NOALLOC_TILE;
        float ew = 0.f, u = 0.f, gn0 = 0.f, gn1 = 0.f, gn2 = 0.f, gx0 = 0.f, gx1 = 0.f, gx2 = 0.f;
        for (int j = 0; j < m; ++j) {
            if (s0 + j == T) continue;
            int sh = na_shared(f0, f1, f2, sf[0][j], sf[1][j], sf[2][j]);
            if (edge_only ? sh >= 2 : sh >= 1) continue;
            float d0 = (t[0] - sd[0][j]) + (t[3] - sd[3][j]);
            float d1 = (t[1] - sd[1][j]) + (t[4] - sd[4][j]);
            float d2 = (t[2] - sd[2][j]) + (t[5] - sd[5][j]);
            float inv = na_rcp(d0 * d0 + d1 * d1 + d2 * d2);
            float a = t[6] * d0 + t[7] * d1 + t[8] * d2;
            float b = sd[6][j] * d0 + sd[7][j] * d1 + sd[8][j] * d2;
            float al = a * inv, be = b * inv;
            float al2 = al * al, be2 = be * be;
            float alq, beq, al5, be5;
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
            float wts = lam * t[9] * sd[9][j];
            float s6 = alq + beq;
            float wi = wts * inv;
            float A5 = wi * al5, B5 = wi * be5, k = lam * wi * s6;
            ew += wts * s6;
            u += A5;
            gn0 += A5 * d0;
            gn1 += A5 * d1;
            gn2 += A5 * d2;
            gx0 += B5 * sd[6][j] - k * d0;
            gx1 += B5 * sd[7][j] - k * d1;
            gx2 += B5 * sd[8][j] - k * d2;
        }
        Ew += ew;
        U += u;
        Gn[0] += gn0;
        Gn[1] += gn1;
        Gn[2] += gn2;
        Gx[0] += gx0;
        Gx[1] += gx1;
        Gx[2] += gx2;
    }
    if (!active) return;
    acc[0 * TP_NOALLOC_MAX_TRIS + T] = Ew;
    acc[1 * TP_NOALLOC_MAX_TRIS + T] = U;
    for (int k = 0; k < 3; ++k) {
        acc[(2 + k) * TP_NOALLOC_MAX_TRIS + T] = Gn[k];
        acc[(5 + k) * TP_NOALLOC_MAX_TRIS + T] = Gx[k];
    }
}

// pull-back of one triangle's derivatives to its three vertices (FP64 atomics)
__global__ void k_na_adjoint(const double* __restrict__ V, const int32_t* __restrict__ F, int64_t nt, int64_t nv,
                             const double* __restrict__ acc, double q, double lam, double scale,
                             double* __restrict__ grad) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= nt) return;
    const int64_t i0 = F[3 * T], i1 = F[3 * T + 1], i2 = F[3 * T + 2];
    if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) return;
    const double *a = V + 3 * i0, *b = V + 3 * i1, *c = V + 3 * i2;
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = b[k] - a[k];
        e2[k] = c[k] - a[k];
    }
    double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    double nu[3] = {N[0] / len, N[1] / len, N[2] / len};
    double w = 0.5 * len;
    double gw = acc[T] / (lam * w);
    double U = acc[TP_NOALLOC_MAX_TRIS + T];
    double gn[3], gx[3];
    for (int k = 0; k < 3; ++k) {
        gn[k] = q * acc[(2 + k) * TP_NOALLOC_MAX_TRIS + T] / lam;
        gx[k] = q * (acc[(5 + k) * TP_NOALLOC_MAX_TRIS + T] + U * nu[k]) / lam;
    }
    double ndg = nu[0] * gn[0] + nu[1] * gn[1] + nu[2] * gn[2];
    double G[3];
    for (int k = 0; k < 3; ++k) G[k] = 0.5 * gw * nu[k] + (gn[k] - nu[k] * ndg) / len;
    double c1[3] = {e2[1] * G[2] - e2[2] * G[1], e2[2] * G[0] - e2[0] * G[2], e2[0] * G[1] - e2[1] * G[0]};
    double c2[3] = {G[1] * e1[2] - G[2] * e1[1], G[2] * e1[0] - G[0] * e1[2], G[0] * e1[1] - G[1] * e1[0]};
    for (int k = 0; k < 3; ++k) {
        double t = gx[k] / 3.0;
        atomicAdd(&grad[3 * i0 + k], scale * (t - c1[k] - c2[k]));
        atomicAdd(&grad[3 * i1 + k], scale * (t + c1[k]));
        atomicAdd(&grad[3 * i2 + k], scale * (t + c2[k]));
    }
}

// energy: Phi = scale * sum_T Ew_T / (2 lam), deterministic two-pass sum
__global__ void k_na_energy_part(const double* __restrict__ acc, int64_t nt, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x)
        s += acc[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_na_energy_final(const double* __restrict__ part, int nb, double mul, double* __restrict__ out) {
    __shared__ double sh[256];
    sh[threadIdx.x] = threadIdx.x < nb ? part[threadIdx.x] : 0.0;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = mul * sh[0];
}

tp_status na_err(char* buf, int64_t len, tp_status s, const char* msg) {
    if (buf && len > 0) snprintf(buf, (size_t)len, "%s", msg);
    return s;
}

}  // namespace

extern "C" tp_status tp_gradient_direct_noalloc(const double* V, int64_t nv, const int32_t* F, int64_t nt,
                                                const tp_params* params, double* energy_out, double* grad_out,
                                                void* cuda_stream, char* errbuf, int64_t errbuf_len) {
    if (errbuf && errbuf_len > 0) errbuf[0] = '\0';
    if (!params) return na_err(errbuf, errbuf_len, TP_E_ARG, "params is NULL");
    if (!((params->q == 6 && params->p == 12) || (params->q == 8 && params->p == 16)))
        return na_err(errbuf, errbuf_len, TP_E_ARG, "unsupported exponents (supported: q=6 p=12, q=8 p=16)");
    if (params->mode != TP_DIRECT) return na_err(errbuf, errbuf_len, TP_E_ARG, "only TP_DIRECT is available here");
    if (params->prec != TP_F32_F64ACC)
        return na_err(errbuf, errbuf_len, TP_E_ARG, "only TP_F32_F64ACC (FP32 pair terms, FP64 sums) is available here");
    if (nv < 0 || nt < 0) return na_err(errbuf, errbuf_len, TP_E_ARG, "negative size");
    if (nt > TP_NOALLOC_MAX_TRIS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "nt=%lld exceeds the maximum of %d triangles of the allocation-free path",
                 (long long)nt, TP_NOALLOC_MAX_TRIS);
        return na_err(errbuf, errbuf_len, TP_E_ARG, msg);
    }
    if (!energy_out || (nv > 0 && !grad_out) || (nt > 0 && (!V || !F)))
        return na_err(errbuf, errbuf_len, TP_E_ARG, "null input or output pointer");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TP_NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return na_err(errbuf, errbuf_len, TP_E_CUDA, "no usable current CUDA device");
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_err(errbuf, errbuf_len, TP_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_na_ptr[dev] = p;
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float* soa = reinterpret_cast<float*>(base);
    double* acc = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + NA_SOA_BYTES);
    double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + NA_SOA_BYTES + NA_ACC_BYTES);
    if (nv > 0 && cudaMemsetAsync(grad_out, 0, sizeof(double) * 3 * nv, st) != cudaSuccess) {
        cudaGetLastError();
        return na_err(errbuf, errbuf_len, TP_E_CUDA, "cudaMemsetAsync of grad_out failed");
    }
    if (nt == 0) {
        if (cudaMemsetAsync(energy_out, 0, sizeof(double), st) != cudaSuccess) {
            cudaGetLastError();
            return na_err(errbuf, errbuf_len, TP_E_CUDA, "cudaMemsetAsync of energy_out failed");
        }
        return TP_OK;
    }
    const int edge = (params->flags & TP_EXCLUDE_EDGE) ? 1 : 0;
    const double lam = (double)params->p / params->q;
    const unsigned nb = (unsigned)((nt + TP_NOALLOC_TILE - 1) / TP_NOALLOC_TILE);
    k_na_tri<<<nb, TP_NOALLOC_TILE, 0, st>>>(V, F, nt, nv, soa);
    if (params->q == 6)
        k_na_pairs<6><<<nb, TP_NOALLOC_TILE, 0, st>>>(soa, F, nt, edge, acc);
    else
        k_na_pairs<8><<<nb, TP_NOALLOC_TILE, 0, st>>>(soa, F, nt, edge, acc);
    k_na_adjoint<<<nb, TP_NOALLOC_TILE, 0, st>>>(V, F, nt, nv, acc, (double)params->q, lam, params->scale, grad_out);
    k_na_energy_part<<<TP_NOALLOC_NPART, 256, 0, st>>>(acc, nt, part);
    k_na_energy_final<<<1, 256, 0, st>>>(part, TP_NOALLOC_NPART, params->scale / (2.0 * lam), energy_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_err(errbuf, errbuf_len, TP_E_CUDA, cudaGetErrorString(e));
    return TP_OK;
}
