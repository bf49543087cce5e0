// tp_peak.cu - FP32 throughput probe: long chains of independent FMAs, scalar
// (FFMA) or packed (FP32x2 FFMA2), at a chosen occupancy.  It gives the
// measured counterpart of the FP32 peak derived from unit counts and clock
// (SMs x 128 lanes x 2 flops x clock) that the pair kernels are compared
// with, and shows what occupancy and instruction-level parallelism the FP32
// pipe needs.  No memory traffic beyond one conditional store per thread.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp.h"

namespace {

template <bool PACKED, int C>
__global__ void k_fp32_peak(float* out, int iters, float m, float c) {
    const float s = 1e-3f * (float)(threadIdx.x & 63);
    if (PACKED) {
        float2 a[C];
        const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll
        for (int i = 0; i < C; ++i) a[i] = make_float2(s + i, s - i);
#pragma unroll 4
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int i = 0; i < C; ++i) a[i] = __ffma2_rn(a[i], m2, c2);
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < C; ++i) t += a[i].x + a[i].y;
        if (t == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = t;
    } else {
        float a[C];
#pragma unroll
        for (int i = 0; i < C; ++i) a[i] = s + i;
#pragma unroll 4
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int i = 0; i < C; ++i) a[i] = __fmaf_rn(a[i], m, c);
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < C; ++i) t += a[i];
        if (t == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = t;
    }
}

template <bool PACKED>
void launch(int chains, dim3 g, dim3 b, cudaStream_t st, float* out, int iters) {
    const float m = 0.9999f, c = 1e-4f;
    switch (chains) {
        case 2: k_fp32_peak<PACKED, 2><<<g, b, 0, st>>>(out, iters, m, c); break;
        case 4: k_fp32_peak<PACKED, 4><<<g, b, 0, st>>>(out, iters, m, c); break;
        case 8: k_fp32_peak<PACKED, 8><<<g, b, 0, st>>>(out, iters, m, c); break;
        default: k_fp32_peak<PACKED, 16><<<g, b, 0, st>>>(out, iters, m, c); break;
    }
}

}  // namespace

extern "C" tp_status tp_measure_fp32_peak(int device, void* cuda_stream, int packed, int warps_per_sm, int chains,
                                          double* tflops_out) {
    if (!tflops_out || warps_per_sm < 1 || warps_per_sm > 64 ||
        !(chains == 2 || chains == 4 || chains == 8 || chains == 16))
        return TP_E_ARG;
    *tflops_out = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) return TP_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TP_E_CUDA;
    // blocks of at most 8 warps, enough blocks for warps_per_sm resident warps on every SM
    const int wpb = warps_per_sm < 8 ? warps_per_sm : 8;
    const int bps = (warps_per_sm + wpb - 1) / wpb;
    const dim3 b(32 * wpb), g(sms * bps);
    // about 2^21 FP32 FMAs per thread at 64 warps per SM, scaled up at lower occupancy
    const int iters = (1 << 17) / chains * (64 / (bps * wpb) > 0 ? 64 / (bps * wpb) : 1);
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)g.x * b.x) != cudaSuccess) return TP_E_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    tp_status status = TP_OK;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (packed) launch<true>(chains, g, b, st, out, iters);
        else launch<false>(chains, g, b, st, out, iters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            status = TP_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // one FMA = 2 flops; a packed FMA = 2 FMAs
        const double flops = 2.0 * (packed ? 2.0 : 1.0) * chains * (double)iters * g.x * b.x;
        if (rep > 0 && ms > 0.f) best = best > flops / (ms * 1e9) ? best : flops / (ms * 1e9);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *tflops_out = best;
    return status;
}
