// tp_tc.cu - the learned far field's network on the 5th-generation tensor
// cores: tcgen05.mma with operands in shared memory (UMMA descriptors, no
// swizzle, K-major core-matrix tiles), FP32 accumulators in tensor memory,
// one elected thread issuing and committing to an mbarrier, all four warps
// reading the accumulator back with tcgen05.ld for the epilogue.
//
// Network (24 -> 64 -> 64 -> 64 -> 7, tanh-form GELU, BF16 weights and
// activations, FP32 accumulation): per tile of 128 rows the CTA runs four
// MMA chains (K = 32, 64, 64, 64 in steps of 16; N = 64, 64, 64, 16) into
// one 64-column tensor-memory accumulator; between layers the 128 threads
// (thread = row = tensor-memory lane) add the bias, apply GELU, round to
// BF16 and store the row into the next layer's operand tile.
//
// Shared-memory operand layout (K-major, SWIZZLE_NONE): 8 x 8 BF16 core
// matrices of 128 contiguous bytes (8 rows of 16 bytes); element (r, k) at
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// SBO = 16 * K bytes; the descriptor's leading-dimension offset is the
// K-direction step between core matrices (128 B), the stride-dimension
// offset the step between 8-row groups (SBO); one MMA of K = 16 covers two
// core matrices along K, so successive K steps advance the start by 256 B.
//
// Waits are bounded: a wait that gives up sets a device error bit, waits
// again (bounded) for the MMAs in flight, frees the tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string.h>

#include "tp_internal.cuh"
#include "tp_mlp_dev.cuh"

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait for the given phase parity; false after TP_SPIN_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < TP_SPIN_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// byte offset of element (r, k) in a K-major core-matrix tile with K columns
__device__ __forceinline__ uint32_t tile_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (16 * K) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// copy a row-major BF16 matrix [rows][K] (global) into a core-matrix tile
__device__ __forceinline__ void load_tile(const __nv_bfloat16* g, int rows, int K, unsigned char* tile, int t, int nt) {
    const int chunks = rows * (K / 8);  // 16-byte pieces
    for (int i = t; i < chunks; i += nt) {
        const int r = i / (K / 8), kc = i % (K / 8);
        const uint4 v = *reinterpret_cast<const uint4*>(g + (size_t)r * K + kc * 8);
        *reinterpret_cast<uint4*>(tile + tile_off(r, kc * 8, K)) = v;
    }
}

}  // namespace

namespace {

// ------------------------------------------------------------ single GEMM (tests)
// D[128][N] = A[128][K] B[N][K]^T with one CTA: the operand layout, the
// descriptors and the accumulator read-back of the network kernel, checked
// on their own.
__global__ void __launch_bounds__(128) k_tc_gemm(const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ B, int K, int N,
                                                 float* __restrict__ D, unsigned* derr) {
    __shared__ __align__(128) unsigned char sA[128 * 64 * 2];
    __shared__ __align__(128) unsigned char sB[64 * 64 * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    load_tile(A, 128, K, sA, tid, 128);
    load_tile(B, N, K, sB, tid, 128);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(su32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init1(&mbar);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        for (int kk = 0; kk < K / 16; ++kk)
            tc_mma(tmem, umma_desc(su32(sA) + 256 * kk, 128, 16 * K), umma_desc(su32(sB) + 256 * kk, 128, 16 * K),
                   umma_idesc(128, N), kk > 0);
        tc_commit(&mbar);
    }
    const bool ok = mbar_wait(&mbar, 0);
    if (__syncthreads_or(!ok)) {  // the same decision in every thread
        if (tid == 0) tp_dev_error(derr, TP_DERR_TIMEOUT);
        mbar_wait(&mbar, 0);  // give the MMAs in flight a second bounded chance before freeing
    } else {
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        const int row = 32 * warp + lane;
        if (N == 64) {
            uint32_t r[64];
            tc_ld64(taddr, r);
            for (int c = 0; c < 64; ++c) D[row * 64 + c] = __uint_as_float(r[c]);
        } else {
            uint32_t r[16];
            tc_ld16(taddr, r);
            for (int c = 0; c < 16; ++c) D[row * 16 + c] = __uint_as_float(r[c]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
    }
}

// ------------------------------------------------------------ network kernel
struct TcSmem {
    unsigned char w1[64 * MLP_NIP * 2];  // W1 (N = 64, K = 32)
    unsigned char w2[64 * 64 * 2];       // W2
    unsigned char w3[64 * 64 * 2];       // W3
    unsigned char w4[16 * 64 * 2];       // W4 padded to N = 16
    // activations: the input tile (K = 32) and then each hidden layer's output
    // (K = 64) in place - a layer's MMAs have completed (mbarrier) before its
    // epilogue overwrites their A operand
    unsigned char act[128 * 64 * 2];
    float bias[MLPF_N];
    float norm[4 * MLP_NI];  // features: mean, 1/std, lower and upper admitted bound (FEAT)
    uint64_t mbar;
    uint32_t tmem;
};

// GELU of two pre-activations rounded to a BF16 pair: the tanh form of the
// training kernels (FP32 tanh.approx), with the polynomial and the final
// product in packed FP32 arithmetic.
__device__ __forceinline__ uint32_t gelu2_bf16(float z0, float z1) {
    const float c = 0.7978845608028654f, a = 0.044715f;
    const float2 z = make_float2(z0, z1);
    const float2 inner = __ffma2_rn(__fmul2_rn(z, z), make_float2(a, a), make_float2(1.f, 1.f));
    const float2 u = __fmul2_rn(__fmul2_rn(z, inner), make_float2(c, c));
    float2 t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.x) : "f"(u.x));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.y) : "f"(u.y));
    const float2 hz = __fmul2_rn(z, make_float2(0.5f, 0.5f));
    const float2 g = __ffma2_rn(hz, t, hz);
    return pack_bf16(g.x, g.y);
}

// bias + GELU on 64 accumulator columns of this thread's row, BF16 row into a K = 64 tile
__device__ __forceinline__ void epi_hidden(const uint32_t (&r)[64], const float* bias, unsigned char* tile, int row) {
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 8 * kc + 2 * j;
            w[j] = gelu2_bf16(__uint_as_float(r[c]) + bias[c], __uint_as_float(r[c + 1]) + bias[c + 1]);
        }
        *reinterpret_cast<uint4*>(tile + tile_off(row, 8 * kc, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Network on the rows of X ([rows][32] BF16 row-major, column 31 the
// training-range flag): kf[row][0..6] = exp(clamp(y, -4, 4)) - 1 (0 outside
// the ranges), kf[row][7] = the flag; with raw != 0 the outputs y themselves
// (kf[row][0..6]).  Persistent over 128-row tiles.
// FEAT: no X; the input row of window row r (listed row w0 + r) is built in
// the kernel from the feature records of its leaf and cluster
// (feature_row_bf16), so the rows never go through global memory.  The
// thread of a row loads the row's node indices one tile ahead.
template <bool FEAT>
__global__ void __launch_bounds__(128) k_mlp_tc(const __nv_bfloat16* __restrict__ wb,
                                                const float* __restrict__ bias_g,
                                                const __nv_bfloat16* __restrict__ X, int64_t rows,
                                                float* __restrict__ kf, int raw, unsigned* derr, tp_feat_src fs,
                                                int64_t w0) {
    extern __shared__ __align__(128) unsigned char tsm[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(tsm);
    const int tid = threadIdx.x, warp = tid >> 5;
    load_tile(wb + MLPB_W1, 64, MLP_NIP, S.w1, tid, 128);
    load_tile(wb + MLPB_W2, 64, 64, S.w2, tid, 128);
    load_tile(wb + MLPB_W3, 64, 64, S.w3, tid, 128);
    load_tile(wb + MLPB_W4, 16, 64, S.w4, tid, 128);
    for (int i = tid; i < MLPF_N; i += 128) S.bias[i] = bias_g[i];
    if (FEAT) {
        for (int i = tid; i < MLP_NI; i += 128) {
            const float lo = fs.mnorm[2 * MLP_NI + i], hi = fs.mnorm[3 * MLP_NI + i], pad = 0.05f * (hi - lo);
            S.norm[i] = fs.mnorm[i];
            S.norm[MLP_NI + i] = 1.0f / fs.mnorm[MLP_NI + i];
            S.norm[2 * MLP_NI + i] = lo - pad;
            S.norm[3 * MLP_NI + i] = hi + pad;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(su32(&S.tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init1(&S.mbar);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t sact = su32(S.act);
    const uint32_t id64 = umma_idesc(128, 64), id16 = umma_idesc(128, 16);
    uint32_t phase = 0;
    bool failed = false;
    const int64_t ntiles = (rows + 127) / 128;
    // this thread's input row of a tile (zero past the end), loaded one tile ahead
    auto load_row = [&](int64_t t, uint4 (&v)[4]) {
        const int64_t r = 128 * t + tid;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_uint4(0, 0, 0, 0);
        if (t < ntiles && r < rows) {
            const uint4* src = reinterpret_cast<const uint4*>(X + r * MLP_NIP);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = src[q];
        }
    };
    // FEAT: the node indices (leaf list index, cluster) of this thread's row of a tile, -1 past the end
    auto load_idx = [&](int64_t t, int& lf, int& cn) {
        const int64_t r = 128 * t + tid;
        lf = cn = -1;
        if (t < ntiles && r < rows) {
            lf = fs.far_leaf[w0 + r];
            cn = fs.far_list[w0 + r];
            if (!tp_dbg_ok(lf >= 0 && lf < fs.nleaves && cn >= 0 && cn < fs.nnodes, derr)) lf = cn = -1;
        }
    };
    auto feat_row = [&](int ln, int cn, uint4 (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_uint4(0, 0, 0, 0);
        if (cn < 0) return;
        float fl[16], cr[16];
        const float4* pl = reinterpret_cast<const float4*>(fs.nodeft + 16 * (int64_t)ln);
        const float4* pc = reinterpret_cast<const float4*>(fs.nodeft + 16 * (int64_t)cn);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = pl[q], b = pc[q];
            fl[4 * q] = a.x;
            fl[4 * q + 1] = a.y;
            fl[4 * q + 2] = a.z;
            fl[4 * q + 3] = a.w;
            cr[4 * q] = b.x;
            cr[4 * q + 1] = b.y;
            cr[4 * q + 2] = b.z;
            cr[4 * q + 3] = b.w;
        }
        uint32_t pk[16];
        feature_row_bf16(fl, cr, S.norm, pk);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    };
    // FEAT: the node indices of the next tile's row are loaded at the start of
    // a tile and its leaf after the first layer; the row itself is built at
    // the start of its tile (building it during the second layer's MMAs needed
    // 110 registers, and spills at 96: both slower)
    int lf_next = -1, c_next = -1, l_next = -1;
    uint4 vnext[4];
    if (FEAT) {
        load_idx(blockIdx.x, lf_next, c_next);
        l_next = c_next >= 0 ? fs.leaves[lf_next] : -1;
        if (!tp_dbg_ok(l_next < fs.nnodes, derr)) c_next = -1;
    } else {
        load_row(blockIdx.x, vnext);
    }
    for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
        const int64_t row = 128 * t + tid;
        uint4 v[4];
        if (FEAT) {
            feat_row(l_next, c_next, v);
            load_idx(t + gridDim.x, lf_next, c_next);  // in flight during this tile's first layer
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = vnext[q];
            load_row(t + gridDim.x, vnext);  // in flight during this tile's layers
        }
        const bool in_dist = (v[3].w >> 16) != 0u;  // column 31
#pragma unroll
        for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(S.act + tile_off(tid, 8 * q, MLP_NIP)) = v[q];
        uint32_t r[64];
        // layers 1..3: GELU epilogues into the hidden tiles
#pragma unroll 1
        for (int layer = 0; layer < 3 && !failed; ++layer) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const int K = layer == 0 ? MLP_NIP : 64;
                const uint32_t b0 = su32(layer == 0 ? S.w1 : (layer == 1 ? S.w2 : S.w3));
                for (int kk = 0; kk < K / 16; ++kk)
                    tc_mma(tmem, umma_desc(sact + 256 * kk, 128, 16 * K), umma_desc(b0 + 256 * kk, 128, 16 * K),
                           id64, kk > 0);
                tc_commit(&S.mbar);
            }
            if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) {  // the same decision in every thread
                failed = true;
                break;
            }
            phase ^= 1u;
            tc_fence_after();
            tc_ld64(taddr, r);
            epi_hidden(r, S.bias + 64 * layer, S.act, tid);
            if (FEAT && layer == 0) {
                l_next = c_next >= 0 ? fs.leaves[lf_next] : -1;  // in flight until the next tile
                if (!tp_dbg_ok(l_next < fs.nnodes, derr)) c_next = -1;
            }
        }
        if (failed) break;
        // output layer (N = 16, rows 7..15 of W4 zero)
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int kk = 0; kk < 4; ++kk)
                tc_mma(tmem, umma_desc(sact + 256 * kk, 128, 1024), umma_desc(su32(S.w4) + 256 * kk, 128, 1024),
                       id16, kk > 0);
            tc_commit(&S.mbar);
        }
        if (__syncthreads_or(!mbar_wait(&S.mbar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        uint32_t y[16];
        tc_ld16(taddr, y);
        if (row < rows) {
            float o[8];
#pragma unroll
            for (int c = 0; c < MLP_NO; ++c) {
                const float yc = __uint_as_float(y[c]) + S.bias[MLPF_B4 + c];
                o[c] = raw ? yc : (in_dist ? __expf(fminf(4.f, fmaxf(-4.f, yc))) - 1.f : 0.f);
            }
            o[7] = in_dist ? 1.f : 0.f;
            float4* dst = reinterpret_cast<float4*>(kf + row * 8);
            dst[0] = make_float4(o[0], o[1], o[2], o[3]);
            dst[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
        tc_fence_before();
        __syncthreads();  // the tiles and the accumulator are reused by the next tile
        tc_fence_after();
    }
    if (failed) {
        if (tid == 0) tp_dev_error(derr, TP_DERR_TIMEOUT);
        mbar_wait(&S.mbar, phase);  // second bounded wait for the MMAs in flight
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

tp_status tp_launch_mlp_tc(tp_ctx* ctx, const __nv_bfloat16* wb, const float* bias, const __nv_bfloat16* X,
                           int64_t rows, float* kf, int raw) {
    TpRange nvtx_range("tp_launch_mlp_tc");
    // per-device attribute: set on the current device at every launch
    TP_CU(cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem)));
    const int64_t ntiles = (rows + 127) / 128;
    if (ntiles == 0) return TP_OK;
    // about 40 KB of shared memory and 64 tensor-memory columns per CTA: 5 CTAs per SM
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * 5);
    tp_feat_src none;
    memset(&none, 0, sizeof(none));
    k_mlp_tc<false><<<grid, 128, sizeof(TcSmem), ctx->stream>>>(wb, bias, X, rows, kf, raw, ctx->derr, none, 0);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_launch_mlp_tc_feat(tp_ctx* ctx, const __nv_bfloat16* wb, const float* bias, const tp_feat_src& fs,
                                int64_t w0, int64_t w1, float* kf) {
    TpRange nvtx_range("tp_launch_mlp_tc_feat");
    TP_CU(cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem)));
    const int64_t rows = w1 - w0;
    const int64_t ntiles = (rows + 127) / 128;
    if (ntiles <= 0) return TP_OK;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * 5);
    k_mlp_tc<true><<<grid, 128, sizeof(TcSmem), ctx->stream>>>(wb, bias, nullptr, rows, kf, 0, ctx->derr, fs, w0);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

extern "C" tp_status tp_debug_tc_gemm(int device, const uint16_t* A, int K, const uint16_t* B, int N, float* D) {
    if (!A || !B || !D || !(K == 16 || K == 32 || K == 64) || !(N == 16 || N == 64)) return TP_E_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return TP_E_CUDA;
    __nv_bfloat16 *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    unsigned* derr = nullptr;
    tp_status st = TP_OK;
    if (cudaMalloc(&dA, 2 * 128 * K) != cudaSuccess || cudaMalloc(&dB, 2 * N * K) != cudaSuccess ||
        cudaMalloc(&dD, 4 * 128 * N) != cudaSuccess || cudaMalloc(&derr, 4) != cudaSuccess) {
        st = TP_E_OOM;
    } else {
        cudaMemcpy(dA, A, 2 * 128 * K, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, 2 * N * K, cudaMemcpyHostToDevice);
        cudaMemset(derr, 0, 4);
        k_tc_gemm<<<1, 128>>>(dA, dB, K, N, dD, derr);
        unsigned h = 0;
        if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) st = TP_E_CUDA;
        else {
            cudaMemcpy(D, dD, 4 * 128 * N, cudaMemcpyDeviceToHost);
            cudaMemcpy(&h, derr, 4, cudaMemcpyDeviceToHost);
            if (h) st = TP_E_TIMEOUT;
        }
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    return st;
}
