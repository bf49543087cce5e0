// tp_capi.cu - the C ABI declared in include/tp.h and the host orchestration
// behind it (buffers, kernel sequencing, error status).
//
// The calls follow the paper's statement of the problem: given the surface
// (a parametrisation X, here the vertex positions of a flat triangle mesh)
// return Phi(X) (Eq. TP, Sec. 2.2.2) and the variation dPhi/dX (Eq. dTP,
// Sec. 3.2), either by the full double sum ("full integration", Sec. 3.2) or
// with the inner integral clustered (Barnes-Hut, Sec. 3.2).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "tp_internal.cuh"

#define TP_VERSION_STR "tpgpu 0.1 (sm_103a)"

tp_status tp_set_err(tp_ctx* c, tp_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

tp_status tp_cuda_check(tp_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return tp_set_err(c, TP_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return tp_set_err(c, TP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

tp_status tp_alloc(tp_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->fail_alloc_after >= 0) {
        if (ctx->fail_alloc_after == 0) {
            ctx->fail_alloc_after = -1;
            tp_drop_mesh_state(ctx);
            *p = nullptr;
            return tp_set_err(ctx, TP_E_OOM, "allocation of %zu bytes failed (simulated by tp_debug_fail_alloc)", bytes);
        }
        --ctx->fail_alloc_after;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        tp_drop_mesh_state(ctx);
        *p = nullptr;
        return tp_set_err(ctx, TP_E_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    ctx->allocs.push_back(*p);
    return TP_OK;
}

void tp_free(tp_ctx* ctx, void* p) {
    if (!p) return;
    for (size_t i = 0; i < ctx->allocs.size(); ++i)
        if (ctx->allocs[i] == p) {
            ctx->allocs[i] = ctx->allocs.back();
            ctx->allocs.pop_back();
            break;
        }
    cudaFree(p);
}

namespace {

template <typename T>
void free_ptr(tp_ctx* ctx, T*& p) {
    tp_free(ctx, (void*)p);
    p = nullptr;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_check_finite_v(const double* __restrict__ V, int64_t n, unsigned* derr) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(V[i])) tp_dev_error(derr, TP_DERR_NONFINITE);
}

tp_status check_params(tp_ctx* ctx, const tp_params* prm) {
    if (!prm) return tp_set_err(ctx, TP_E_ARG, "params is NULL");
    if (!((prm->q == 6 && prm->p == 12) || (prm->q == 8 && prm->p == 16)))
        return tp_set_err(ctx, TP_E_ARG, "unsupported exponents q=%d p=%d (supported: 6/12, 8/16)", prm->q, prm->p);
    if (prm->mode < TP_DIRECT || prm->mode > TP_BH_DUAL) return tp_set_err(ctx, TP_E_ARG, "bad mode %d", prm->mode);
    if (prm->prec < TP_F32_F64ACC || prm->prec > TP_F64) return tp_set_err(ctx, TP_E_ARG, "bad prec %d", prm->prec);
    if (!std::isfinite(prm->scale)) return tp_set_err(ctx, TP_E_ARG, "scale is not finite");
    if (prm->mode != TP_DIRECT && !(prm->theta >= 0.0 && std::isfinite(prm->theta)))
        return tp_set_err(ctx, TP_E_ARG, "theta must be finite and >= 0");
    if (prm->mode != TP_DIRECT && prm->prec != TP_F32_F64ACC)
        return tp_set_err(ctx, TP_E_ARG, "the clustered forms evaluate FP32 terms with FP64 sums only (prec %d)",
                          prm->prec);
    if (!ctx->have_mesh) return tp_set_err(ctx, TP_E_STATE, "no mesh uploaded");
    if (prm->mode != TP_DIRECT && !ctx->tree.valid && ctx->nt > 0)
        return tp_set_err(ctx, TP_E_STATE, "mode %d needs tp_tree_build first", prm->mode);
    if (prm->mode == TP_LEARNED && !tp_mlp_ready(ctx))
        return tp_set_err(ctx, TP_E_STATE, "TP_LEARNED needs a far-field model (tp_far_model_load)");
    return TP_OK;
}


void release_mesh(tp_ctx* ctx) {
    free_ptr(ctx, ctx->V64);
    free_ptr(ctx, ctx->F);
    free_ptr(ctx, ctx->v2t_off);
    free_ptr(ctx, ctx->v2t);
    free_ptr(ctx, ctx->x64);
    free_ptr(ctx, ctx->nu64);
    free_ptr(ctx, ctx->w64);
    free_ptr(ctx, ctx->perm);
    free_ptr(ctx, ctx->iperm);
    free_ptr(ctx, ctx->codes);
    free_ptr(ctx, ctx->codes_sorted);
    free_ptr(ctx, ctx->idx_tmp);
    free_ptr(ctx, ctx->soa);
    free_ptr(ctx, ctx->src);
    free_ptr(ctx, ctx->Fs);
    free_ptr(ctx, ctx->acc);
    free_ptr(ctx, ctx->adjc);
    free_ptr(ctx, ctx->red);
    free_ptr(ctx, ctx->flagged);
    free_ptr(ctx, ctx->adjbm);
    free_ptr(ctx, ctx->bmask);
    free_ptr(ctx, ctx->mlist);
    free_ptr(ctx, ctx->item_index);
    free_ptr(ctx, ctx->xeff);
    free_ptr(ctx, ctx->xbase);
    free_ptr(ctx, ctx->xcount);
    free_ptr(ctx, ctx->xmask);
    free_ptr(ctx, ctx->xptrs);
    ctx->x_cap = ctx->x_item_cap = ctx->x_slots = 0;
    free_ptr(ctx, ctx->plist);
    free_ptr(ctx, ctx->flist);
    free_ptr(ctx, ctx->tbox);
    free_ptr(ctx, ctx->gradbuf);
    free_ptr(ctx, ctx->fieldbuf);
    free_ptr(ctx, ctx->F_tri);
    free_ptr(ctx, ctx->vtmp);
    tp_tree& t = ctx->tree;
    free_ptr(ctx, t.codes);
    free_ptr(ctx, t.left);
    free_ptr(ctx, t.right);
    free_ptr(ctx, t.parent);
    free_ptr(ctx, t.first);
    free_ptr(ctx, t.last);
    free_ptr(ctx, t.leaves);
    free_ptr(ctx, t.counter);
    free_ptr(ctx, t.mom);
    free_ptr(ctx, t.box);
    free_ptr(ctx, t.nodef);
    free_ptr(ctx, t.adm64);
    free_ptr(ctx, t.adm32);
    free_ptr(ctx, t.nodeft);
    t.valid = false;
    t.cap = 0;
    ctx->cap_nv = ctx->cap_nt = 0;
    ctx->have_mesh = false;
}

}  // namespace

void tp_drop_mesh_state(tp_ctx* ctx) {
    release_mesh(ctx);
    free_ptr(ctx, ctx->near_list);
    free_ptr(ctx, ctx->near_runs);
    ctx->near_cap = ctx->nrun_cap = 0;
    free_ptr(ctx, ctx->far_list);
    free_ptr(ctx, ctx->far_leaf);
    free_ptr(ctx, ctx->far_runs);
    free_ptr(ctx, ctx->run_key);
    free_ptr(ctx, ctx->run_key_s);
    free_ptr(ctx, ctx->run_ord);
    free_ptr(ctx, ctx->run_ord_s);
    ctx->far_cap = ctx->run_cap = 0;
    free_ptr(ctx, ctx->far_kf);
    ctx->far_xcap = 0;
    free_ptr(ctx, ctx->win_bnd);
    ctx->win_bnd_cap = 0;
    free_ptr(ctx, ctx->dt_front[0]);
    free_ptr(ctx, ctx->dt_front[1]);
    free_ptr(ctx, ctx->dt_far);
    free_ptr(ctx, ctx->dt_near);
    ctx->dt_cap = ctx->dt_far_cap = ctx->dt_near_cap = 0;
    free_ptr(ctx, ctx->dt_off);
    free_ptr(ctx, ctx->dt_cursor);
    free_ptr(ctx, ctx->dt_node2leaf);
    free_ptr(ctx, ctx->dt_G);
    free_ptr(ctx, ctx->dt_P);
    free_ptr(ctx, ctx->dt_list);
    free_ptr(ctx, ctx->dt_runs);
    ctx->dt_leaf_cap = ctx->dt_node_cap = ctx->dt_list_cap = ctx->dt_run_cap = 0;
    free_ptr(ctx, ctx->sort_hist);
    free_ptr(ctx, ctx->sort_ktmp);
    free_ptr(ctx, ctx->sort_vtmp);
    ctx->sort_hist_cap = ctx->sort_kv_cap = 0;
    free_ptr(ctx, ctx->conf_V64);
    free_ptr(ctx, ctx->conf_F);
    free_ptr(ctx, ctx->conf_vtmp);
    free_ptr(ctx, ctx->conf_y64);
    free_ptr(ctx, ctx->conf_a64);
    free_ptr(ctx, ctx->conf_src);
    ctx->conf_cap_nv = ctx->conf_cap_nt = 0;
    ctx->have_conf = false;
    ctx->have_mesh = false;
    ctx->tree.valid = false;
}

namespace {

tp_status ensure_buffers(tp_ctx* ctx, int64_t nv, int64_t nt) {
    const int64_t ntp = ((nt + TP_SUPER - 1) / TP_SUPER) * TP_SUPER;
    const int64_t nsup = ntp / TP_SUPER;
    if (nv <= ctx->cap_nv && nt <= ctx->cap_nt && ntp <= ctx->cap_ntp) {
        ctx->ntp = ntp;
        ctx->nsup = nsup;
        return TP_OK;
    }
    release_mesh(ctx);
    TP_TRY(tp_alloc_t(ctx, &ctx->V64, 3 * nv));
    TP_TRY(tp_alloc_t(ctx, &ctx->vtmp, 3 * nv));
    TP_TRY(tp_alloc_t(ctx, &ctx->gradbuf, 3 * nv));
    TP_TRY(tp_alloc_t(ctx, &ctx->F, 3 * nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->v2t_off, nv + 1));
    TP_TRY(tp_alloc_t(ctx, &ctx->v2t, 3 * nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->x64, 3 * nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->nu64, 3 * nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->w64, nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->perm, nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->iperm, nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->codes, nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->codes_sorted, nt));
    TP_TRY(tp_alloc_t(ctx, &ctx->idx_tmp, std::max(nt, nv) + 1));
    TP_TRY(tp_alloc_t(ctx, &ctx->soa, 10 * ntp));
    TP_TRY(tp_alloc_t(ctx, &ctx->src, (int64_t)TP_SRCW * ntp));
    TP_TRY(tp_alloc_t(ctx, &ctx->Fs, 3 * ntp));
    TP_TRY(tp_alloc_t(ctx, &ctx->acc, (int64_t)TP_NACC * ntp));
    TP_TRY(tp_alloc_t(ctx, &ctx->adjc, 9 * nt));
    ctx->red_cap = std::max<int64_t>(nt, 6 * 1024) + 4096;
    TP_TRY(tp_alloc_t(ctx, &ctx->red, ctx->red_cap));
    const int64_t nbits = nsup * nsup;
    TP_TRY(tp_alloc_t(ctx, &ctx->flagged, (nbits + 31) / 32));
    TP_TRY(tp_alloc_t(ctx, &ctx->adjbm, (nbits + 31) / 32));
    TP_TRY(tp_alloc_t(ctx, &ctx->bmask, nbits * TP_BMASK_WORDS));
    TP_TRY(tp_alloc_t(ctx, &ctx->mlist, nsup * (nsup + 1) / 2 + 1));
    TP_TRY(tp_alloc_t(ctx, &ctx->plist, nsup * (nsup + 1) / 2 + 1));
    TP_TRY(tp_alloc_t(ctx, &ctx->flist, nsup * (nsup + 1) / 2 + 1));
    TP_TRY(tp_alloc_t(ctx, &ctx->tbox, 6 * nsup));
    ctx->cap_nv = nv;
    ctx->cap_nt = nt;
    ctx->cap_ntp = ntp;
    ctx->ntp = ntp;
    ctx->nsup = nsup;
    return TP_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

int64_t n_direct_pairs(const tp_ctx* ctx, bool edge_only) {
    // ordered pairs: nt (nt - 1) minus the excluded ones (counted on upload)
    return ctx->nt * (ctx->nt - 1) - (edge_only ? ctx->n_excluded_edge_ordered : ctx->n_excluded_ordered);
}

}  // namespace

// read and clear the device error word; map to a status
tp_status take_device_error(tp_ctx* ctx, const char* where) {
    unsigned h = 0;
    TP_CU(cudaMemcpyAsync(&h, ctx->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    if (!h) return TP_OK;
    TP_CU(cudaMemsetAsync(ctx->derr, 0, sizeof(unsigned), ctx->stream));
    if (h & TP_DERR_TIMEOUT) return tp_set_err(ctx, TP_E_TIMEOUT, "%s: a device-side wait timed out", where);
    if (h & TP_DERR_INDEX) return tp_set_err(ctx, TP_E_ARG, "%s: face index outside [0, nv)", where);
    if (h & TP_DERR_STACK) return tp_set_err(ctx, TP_E_CUDA, "%s: traversal stack overflow", where);
    if (h & TP_DERR_INTERNAL) return tp_set_err(ctx, TP_E_CUDA, "%s: internal work-list check failed", where);
    if (h & TP_DERR_BOUNDS) return tp_set_err(ctx, TP_E_CUDA, "%s: bounds check of the checked build failed", where);
    if (h & TP_DERR_NONFINITE)
        return tp_set_err(ctx, TP_E_NONFINITE, "%s: degenerate triangle or non-finite coordinate", where);
    return tp_set_err(ctx, TP_E_CUDA, "%s: device error 0x%x", where, h);
}

namespace {
// Test kernel of the bounded waits: one mbarrier armed for 16 bytes that no
// copy will deliver, waited on with mbar_wait_bounded and the given limit; on
// expiry the device error word gets the timeout bit.  No copy is in flight
// when the block exits.
__global__ void k_debug_wait(uint64_t limit_ns, unsigned* derr) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!ok && threadIdx.x == 0) tp_dev_error(derr, TP_DERR_TIMEOUT);
}
}  // namespace

extern "C" {

tp_status tp_debug_wait_timeout(tp_ctx* ctx, double limit_ms) {
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return tp_set_err(ctx, TP_E_ARG, "limit_ms must be in (0, 1000]");
    k_debug_wait<<<1, 32, 0, ctx->stream>>>((uint64_t)(limit_ms * 1e6), ctx->derr);
    TP_CU(cudaGetLastError());
    return take_device_error(ctx, "tp_debug_wait_timeout");
}

tp_status tp_debug_sort(tp_ctx* ctx, const uint32_t* keys, int64_t n, int bits, uint32_t* keys_out,
                        int32_t* perm_out, int32_t* compact_out, int32_t* ncompact) {
    if (!ctx || n < 0 || (n > 0 && (!keys || !keys_out || !perm_out))) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    if (bits < 1 || bits > 32) return tp_set_err(ctx, TP_E_ARG, "bits must be in [1, 32]");
    if (n == 0) {
        if (ncompact) *ncompact = 0;
        return TP_OK;
    }
    uint32_t *kin = nullptr, *kout = nullptr;
    int32_t *vin = nullptr, *vout = nullptr, *cnt = nullptr;
    tp_status st = TP_OK;
    auto done = [&](tp_status s) {
        tp_free(ctx, kin);
        tp_free(ctx, kout);
        tp_free(ctx, vin);
        tp_free(ctx, vout);
        tp_free(ctx, cnt);
        return s;
    };
    if ((st = tp_alloc_t(ctx, &kin, n)) != TP_OK || (st = tp_alloc_t(ctx, &kout, n)) != TP_OK ||
        (st = tp_alloc_t(ctx, &vin, n)) != TP_OK || (st = tp_alloc_t(ctx, &vout, n)) != TP_OK ||
        (st = tp_alloc_t(ctx, &cnt, 1)) != TP_OK)
        return done(st);
    std::vector<int32_t> iota((size_t)n);
    for (int64_t i = 0; i < n; ++i) iota[(size_t)i] = (int32_t)i;
    if (cudaMemcpyAsync(kin, keys, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(vin, iota.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return done(tp_cuda_check(ctx, cudaGetLastError(), "tp_debug_sort upload"));
    if ((st = tp_sort_pairs_u32(ctx, kin, vin, kout, vout, n, bits)) != TP_OK) return done(st);
    if (compact_out && ncompact) {
        // compaction of the keys read as int32 (the entries >= 0 in order)
        if ((st = tp_compact_nonneg(ctx, reinterpret_cast<const int32_t*>(kin), n, vin, cnt)) != TP_OK) return done(st);
    }
    cudaMemcpyAsync(keys_out, kout, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(perm_out, vout, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (compact_out && ncompact) {
        cudaMemcpyAsync(ncompact, cnt, 4, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(compact_out, vin, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    }
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return done(tp_cuda_check(ctx, e, "tp_debug_sort"));
    return done(TP_OK);
}

tp_status tp_debug_fail_alloc(tp_ctx* ctx, int64_t after) {
    if (!ctx) return TP_E_ARG;
    ctx->fail_alloc_after = after < 0 ? -1 : after;
    return TP_OK;
}

void tp_params_default(tp_params* p) {
    if (!p) return;
    p->q = 6;
    p->p = 12;
    p->scale = 1.0;
    p->mode = TP_DIRECT;
    p->theta = 0.25;
    p->prec = TP_F32_F64ACC;
    p->flags = 0u;
}

const char* tp_version(void) { return TP_VERSION_STR; }

tp_status tp_create(tp_ctx** out, int device, void* cuda_stream) {
    if (!out) return TP_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return TP_E_CUDA;
    }
    if (device < 0 || device >= ndev) return TP_E_ARG;
    DeviceGuard g(device);
    tp_ctx* ctx = new tp_ctx();
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return TP_E_CUDA;
    }
    if (prop.major < 10) {
        delete ctx;
        return TP_E_CUDA;  // built for sm_103a only
    }
    ctx->num_sms = prop.multiProcessorCount;
    for (int i = 0; i < 4; ++i) cudaEventCreate(&ctx->ev[i]);
    if (tp_alloc_t(ctx, &ctx->derr, 4) != TP_OK || tp_alloc_t(ctx, &ctx->scalar, 16) != TP_OK ||
        tp_alloc_t(ctx, &ctx->center, 3) != TP_OK || tp_alloc_t(ctx, &ctx->bounds, 6) != TP_OK ||
        tp_alloc_t(ctx, &ctx->mcount, 16) != TP_OK || tp_alloc_t(ctx, &ctx->work, 4) != TP_OK) {
        tp_destroy(ctx);
        return TP_E_OOM;
    }
    cudaMemsetAsync(ctx->derr, 0, 4 * sizeof(unsigned), ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        tp_destroy(ctx);
        return TP_E_CUDA;
    }
    *out = ctx;
    return TP_OK;
}

void tp_destroy(tp_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    tp_mlp_release(ctx);
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    for (int i = 0; i < 4; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

const char* tp_last_error(const tp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tp_status tp_mesh_upload(tp_ctx* ctx, const void* V, int64_t nv, int v_dtype, const int32_t* F, int64_t nt,
                         uint32_t flags) {
    TpRange nvtx_range("tp_mesh_upload");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    ctx->nlaunch = 0;
    const bool dev = flags & TP_DEVICE_PTR;
    const bool posonly = flags & TP_POSITIONS_ONLY;
    if (v_dtype != TP_DTYPE_F32 && v_dtype != TP_DTYPE_F64) return tp_set_err(ctx, TP_E_ARG, "bad v_dtype %d", v_dtype);
    if (nv < 0 || nt < 0) return tp_set_err(ctx, TP_E_ARG, "negative size");
    if (nt >= (int64_t)1 << 30 || nv >= (int64_t)1 << 30) return tp_set_err(ctx, TP_E_ARG, "mesh too large");
    if (posonly) {
        if (!ctx->have_mesh) return tp_set_err(ctx, TP_E_STATE, "TP_POSITIONS_ONLY before a full upload");
        if (nv != ctx->nv) return tp_set_err(ctx, TP_E_ARG, "TP_POSITIONS_ONLY with nv=%lld != %lld", (long long)nv,
                                             (long long)ctx->nv);
        nt = ctx->nt;
    }
    if (nv > 0 && !V) return tp_set_err(ctx, TP_E_ARG, "V is NULL");
    if (!posonly && nt > 0 && !F) return tp_set_err(ctx, TP_E_ARG, "F is NULL");
    int64_t nt_tri = nt;  // caller's triangles; the elements are triangles x quadrature points
    if (!posonly) {
        const int k = ctx->quad_next.k;
        if (nt * k >= (int64_t)1 << 30) return tp_set_err(ctx, TP_E_ARG, "mesh too large for the quadrature rule");
        ctx->quad = ctx->quad_next;
        nt = nt_tri * k;
        TP_TRY(ensure_buffers(ctx, std::max<int64_t>(nv, 1), std::max<int64_t>(nt, 1)));
        if (k > 1) {
            free_ptr(ctx, ctx->F_tri);
            TP_TRY(tp_alloc_t(ctx, &ctx->F_tri, 3 * std::max<int64_t>(nt_tri, 1)));
        }
        ctx->nv = nv;
        ctx->nt = nt;
        ctx->nt_tri = nt_tri;
        ctx->ntp = ((nt + TP_SUPER - 1) / TP_SUPER) * TP_SUPER;
        ctx->nsup = ctx->ntp / TP_SUPER;
        ctx->tree.valid = false;
        ctx->have_mesh = false;
    }
    cudaEventRecord(ctx->ev[2], ctx->stream);
    // positions
    const size_t vbytes = (size_t)(3 * nv) * (v_dtype == TP_DTYPE_F64 ? 8 : 4);
    if (nv > 0) {
        if (v_dtype == TP_DTYPE_F64) {
            TP_CU(cudaMemcpyAsync(ctx->V64, V, vbytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  ctx->stream));
        } else {
            TP_CU(cudaMemcpyAsync(ctx->vtmp, V, vbytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  ctx->stream));
            k_f32_to_f64<<<(unsigned)((3 * nv + 255) / 256), 256, 0, ctx->stream>>>(ctx->vtmp, ctx->V64, 3 * nv);
            ++ctx->nlaunch;
        }
        k_check_finite_v<<<(unsigned)((3 * nv + 255) / 256), 256, 0, ctx->stream>>>(ctx->V64, 3 * nv, ctx->derr);
        ++ctx->nlaunch;
    }
    if (!posonly && nt > 0) {
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (ctx->quad.k == 1) {
            TP_CU(cudaMemcpyAsync(ctx->F, F, (size_t)(3 * nt) * 4, kind, ctx->stream));
        } else {
            TP_CU(cudaMemcpyAsync(ctx->F_tri, F, (size_t)(3 * nt_tri) * 4, kind, ctx->stream));
            TP_TRY(tp_launch_expand_faces(ctx));
        }
    }
    if (nt > 0) {
        TP_TRY(tp_launch_tri_data(ctx));
        if (!posonly) {
            TP_TRY(take_device_error(ctx, "tp_mesh_upload"));
            TP_TRY(tp_build_v2t(ctx));
            TP_TRY(tp_launch_morton_order(ctx, 30));
        }
        if (posonly) {
            // the Morton-order records and the direct kernels' item lists are
            // refreshed when a kernel needs them (a tree build redoes both)
            ctx->soa_stale = true;
            if (ctx->flags_stale < 1) ctx->flags_stale = 1;
        } else {
            TP_TRY(tp_launch_sorted_soa(ctx));
            TP_TRY(tp_launch_flagged(ctx, true));
            ctx->flags_stale = 0;
        }
        if (!posonly) TP_TRY(tp_count_excluded(ctx));
    }
    cudaEventRecord(ctx->ev[3], ctx->stream);
    TP_TRY(take_device_error(ctx, "tp_mesh_upload"));
    ctx->have_mesh = true;
    ctx->stats = tp_stats{};
    ctx->stats.nt = nt;
    ctx->stats.nv = nv;
    ctx->stats.ms_total = elapsed(ctx->ev[2], ctx->ev[3]);
    ctx->stats.kernel_launches = ctx->nlaunch;
    return TP_OK;
}

tp_status tp_tree_build(tp_ctx* ctx, int leaf_size, int morton_bits) {
    TpRange nvtx_range("tp_tree_build");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    if (!ctx->have_mesh) return tp_set_err(ctx, TP_E_STATE, "no mesh uploaded");
    if (leaf_size < 1 || leaf_size > 32) return tp_set_err(ctx, TP_E_ARG, "leaf_size must be in [1, 32]");
    if (morton_bits < 3 || morton_bits > 30 || morton_bits % 3) return tp_set_err(ctx, TP_E_ARG, "bad morton_bits");
    if (ctx->nt == 0) {
        ctx->tree.valid = true;
        return TP_OK;
    }
    ctx->nlaunch = 0;
    cudaEventRecord(ctx->ev[2], ctx->stream);
    TP_TRY(tp_launch_tree_build(ctx, leaf_size, morton_bits));
    cudaEventRecord(ctx->ev[3], ctx->stream);
    TP_TRY(take_device_error(ctx, "tp_tree_build"));
    ctx->tree.valid = true;
    ctx->stats.ms_total = elapsed(ctx->ev[2], ctx->ev[3]);
    ctx->stats.kernel_launches = ctx->nlaunch;
    return TP_OK;
}

// Per-triangle outputs of tp_fields (null: tp_energy / tp_gradient).
struct FieldOut {
    double *fw, *fnu, *fx;
};

static tp_status run_eval(tp_ctx* ctx, const tp_params* prm, bool want_grad, void* grad_out, int g_dtype,
                          uint32_t flags, double* energy_out, const FieldOut* fields = nullptr) {
    TP_TRY(check_params(ctx, prm));
    const int64_t nt = ctx->nt, nv = ctx->nv;
    ctx->stats = tp_stats{};
    ctx->stats.nt = nt;
    ctx->stats.nv = nv;
    ctx->nlaunch = 0;
    ctx->last_q = prm->q;
    ctx->last_pq = (double)prm->p / prm->q;
    const bool dev = flags & TP_DEVICE_PTR;
    if (want_grad && g_dtype != TP_DTYPE_F32 && g_dtype != TP_DTYPE_F64)
        return tp_set_err(ctx, TP_E_ARG, "bad g_dtype %d", g_dtype);
    if (want_grad && !fields && nv > 0 && !grad_out) return tp_set_err(ctx, TP_E_ARG, "grad_out is NULL");
    const size_t gbytes = (size_t)(3 * nv) * (g_dtype == TP_DTYPE_F64 ? 8 : 4);
    if (nt == 0) {
        if (energy_out) *energy_out = 0.0;
        if (want_grad && !fields && nv > 0) {
            if (dev) TP_CU(cudaMemsetAsync(grad_out, 0, gbytes, ctx->stream));
            else memset(grad_out, 0, gbytes);
            TP_CU(cudaStreamSynchronize(ctx->stream));
        }
        return TP_OK;
    }
    cudaEventRecord(ctx->ev[2], ctx->stream);
    bool energy_from_acc = true;
    if (prm->mode == TP_DIRECT) {
        if (prm->prec == TP_F64) {
            TP_TRY(tp_launch_direct_f64(ctx, prm, want_grad));
            if (!want_grad) {
                energy_from_acc = false;
                TP_TRY(tp_launch_reduce_sum(ctx, ctx->red, nt, ctx->scalar + 1));
            }
        } else if (prm->prec == TP_F32_KAHAN) {
            TP_TRY(tp_launch_direct_kahan(ctx, prm));
        } else if (want_grad) {
            TP_TRY(tp_launch_direct_grad(ctx, prm));
        } else {
            int nparts = 0;
            TP_TRY(tp_launch_direct_energy(ctx, prm, ctx->red, &nparts));
            TP_TRY(tp_launch_reduce_sum(ctx, ctx->red, nparts, ctx->scalar + 1));
            energy_from_acc = false;
        }
        ctx->stats.pairs_exact = n_direct_pairs(ctx, (prm->flags & TP_EXCLUDE_EDGE) != 0);
        ctx->stats.tile_pairs = ctx->nsup * (ctx->nsup + 1) / 2;
        ctx->stats.tile_pairs_masked = ctx->n_masked;
        ctx->stats.tile_pairs_precise = ctx->n_precise;
        ctx->stats.kernel_pairs = tp_direct_timed_pairs(ctx);  // the timed (non-masked) launch
    } else if (prm->mode == TP_BH_DUAL) {
        TP_TRY(tp_launch_dual(ctx, prm));
    } else {
        TP_TRY(tp_launch_bh(ctx, prm, prm->mode == TP_LEARNED));
    }
    double pq = (double)prm->p / prm->q;
    if (energy_from_acc) {
        TP_TRY(tp_launch_energy_from_acc(ctx, prm, ctx->scalar));
    }
    void* gdst = nullptr;
    if (fields) {
        double* st = nullptr;
        if (!dev) {
            if (!ctx->fieldbuf) TP_TRY(tp_alloc_t(ctx, &ctx->fieldbuf, 7 * ctx->cap_nt));
            st = ctx->fieldbuf;
        }
        TP_TRY(tp_launch_fields(ctx, prm, dev ? fields->fw : (fields->fw ? st : nullptr),
                                dev ? fields->fnu : (fields->fnu ? st + nt : nullptr),
                                dev ? fields->fx : (fields->fx ? st + 4 * nt : nullptr)));
    } else if (want_grad) {
        gdst = dev ? grad_out : (void*)ctx->gradbuf;
        TP_TRY(tp_launch_adjoint(ctx, prm, gdst, g_dtype));
    }
    cudaEventRecord(ctx->ev[3], ctx->stream);
    double e = 0.0;
    if (energy_from_acc) {
        TP_CU(cudaMemcpyAsync(&e, ctx->scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    } else {
        TP_CU(cudaMemcpyAsync(&e, ctx->scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (want_grad && !fields && !dev && nv > 0)
        TP_CU(cudaMemcpyAsync(grad_out, ctx->gradbuf, gbytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (fields && !dev) {
        if (fields->fw) TP_CU(cudaMemcpyAsync(fields->fw, ctx->fieldbuf, 8 * nt, cudaMemcpyDeviceToHost, ctx->stream));
        if (fields->fnu)
            TP_CU(cudaMemcpyAsync(fields->fnu, ctx->fieldbuf + nt, 24 * nt, cudaMemcpyDeviceToHost, ctx->stream));
        if (fields->fx)
            TP_CU(cudaMemcpyAsync(fields->fx, ctx->fieldbuf + 4 * nt, 24 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    }
    TP_CU(cudaStreamSynchronize(ctx->stream));
    TP_TRY(take_device_error(ctx, want_grad ? "tp_gradient" : "tp_energy"));
    if (!energy_from_acc && prm->mode == TP_DIRECT) {
        if (prm->prec == TP_F64) e = prm->scale * e;
        else e = prm->scale * e / pq;
    }
    ctx->stats.ms_kernel = elapsed(ctx->ev[0], ctx->ev[1]);
    ctx->stats.ms_total = elapsed(ctx->ev[2], ctx->ev[3]);
    ctx->stats.kernel_launches = ctx->nlaunch;
    if (energy_out) *energy_out = e;
    if (!std::isfinite(e)) {
        if (energy_out) *energy_out = INFINITY;
        return tp_set_err(ctx, TP_E_NONFINITE,
                          "energy is not finite: two admitted triangles have coincident centroids (not embedded)");
    }
    return TP_OK;
}

tp_status tp_energy(tp_ctx* ctx, const tp_params* params, double* energy_out) {
    TpRange nvtx_range("tp_energy");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    if (!energy_out) return tp_set_err(ctx, TP_E_ARG, "energy_out is NULL");
    return run_eval(ctx, params, false, nullptr, TP_DTYPE_F64, 0u, energy_out);
}

tp_status tp_gradient(tp_ctx* ctx, const tp_params* params, double* energy_out, void* grad_out, int g_dtype,
                      uint32_t flags) {
    TpRange nvtx_range("tp_gradient");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    return run_eval(ctx, params, true, grad_out, g_dtype, flags, energy_out);
}

tp_status tp_fields(tp_ctx* ctx, const tp_params* params, double* energy_out, double* fw, double* fnu, double* fx,
                    uint32_t flags) {
    TpRange nvtx_range("tp_fields");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    const FieldOut fo{fw, fnu, fx};
    return run_eval(ctx, params, true, nullptr, TP_DTYPE_F64, flags, energy_out, &fo);
}

tp_status tp_set_quadrature(tp_ctx* ctx, int npoints) {
    if (!ctx) return TP_E_ARG;
    ctx->err.clear();
    tp_quad_rule r{};
    r.k = npoints;
    if (npoints == 1) {
        r.bary[0][0] = r.bary[0][1] = r.bary[0][2] = 1.0 / 3.0;
        r.w[0] = 1.0;
    } else if (npoints == 3) {
        // degree 2: the points (2/3, 1/6, 1/6) and permutations, equal weights
        for (int q = 0; q < 3; ++q) {
            for (int j = 0; j < 3; ++j) r.bary[q][j] = j == q ? 2.0 / 3.0 : 1.0 / 6.0;
            r.w[q] = 1.0 / 3.0;
        }
    } else if (npoints == 6) {
        // degree 4 (Strang and Fix): two orbits (a, a, 1 - 2a) with closed-form a and weights
        const double s10 = std::sqrt(10.0), rr = std::sqrt(38.0 - 44.0 * std::sqrt(2.0 / 5.0));
        const double t = std::sqrt(213125.0 - 53320.0 * s10);
        const double a[2] = {(8.0 - s10 + rr) / 18.0, (8.0 - s10 - rr) / 18.0};
        const double w[2] = {(620.0 + t) / 3720.0, (620.0 - t) / 3720.0};
        for (int o = 0; o < 2; ++o)
            for (int j = 0; j < 3; ++j) {
                const int q = 3 * o + j;
                for (int m = 0; m < 3; ++m) r.bary[q][m] = m == j ? 1.0 - 2.0 * a[o] : a[o];
                r.w[q] = w[o];
            }
    } else {
        return tp_set_err(ctx, TP_E_ARG, "quadrature with %d points (supported: 1, 3, 6)", npoints);
    }
    ctx->quad_next = r;
    return TP_OK;
}

tp_status tp_conf_upload(tp_ctx* ctx, const void* V, int64_t nv, int v_dtype, const int32_t* F, int64_t nt,
                         uint32_t flags) {
    TpRange nvtx_range("tp_conf_upload");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    ctx->nlaunch = 0;
    const bool dev = flags & TP_DEVICE_PTR;
    if (v_dtype != TP_DTYPE_F32 && v_dtype != TP_DTYPE_F64) return tp_set_err(ctx, TP_E_ARG, "bad v_dtype %d", v_dtype);
    if (nv < 0 || nt < 0) return tp_set_err(ctx, TP_E_ARG, "negative size");
    if (nt >= (int64_t)1 << 30 || nv >= (int64_t)1 << 30) return tp_set_err(ctx, TP_E_ARG, "mesh too large");
    if ((nv > 0 && !V) || (nt > 0 && !F)) return tp_set_err(ctx, TP_E_ARG, "V or F is NULL");
    ctx->have_conf = false;
    const int64_t ntp = ((nt + TP_SUPER - 1) / TP_SUPER) * TP_SUPER;
    if (nv > ctx->conf_cap_nv || nt > ctx->conf_cap_nt || !ctx->conf_src) {
        free_ptr(ctx, ctx->conf_V64);
        free_ptr(ctx, ctx->conf_F);
        free_ptr(ctx, ctx->conf_vtmp);
        free_ptr(ctx, ctx->conf_y64);
        free_ptr(ctx, ctx->conf_a64);
        free_ptr(ctx, ctx->conf_src);
        const int64_t cnv = std::max<int64_t>(nv, 1), cnt = std::max<int64_t>(nt, 1);
        const int64_t cntp = std::max<int64_t>(ntp, TP_SUPER);
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_V64, 3 * cnv));
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_F, 3 * cnt));
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_vtmp, 3 * cnv));
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_y64, 3 * cnt));
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_a64, cnt));
        TP_TRY(tp_alloc_t(ctx, &ctx->conf_src, (int64_t)TP_SRCW * cntp));
        ctx->conf_cap_nv = cnv;
        ctx->conf_cap_nt = cnt;
    }
    ctx->conf_nv = nv;
    ctx->conf_nt = nt;
    ctx->conf_ntp = ntp;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nv > 0) {
        if (v_dtype == TP_DTYPE_F64) {
            TP_CU(cudaMemcpyAsync(ctx->conf_V64, V, 24 * nv, kind, ctx->stream));
        } else {
            TP_CU(cudaMemcpyAsync(ctx->conf_vtmp, V, 12 * nv, kind, ctx->stream));
            k_f32_to_f64<<<(unsigned)((3 * nv + 255) / 256), 256, 0, ctx->stream>>>(ctx->conf_vtmp, ctx->conf_V64,
                                                                                  3 * nv);
            ++ctx->nlaunch;
        }
    }
    if (nt > 0) {
        TP_CU(cudaMemcpyAsync(ctx->conf_F, F, 12 * nt, kind, ctx->stream));
        TP_TRY(tp_launch_conf_tri(ctx));
    }
    TP_TRY(take_device_error(ctx, "tp_conf_upload"));
    ctx->have_conf = true;
    return TP_OK;
}

tp_status tp_conf_gradient(tp_ctx* ctx, const tp_params* params, double* energy_out, void* grad_out, int g_dtype,
                           uint32_t flags) {
    TpRange nvtx_range("tp_conf_gradient");
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    ctx->err.clear();
    const tp_params* prm = params;
    TP_TRY(check_params(ctx, prm));
    if (prm->mode != TP_DIRECT) return tp_set_err(ctx, TP_E_ARG, "the confinement energy is evaluated directly");
    if (prm->prec == TP_F32_KAHAN)
        return tp_set_err(ctx, TP_E_ARG, "the confinement energy has FP32 terms with FP64 sums or the FP64 form only");
    if (!ctx->have_conf) return tp_set_err(ctx, TP_E_STATE, "no confining surface uploaded (tp_conf_upload)");
    const bool want_grad = grad_out != nullptr;
    if (want_grad && g_dtype != TP_DTYPE_F32 && g_dtype != TP_DTYPE_F64)
        return tp_set_err(ctx, TP_E_ARG, "bad g_dtype %d", g_dtype);
    const int64_t nt = ctx->nt, nv = ctx->nv;
    const bool dev = flags & TP_DEVICE_PTR;
    const size_t gbytes = (size_t)(3 * nv) * (g_dtype == TP_DTYPE_F64 ? 8 : 4);
    ctx->stats = tp_stats{};
    ctx->stats.nt = nt;
    ctx->stats.nv = nv;
    ctx->nlaunch = 0;
    if (nt == 0 || ctx->conf_nt == 0) {
        if (energy_out) *energy_out = 0.0;
        if (want_grad && nv > 0) {
            if (dev) TP_CU(cudaMemsetAsync(grad_out, 0, gbytes, ctx->stream));
            else memset(grad_out, 0, gbytes);
            TP_CU(cudaStreamSynchronize(ctx->stream));
        }
        return TP_OK;
    }
    cudaEventRecord(ctx->ev[2], ctx->stream);
    TP_TRY(tp_launch_conf(ctx, prm));
    const double pq = (double)prm->p / prm->q;
    TP_TRY(tp_launch_energy_scaled(ctx, prm->scale / pq, ctx->scalar));
    if (want_grad) TP_TRY(tp_launch_adjoint(ctx, prm, dev ? grad_out : (void*)ctx->gradbuf, g_dtype));
    cudaEventRecord(ctx->ev[3], ctx->stream);
    double e = 0.0;
    TP_CU(cudaMemcpyAsync(&e, ctx->scalar, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (want_grad && !dev && nv > 0)
        TP_CU(cudaMemcpyAsync(grad_out, ctx->gradbuf, gbytes, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    TP_TRY(take_device_error(ctx, "tp_conf_gradient"));
    ctx->stats.pairs_exact = nt * ctx->conf_nt;
    ctx->stats.kernel_pairs = nt * ctx->conf_nt;
    ctx->stats.ms_kernel = elapsed(ctx->ev[0], ctx->ev[1]);
    ctx->stats.ms_total = elapsed(ctx->ev[2], ctx->ev[3]);
    ctx->stats.kernel_launches = ctx->nlaunch;
    if (energy_out) *energy_out = e;
    if (!std::isfinite(e)) {
        if (energy_out) *energy_out = INFINITY;
        return tp_set_err(ctx, TP_E_NONFINITE, "confinement energy is not finite: the surfaces touch");
    }
    return TP_OK;
}

tp_status tp_get_stats(const tp_ctx* ctx, tp_stats* out) {
    if (!ctx || !out) return TP_E_ARG;
    *out = ctx->stats;
    return TP_OK;
}

tp_status tp_debug_tri_data(tp_ctx* ctx, int32_t* perm, double* x, double* nu, double* w) {
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    if (!ctx->have_mesh) return tp_set_err(ctx, TP_E_STATE, "no mesh uploaded");
    const int64_t nt = ctx->nt;
    if (nt == 0) return TP_OK;
    std::vector<int32_t> hp(nt);
    std::vector<double> hx(3 * nt), hn(3 * nt), hw(nt);
    TP_CU(cudaMemcpyAsync(hp.data(), ctx->perm, 4 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hx.data(), ctx->x64, 24 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hn.data(), ctx->nu64, 24 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hw.data(), ctx->w64, 8 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    for (int64_t k = 0; k < nt; ++k) {
        if (perm) perm[k] = hp[k];
        int64_t T = hp[k];
        for (int a = 0; a < 3; ++a) {
            if (x) x[3 * k + a] = hx[a * nt + T];
            if (nu) nu[3 * k + a] = hn[a * nt + T];
        }
        if (w) w[k] = hw[T];
    }
    return TP_OK;
}

tp_status tp_debug_accum(tp_ctx* ctx, double* gw, double* gnu, double* gx) {
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    if (!ctx->have_mesh) return tp_set_err(ctx, TP_E_STATE, "no mesh uploaded");
    const int64_t nt = ctx->nt, ntp = ctx->ntp;
    if (nt == 0) return TP_OK;
    std::vector<double> acc((size_t)TP_NACC * ntp), hn(3 * nt), hw(nt);
    std::vector<int32_t> ip(nt);
    TP_CU(cudaMemcpyAsync(acc.data(), ctx->acc, 8 * TP_NACC * ntp, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(ip.data(), ctx->iperm, 4 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hn.data(), ctx->nu64, 24 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaMemcpyAsync(hw.data(), ctx->w64, 8 * nt, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    const double q = ctx->last_q, pq = ctx->last_pq;
    for (int64_t T = 0; T < nt; ++T) {
        int64_t k = ip[T];
        if (gw) gw[T] = acc[k] / (pq * hw[T]);
        for (int a = 0; a < 3; ++a) {
            if (gnu) gnu[3 * T + a] = q * acc[(2 + a) * ntp + k] / pq;
            if (gx) gx[3 * T + a] = q * (acc[(5 + a) * ntp + k] + acc[ntp + k] * hn[a * nt + T]) / pq;
        }
    }
    return TP_OK;
}

tp_status tp_set_learned_window(tp_ctx* ctx, int64_t rows) {
    if (!ctx) return TP_E_ARG;
    ctx->err.clear();
    if (rows != 0 && rows < 32) return tp_set_err(ctx, TP_E_ARG, "learned window of %lld rows (minimum 32)", (long long)rows);
    ctx->learned_window = rows == 0 ? TP_LEARNED_WINDOW : rows;
    return TP_OK;
}

tp_status tp_debug_tree(tp_ctx* ctx, uint32_t* codes, int32_t* perm, int32_t* left, int32_t* right, int32_t* first,
                        int32_t* last, int32_t* leaves, int64_t* nleaves, double* mom, double* box) {
    if (!ctx) return TP_E_ARG;
    DeviceGuard g(ctx->device);
    if (!ctx->tree.valid) return tp_set_err(ctx, TP_E_STATE, "no tree built");
    const int64_t n = ctx->nt;
    if (n == 0) return TP_OK;
    const int64_t nn = 2 * n - 1;
    tp_tree& t = ctx->tree;
    if (codes) TP_CU(cudaMemcpyAsync(codes, ctx->codes, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (perm) TP_CU(cudaMemcpyAsync(perm, ctx->perm, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (left && n > 1) TP_CU(cudaMemcpyAsync(left, t.left, 4 * (n - 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (right && n > 1) TP_CU(cudaMemcpyAsync(right, t.right, 4 * (n - 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (first) TP_CU(cudaMemcpyAsync(first, t.first, 4 * nn, cudaMemcpyDeviceToHost, ctx->stream));
    if (last) TP_CU(cudaMemcpyAsync(last, t.last, 4 * nn, cudaMemcpyDeviceToHost, ctx->stream));
    if (leaves) TP_CU(cudaMemcpyAsync(leaves, t.leaves, 4 * t.nleaves, cudaMemcpyDeviceToHost, ctx->stream));
    if (mom) TP_CU(cudaMemcpyAsync(mom, t.mom, 8 * 13 * nn, cudaMemcpyDeviceToHost, ctx->stream));
    if (box) TP_CU(cudaMemcpyAsync(box, t.box, 8 * 6 * nn, cudaMemcpyDeviceToHost, ctx->stream));
    TP_CU(cudaStreamSynchronize(ctx->stream));
    if (nleaves) *nleaves = t.nleaves;
    return TP_OK;
}

}  // extern "C"
