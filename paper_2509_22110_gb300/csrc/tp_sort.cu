// tp_sort.cu - stable key sort and stream compaction of the cluster-tree build.
//
// The LBVH (Sec. 3.2's cluster tree, built as a linear BVH over Morton codes)
// needs the triangles in ascending order of their 30-bit codes with ties in
// ascending triangle index, and the list of cluster leaves compacted from a
// per-primitive marker array.  Both are written here for sm_103a:
//
// Sort.  Least-significant-digit radix sort, 8-bit digits (four passes for
// 30-bit codes), each pass three launches over tiles of SORT_TILE keys:
//   k_sort_hist     per tile, a 256-bin histogram of the pass's digit in
//                   shared memory, stored digit-major: hist[d * ntiles + tile];
//   k_sort_rows     one warp per digit d: exclusive prefix sum of row d of
//                   hist over the tiles (in place) and the row total tot[d];
//                   the scatter adds the prefix of tot over the digits, so
//                   that tile's keys with digit d start at
//                   sum_{d' < d} tot[d'] + hist[d * ntiles + tile];
//   k_sort_scatter  per tile, the stable rank of every key among the tile's
//                   keys with the same digit, then the scatter.  Each warp
//                   owns 32 x SORT_ITEMS consecutive keys and walks them in
//                   rows of 32 (row r = keys r*32 .. r*32+31 of its slice):
//                   lanes holding the same digit find each other with
//                   __match_any_sync, a lane's rank in the row is the number
//                   of its peers in lower lanes, and a per-warp digit counter
//                   in shared memory carries the ranks across rows.  After a
//                   block barrier the warps' counts are prefix-summed per
//                   digit, which orders the warps' slices.
// Every pass keeps the order of equal digits, so the result is sorted by the
// whole key with ties in input order.
//
// Compaction.  k_compact_count counts the entries >= 0 of every tile,
// k_scan prefix-sums the tile counts (one block) and writes the total,
// k_compact_write stores each tile's entries in order at its offset.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tp_internal.cuh"

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 8;                               // keys per lane per tile
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;        // 2048 keys per tile
constexpr int SORT_BINS = 256;
constexpr int SCAN_THREADS = 1024;

// Position of key i of a tile: warp w owns keys [w * 32 * ITEMS, (w + 1) * 32 *
// ITEMS); lane l, item r holds key w * 32 * ITEMS + r * 32 + l.
__device__ __forceinline__ int tile_pos(int warp, int lane, int r) { return warp * 32 * SORT_ITEMS + r * 32 + lane; }

template <class K>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                            int ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[SORT_BINS];
    for (int d = threadIdx.x; d < SORT_BINS; d += SORT_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int i = threadIdx.x; i < SORT_TILE; i += SORT_THREADS) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&h[(uint32_t)(keys[k] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < SORT_BINS; d += SORT_THREADS) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Block-wide exclusive prefix sum of one value per thread (SCAN_THREADS or
// SORT_THREADS threads); *total receives the block's sum.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* wsum, uint32_t& total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t r = x - v + (warp > 0 ? wsum[warp - 1] : 0u);
    total = wsum[NT / 32 - 1];
    __syncthreads();  // wsum is reused by the next call
    return r;
}

// Prefix sum of m 32-bit counts by one block, in rounds of SCAN_THREADS
// consecutive entries: out[i] = sum of in[j] for j < i (exclusive) or j <= i
// (inclusive); out may be in.  The total goes to *total when not null.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const uint32_t* in, uint32_t* out, int64_t m, int inclusive,
                                                       int32_t* __restrict__ total) {
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < m; b += SCAN_THREADS) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < m ? in[i] : 0u;
        uint32_t rt;
        const uint32_t r = block_exclusive_scan<SCAN_THREADS>(v, wsum, rt);
        if (i < m) out[i] = carry + r + (inclusive ? v : 0u);
        carry += rt;
    }
    if (total && threadIdx.x == 0) *total = (int32_t)carry;
}

// One warp per digit: exclusive prefix of hist row d over the tiles, in place,
// and the row total tot[d].
__global__ void __launch_bounds__(SORT_THREADS) k_sort_rows(uint32_t* __restrict__ hist, int ntiles,
                                                            uint32_t* __restrict__ tot) {
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * SORT_WARPS + (threadIdx.x >> 5);
    if (d >= SORT_BINS) return;
    uint32_t* row = hist + (int64_t)d * ntiles;
    uint32_t carry = 0;
    for (int c = 0; c < ntiles; c += 32) {
        const int t = c + lane;
        const uint32_t v = t < ntiles ? row[t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (t < ntiles) row[t] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) tot[d] = carry;
}

// vin == nullptr: keys only (vout is not touched)
template <class K>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const K* __restrict__ kin, const int32_t* __restrict__ vin,
                                                               int64_t n, int shift, int ntiles,
                                                               const uint32_t* __restrict__ offs,
                                                               const uint32_t* __restrict__ tot, K* __restrict__ kout,
                                                               int32_t* __restrict__ vout) {
    __shared__ uint32_t wcnt[SORT_WARPS][SORT_BINS];  // per-warp digit counts, then their exclusive prefix over warps
    __shared__ uint32_t dbase[SORT_BINS];             // first output slot of each digit
    __shared__ uint32_t wsum[SORT_WARPS];
    static_assert(SORT_THREADS == SORT_BINS, "one thread per digit for the digit bases");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < SORT_WARPS * SORT_BINS; i += SORT_THREADS) (&wcnt[0][0])[i] = 0;
    {
        uint32_t all;
        dbase[tid] = block_exclusive_scan<SORT_THREADS>(tot[tid], wsum, all);
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const unsigned lt = (1u << lane) - 1u;
    K key[SORT_ITEMS];
    int32_t val[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t k = base + tile_pos(warp, lane, r);
        const bool ok = k < n;
        key[r] = ok ? kin[k] : K(0);
        val[r] = (ok && vin) ? vin[k] : 0;
        // absent keys take digit 256: they form their own peer group and are never stored
        const uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & 0xffu) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = __popc(peers & lt);
        uint32_t prior = 0;
        if (ok) prior = wcnt[warp][d];
        __syncwarp();
        if (ok && before == 0) wcnt[warp][d] = prior + __popc(peers);
        __syncwarp();
        rank[r] = prior + before;
    }
    __syncthreads();
    // exclusive prefix of the warps' counts, per digit
    for (int d = tid; d < SORT_BINS; d += SORT_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t k = base + tile_pos(warp, lane, r);
        if (k >= n) continue;
        const uint32_t d = (uint32_t)(key[r] >> shift) & 0xffu;
        const int64_t dst = (int64_t)dbase[d] + offs[(int64_t)d * ntiles + blockIdx.x] + wcnt[warp][d] + rank[r];
        kout[dst] = key[r];
        if (vin) vout[dst] = val[r];
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_compact_count(const int32_t* __restrict__ in, int64_t n,
                                                                uint32_t* __restrict__ cnt) {
    __shared__ uint32_t ws[SORT_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    uint32_t c = 0;
    for (int i = tid; i < SORT_TILE; i += SORT_THREADS) {
        const int64_t k = base + i;
        c += (k < n && in[k] >= 0) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) ws[warp] = c;
    __syncthreads();
    if (tid == 0) {
        uint32_t s = 0;
        for (int w = 0; w < SORT_WARPS; ++w) s += ws[w];
        cnt[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_compact_write(const int32_t* __restrict__ in, int64_t n,
                                                                const uint32_t* __restrict__ offs,
                                                                int32_t* __restrict__ out) {
    __shared__ uint32_t wsum[SORT_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const unsigned lt = (1u << lane) - 1u;
    // the tile in rounds of SORT_THREADS consecutive entries, in order
    uint32_t run = offs[blockIdx.x];
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t k = base + (int64_t)r * SORT_THREADS + tid;
        const int32_t v = k < n ? in[k] : -1;
        const unsigned b = __ballot_sync(0xffffffffu, v >= 0);
        if (lane == 0) wsum[warp] = __popc(b);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = wsum[w];
            before += w < warp ? c : 0u;
            total += c;
        }
        if (v >= 0) out[run + before + __popc(b & lt)] = v;
        run += total;
        __syncthreads();
    }
}

}  // namespace

// scratch of the sort (key width kbytes) and of the compaction, grown to the need
tp_status tp_sort_scratch(tp_ctx* ctx, int64_t n, int kbytes) {
    const int64_t ntiles = std::max<int64_t>(1, (n + SORT_TILE - 1) / SORT_TILE);
    const int64_t need_hist = ntiles * SORT_BINS + SORT_BINS;  // per-tile digit counts, then the digit totals
    if (ctx->sort_hist_cap < need_hist) {
        tp_free(ctx, ctx->sort_hist);
        ctx->sort_hist = nullptr;
        ctx->sort_hist_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->sort_hist, need_hist));
        ctx->sort_hist_cap = need_hist;
    }
    const int64_t kwords = std::max<int64_t>(n, 1) * (kbytes / 4);  // 32-bit words of ping-pong keys
    if (ctx->sort_kv_cap < kwords) {
        tp_free(ctx, ctx->sort_ktmp);
        tp_free(ctx, ctx->sort_vtmp);
        ctx->sort_ktmp = nullptr;
        ctx->sort_vtmp = nullptr;
        ctx->sort_kv_cap = 0;
        TP_TRY(tp_alloc_t(ctx, &ctx->sort_ktmp, kwords));
        TP_TRY(tp_alloc_t(ctx, &ctx->sort_vtmp, kwords));
        ctx->sort_kv_cap = kwords;
    }
    return TP_OK;
}

namespace {
template <class K>
tp_status sort_pairs(tp_ctx* ctx, const K* keys_in, const int32_t* vals_in, K* keys_out, int32_t* vals_out, int64_t n,
                     int bits) {
    if (n <= 0) return TP_OK;
    if (bits < 1 || bits > 8 * (int)sizeof(K)) return tp_set_err(ctx, TP_E_ARG, "sort: bad key width %d", bits);
    TP_TRY(tp_sort_scratch(ctx, n, sizeof(K)));
    const int ntiles = (int)((n + SORT_TILE - 1) / SORT_TILE);
    const int passes = (bits + 7) / 8;
    K* ktmp = reinterpret_cast<K*>(ctx->sort_ktmp);
    // ping-pong between the scratch pair and the output, ending in the output
    const K* ks = keys_in;
    const int32_t* vs = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) & 1) == 0;
        K* kd = to_out ? keys_out : ktmp;
        int32_t* vd = vals_in ? (to_out ? vals_out : ctx->sort_vtmp) : nullptr;
        uint32_t* tot = ctx->sort_hist + (int64_t)ntiles * SORT_BINS;
        k_sort_hist<K><<<ntiles, SORT_THREADS, 0, ctx->stream>>>(ks, n, 8 * p, ntiles, ctx->sort_hist);
        k_sort_rows<<<SORT_BINS / SORT_WARPS, SORT_THREADS, 0, ctx->stream>>>(ctx->sort_hist, ntiles, tot);
        k_sort_scatter<K><<<ntiles, SORT_THREADS, 0, ctx->stream>>>(ks, vs, n, 8 * p, ntiles, ctx->sort_hist, tot, kd,
                                                                    vd);
        ctx->nlaunch += 3;
        ks = kd;
        vs = vd;
    }
    TP_CU(cudaGetLastError());
    return TP_OK;
}
}  // namespace

tp_status tp_sort_pairs_u32(tp_ctx* ctx, const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_out,
                            int32_t* vals_out, int64_t n, int bits) {
    TpRange nvtx_range("tp_sort_pairs_u32");
    return sort_pairs<uint32_t>(ctx, keys_in, vals_in, keys_out, vals_out, n, bits);
}

tp_status tp_sort_pairs_u64(tp_ctx* ctx, const uint64_t* keys_in, const int32_t* vals_in, uint64_t* keys_out,
                            int32_t* vals_out, int64_t n, int bits) {
    TpRange nvtx_range("tp_sort_pairs_u64");
    return sort_pairs<uint64_t>(ctx, keys_in, vals_in, keys_out, vals_out, n, bits);
}

tp_status tp_scan_u32(tp_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t m, bool inclusive, int32_t* total_d) {
    TpRange nvtx_range("tp_scan_u32");
    if (m <= 0) return TP_OK;
    k_scan<<<1, SCAN_THREADS, 0, ctx->stream>>>(in, out, m, inclusive ? 1 : 0, total_d);
    ++ctx->nlaunch;
    TP_CU(cudaGetLastError());
    return TP_OK;
}

tp_status tp_compact_nonneg(tp_ctx* ctx, const int32_t* in, int64_t n, int32_t* out, int32_t* count_d) {
    TpRange nvtx_range("tp_compact_nonneg");
    if (n <= 0) {
        TP_CU(cudaMemsetAsync(count_d, 0, sizeof(int32_t), ctx->stream));
        return TP_OK;
    }
    TP_TRY(tp_sort_scratch(ctx, n, 4));
    const int ntiles = (int)((n + SORT_TILE - 1) / SORT_TILE);
    k_compact_count<<<ntiles, SORT_THREADS, 0, ctx->stream>>>(in, n, ctx->sort_hist);
    k_scan<<<1, SCAN_THREADS, 0, ctx->stream>>>(ctx->sort_hist, ctx->sort_hist, ntiles, 0, count_d);
    k_compact_write<<<ntiles, SORT_THREADS, 0, ctx->stream>>>(in, n, ctx->sort_hist, out);
    ctx->nlaunch += 3;
    TP_CU(cudaGetLastError());
    return TP_OK;
}
