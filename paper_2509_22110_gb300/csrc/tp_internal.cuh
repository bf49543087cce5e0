// tp_internal.cuh - context, device buffers and launch helpers of libtp.
//
// Data layout in HBM (all device memory owned by the context):
//   V64[nv][3]            f64  vertex positions (input copy)
//   F[nt][3]              i32  faces in the caller's order
//   v2t_off[nv+1], v2t[3nt]    vertex -> (triangle*4 + corner) incidence (CSR)
//   x64/nu64[3][nt], w64[nt]   f64 triangle data in the caller's order
//   perm[nt], iperm[nt]        library order (Morton) <-> caller's order
//   soa: 10 planes of ntp f32  (x_hi[3], x_lo[3], nu[3], sqrt(2) w) in
//        library order, padded to a multiple of TP_SUPER (1536) with zero-area
//        triangles placed far away
//   src[ntp][20] f32           the same 10 values, each stored twice, one
//                              80-byte record per triangle: the unit the
//                              pair kernel stages into shared memory
//   Fs[ntp][3] i32             faces in library order (padding: unique negatives)
//   acc[8][ntp] f64            per-triangle accumulators of the pair kernels
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tp.h"

#include <nvtx3/nvToolsExt.h>

// NVTX range over the lifetime of the object: every C-ABI call and every
// launch phase (one or a few kernels) is marked on the host timeline of a
// profiler (nsys, ncu --nvtx).  Header-only NVTX costs a predictable branch
// when no tool is attached.
struct TpRange {
    explicit TpRange(const char* name) { nvtxRangePushA(name); }
    ~TpRange() { nvtxRangePop(); }
    TpRange(const TpRange&) = delete;
    TpRange& operator=(const TpRange&) = delete;
};

#define TP_SUPER 1536      // triangles per super-tile (one block's target set)
#define TP_CHUNK 128       // sources staged per shared-memory chunk
#define TP_SRCW 20         // floats per staged source record
#define TP_NACC 8          // accumulators per triangle
#define TP_NBLK (TP_SUPER / TP_CHUNK)  // 128-triangle blocks per super-tile side
#define TP_BMASK_WORDS ((TP_NBLK * TP_NBLK + 31) / 32)  // bits of one super-tile pair's block mask
#define TP_SPIN_LIMIT (1u << 26)
// Pair arithmetic of the gradient kernels: 1 forms wi s6 = wi (al^q + be^q) as
// A5 al + B5 be and the pair energy as that times |d|^2 (one packed operation
// fewer per pair), 0 forms al^q, be^q and s6 explicitly.
#ifndef TP_PAIR_T
#define TP_PAIR_T 1
#endif
// a bounded device wait gives up after this much wall-clock time (ns), or
// after TP_SPIN_LIMIT polls, whichever comes first
#define TP_WAIT_NS 1000000000ull
// super-tile pairs whose centroid boxes are closer than this fraction of the
// mesh's centroid-box diagonal form centroid differences from hi + lo parts
#define TP_PRECISE_GAP_REL 0.02f

// clusters per run of the near-field kernels' lists (the Barnes-Hut and the
// cluster-cluster forms write runs of at most this length)
#ifndef TP_BH_NEAR
#define TP_BH_NEAR 256
#endif

// floats per node of the FP32 admissibility record: outward box [6], X_C [3],
// diag_C [1], first, last, left, right as int bits (children -1 for
// single-triangle nodes), 2 unused: 64 bytes, so one round of four 16-byte
// loads gives a traversal everything it needs about a node.  The inward box
// of the pre-test is derived from the outward one (tp_inward_lo/hi).
#define TP_ADM32_W 16

// listed far rows per window of the learned passes: 32 Mi rows, 1 GB of
// network factors (tp_set_learned_window changes it)
#define TP_LEARNED_WINDOW ((int64_t)1 << 25)

// device error bits
#define TP_DERR_TIMEOUT 0x1u
#define TP_DERR_STACK 0x2u
#define TP_DERR_INDEX 0x4u
#define TP_DERR_NONFINITE 0x8u
#define TP_DERR_INTERNAL 0x10u  // a consistency check of a kernel's own work lists failed
#define TP_DERR_BOUNDS 0x20u    // a bounds check of the checked build (TP_DEBUG) failed

// TP_DEBUG = 1 builds libtp_debug.so: the list-driven kernels also check every
// index they read from a work list (node ids, member ranges, listed rows, CSR
// entries, item tiles) against its array, record a failure in the device
// error word (TP_DERR_BOUNDS) and skip the access.  The release build checks
// list capacities only.
#ifndef TP_DEBUG
#define TP_DEBUG 0
#endif

struct tp_tree {
    bool valid = false;
    bool feat_stale = true;  // nodeft is computed when the learned form first needs it after a build
    int leaf_size = 16, morton_bits = 30;
    int64_t nleaves = 0;
    uint32_t* codes = nullptr;   // [nt] by caller's index
    int32_t* left = nullptr;     // [nt-1]
    int32_t* right = nullptr;    // [nt-1]
    int32_t* parent = nullptr;   // [2nt-1]
    int32_t* first = nullptr;    // [2nt-1]
    int32_t* last = nullptr;     // [2nt-1]
    int32_t* leaves = nullptr;   // [nt]
    int32_t* counter = nullptr;  // [nt-1] visit counters of the bottom-up pass
    double* mom = nullptr;       // [2nt-1][13]
    double* box = nullptr;       // [2nt-1][6]
    float* nodef = nullptr;      // [2nt-1][16] f32 node summary used by the far-field terms
    double* adm64 = nullptr;     // [2nt-1][4] f64 X_C, diag_C of the admissibility test
    float* adm32 = nullptr;      // [2nt-1][TP_ADM32_W] f32 outward/inward boxes, X_C, diag_C (pre-test),
                                 // and the member range and children (int bits)
    float* nodeft = nullptr;     // [2nt-1][16] f32 feature record (A, X, nubar, M2/A, diag) of the network
    int32_t* nleaves_d = nullptr;
    int64_t cap = 0;
};

struct tp_mlp_model;

// Quadrature rule per triangle (Sec. 3.1, 3.2): k points with barycentric
// coordinates bary[q][0..2] and weights w[q] (summing to 1).  k = 1 is the
// centroid rule; every point is then treated as an element carrying its
// triangle's vertices (for the exclusion) and normal.
struct tp_quad_rule {
    int k;
    double bary[6][3];
    double w[6];
};

// A run of a Barnes-Hut pair list: the far nodes (learned far field) or the
// near clusters apart from the leaf (near field) of one target leaf (leaf
// index li) at list[start, start + len), in traversal order.
struct tp_far_run {
    int64_t start;
    int32_t li;
    int32_t len;
};

struct tp_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    int64_t nv = 0, nt = 0, ntp = 0, nsup = 0;  // nt: elements = triangles x quadrature points
    bool have_mesh = false;
    tp_quad_rule quad{1, {{1.0 / 3, 1.0 / 3, 1.0 / 3}}, {1.0}};       // rule of the uploaded mesh
    tp_quad_rule quad_next{1, {{1.0 / 3, 1.0 / 3, 1.0 / 3}}, {1.0}};  // rule for the next full upload
    int64_t nt_tri = 0;             // triangles of the uploaded mesh
    int32_t* F_tri = nullptr;       // [nt_tri][3] caller's faces (quadrature rules with k > 1)

    // mesh
    double* V64 = nullptr;
    int32_t* F = nullptr;
    int32_t* v2t_off = nullptr;
    int32_t* v2t = nullptr;
    double* x64 = nullptr;
    double* nu64 = nullptr;
    double* w64 = nullptr;
    int32_t* perm = nullptr;
    int32_t* iperm = nullptr;
    uint32_t* codes = nullptr;      // Morton codes by caller's index
    uint32_t* codes_sorted = nullptr;
    int32_t* idx_tmp = nullptr;
    float* soa = nullptr;           // 10 planes of ntp
    float* src = nullptr;           // [ntp][TP_SRCW]
    int32_t* Fs = nullptr;          // [ntp][3]
    double* acc = nullptr;          // [TP_NACC][ntp]
    double* adjc = nullptr;         // [nt][3][3]: per element, its corners' contributions to dPhi/dV
    double* center = nullptr;       // [3] f64 centre subtracted before the f32 split
    double* bounds = nullptr;       // [6] min/max of centroids
    double* red = nullptr;          // reduction scratch
    double* scalar = nullptr;       // [16] device scalars: energies [0..1], Barnes-Hut counts [2..5], learned
                                    // energy correction [6], far rows [7], excluded pairs [8..9], pairs listed
                                    // for the near-field kernel [10..11]
    unsigned* derr = nullptr;       // device error word
    unsigned* adjbm = nullptr;      // bitmap nsup*nsup: super-tile pairs holding a vertex-sharing pair (or I == J)
    unsigned* flagged = nullptr;    // bitmap nsup*nsup: super-tile pairs not handled by the fast kernel
    unsigned* bmask = nullptr;      // [nsup*nsup][TP_BMASK_WORDS]: per super-tile pair (I, J), bit i*TP_NBLK+j set
                                    // when target block i of I and source block j of J hold a vertex-sharing pair
    int32_t* mlist = nullptr;       // compact list of masked super-tile pairs (I,J): a vertex-sharing pair inside
                                    // (sorted, so the order does not change between uploads)
    // exclusion bits of the masked blocks: per masked item m the blocks that need a per-pair test (xeff,
    // TP_BMASK_WORDS words), their first slot xbase[m]; per slot and target of the block 128 bits, set
    // where the pair is not admitted (shares a vertex; on diagonal blocks also source <= target)
    int32_t* item_index = nullptr;  // [nsup*nsup] masked item of (I, J), -1 for others
    unsigned* xeff = nullptr;       // [n_masked][TP_BMASK_WORDS]
    int32_t* xbase = nullptr;       // [n_masked + 1]
    int32_t* xcount = nullptr;      // [n_masked + 1] scratch of the prefix sum
    uint32_t* xmask = nullptr;      // [slots][128][4]
    int64_t x_slots = 0, x_cap = 0, x_item_cap = 0;
    uint64_t* xptrs = nullptr;      // [3] device copy of (xmask, xeff, xbase) for the masked kernel
    int32_t* plist = nullptr;       // compact list of unmasked pairs of nearby super-tiles (hi/lo centroids)
    int32_t* flist = nullptr;       // compact list of the remaining (fast) super-tile pairs
    int32_t* mcount = nullptr;      // [10]: counts of mlist, plist, 3 u64 pair counts (fast, precise, masked), count of flist
    unsigned* work = nullptr;       // [2] dynamic work counters of the persistent pair kernels
    float* tbox = nullptr;          // [nsup][6] f32 centroid boxes of the super-tiles
    // scratch of the hand-written key sort and compaction (tp_sort.cu)
    uint32_t* sort_hist = nullptr;  // per-tile digit counts and digit totals
    uint32_t* sort_ktmp = nullptr;  // ping-pong keys (32- or 64-bit)
    int32_t* sort_vtmp = nullptr;   // ping-pong values
    int64_t sort_hist_cap = 0, sort_kv_cap = 0;  // sort_kv_cap in 32-bit words
    double* host_pinned = nullptr;  // small pinned staging

    int64_t n_masked = 0;
    // the item lists above are refreshed on the next direct evaluation: 1 after a
    // positions-only upload (classification), 2 after a tree build re-sorted the
    // triangles (also the vertex-sharing blocks and exclusion bits)
    bool soa_stale = false;  // soa/src/Fs lag the positions (positions-only upload since the last refresh)
    int flags_stale = 0;
    int64_t n_precise = 0;
    int64_t n_fast = 0;
    int64_t pairs_fast = 0, pairs_precise = 0, pairs_masked_items = 0;  // unordered real pairs per item kind
    int64_t n_excluded_ordered = 0;       // ordered pairs T != S sharing a vertex
    int64_t n_excluded_edge_ordered = 0;  // ordered pairs T != S sharing an edge
    int64_t cap_nv = 0, cap_nt = 0, cap_ntp = 0, red_cap = 0;
    double* gradbuf = nullptr;      // [3nv] device staging of host gradients
    double* fieldbuf = nullptr;     // [7nt] device staging of host per-triangle fields (allocated on first use)
    float* vtmp = nullptr;          // [3nv] f32 staging of f32 positions
    double last_q = 6.0, last_pq = 2.0;
    int64_t nlaunch = 0;            // library kernels launched in the current call
    tp_tree tree;
    tp_mlp_model* mlp = nullptr;
    // fixed confining surface of the confinement energy (Eq. TPConf)
    bool have_conf = false;
    int64_t conf_nv = 0, conf_nt = 0, conf_ntp = 0, conf_cap_nv = 0, conf_cap_nt = 0;
    double* conf_V64 = nullptr;  // [nv][3]
    int32_t* conf_F = nullptr;   // [nt][3]
    float* conf_vtmp = nullptr;  // [3nv] f32 staging
    double* conf_y64 = nullptr;  // [3][nt] centroids
    double* conf_a64 = nullptr;  // [nt] areas
    float* conf_src = nullptr;   // [ntp][TP_SRCW] records relative to the evolving mesh's centre
    // far (leaf, cluster) pairs listed by the Barnes-Hut pass for the learned correction
    int32_t* far_list = nullptr;
    int32_t* far_leaf = nullptr;  // [far_cap] the leaf (index into the leaf list) of each listed row
    tp_far_run* far_runs = nullptr;
    unsigned long long* far_count = nullptr;  // [0] rows, [1] runs listed (may exceed the capacities), [2] work counter
    float* far_kf = nullptr;         // [far_xcap][8] factors - 1 of one window (column 7: in the training ranges)
    int64_t far_cap = 0, run_cap = 0;
    int64_t far_xcap = 0;             // rows of far_kf
    // the far runs sorted by first row (keys, run indices; unsorted inputs too), so
    // that each window of the learned passes visits only its own runs
    int64_t *run_key = nullptr, *run_key_s = nullptr;
    int32_t *run_ord = nullptr, *run_ord_s = nullptr;
    int64_t learned_window = TP_LEARNED_WINDOW;  // listed far rows per window of the learned passes
    int64_t* win_bnd = nullptr;  // first row of each window of the learned passes (a run's first row)
    int64_t win_bnd_cap = 0;
    // Barnes-Hut near field: (first member, count) of every near cluster whose
    // vertex box is apart from the target leaf's, in runs of one leaf
    int2* near_list = nullptr;
    tp_far_run* near_runs = nullptr;
    unsigned long long* near_count = nullptr;  // [0] entries, [1] runs listed (may exceed the capacities), [2] work counter
    int64_t near_cap = 0, nrun_cap = 0;
    // cluster-cluster form (tp_dual.cu): traversal frontier, far and near node
    // pairs, per-leaf partner lists, per-node derivative sums
    unsigned long long* dt_cnt = nullptr;  // [8] counters of the traversal and the passes
    int2* dt_front[2] = {nullptr, nullptr};
    int2* dt_far = nullptr;
    int2* dt_near = nullptr;
    int64_t dt_cap = 0, dt_far_cap = 0, dt_near_cap = 0;
    uint32_t* dt_off = nullptr;     // [nleaves + 1] partner-list offsets
    uint32_t* dt_cursor = nullptr;  // [nleaves + 1]
    int32_t* dt_node2leaf = nullptr;  // [2n - 1]
    double* dt_G = nullptr;         // [2n - 1][7] far-field derivatives per node
    double* dt_P = nullptr;         // [2n - 1][7] the same divided by the node area, weight term
    int2* dt_list = nullptr;        // partner leaves as (first member, count): touching, then apart
    tp_far_run* dt_runs = nullptr;  // runs of at most 128 apart partners of one leaf, for the near-field kernel
    int64_t dt_leaf_cap = 0, dt_node_cap = 0, dt_list_cap = 0, dt_run_cap = 0;

    tp_stats stats{};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};

    // allocation bookkeeping
    std::vector<void*> allocs;
    // test hook (tp_debug_fail_alloc): the allocation after this many more
    // successful ones fails as if the device were out of memory; -1 = never
    int64_t fail_alloc_after = -1;
};

// ---------------------------------------------------------------- host helpers
tp_status tp_set_err(tp_ctx* c, tp_status s, const char* fmt, ...);
tp_status tp_cuda_check(tp_ctx* c, cudaError_t e, const char* what);
#define TP_CU(call)                                                   \
    do {                                                              \
        cudaError_t _e = (call);                                      \
        if (_e != cudaSuccess) return tp_cuda_check(ctx, _e, #call);  \
    } while (0)
#define TP_TRY(call)                        \
    do {                                    \
        tp_status _s = (call);              \
        if (_s != TP_OK) return _s;         \
    } while (0)

tp_status tp_alloc(tp_ctx* ctx, void** p, size_t bytes);
void tp_free(tp_ctx* ctx, void* p);
// After a failed allocation: release every buffer derived from the mesh
// (mesh, tree, item lists, Barnes-Hut lists, sort scratch, confining surface)
// and zero their capacities, so that no later call sees a buffer that a
// half-finished resize left missing.  The model, stream and settings stay.
void tp_drop_mesh_state(tp_ctx* ctx);
template <typename T>
inline tp_status tp_alloc_t(tp_ctx* ctx, T** p, size_t n) {
    return tp_alloc(ctx, reinterpret_cast<void**>(p), n * sizeof(T) + 16);
}

// ---------------------------------------------------------------- launchers (per .cu file)
// tp_tri.cu
tp_status tp_launch_tri_data(tp_ctx* ctx);
tp_status tp_launch_morton_order(tp_ctx* ctx, int morton_bits);
tp_status tp_launch_sorted_soa(tp_ctx* ctx);
tp_status tp_launch_flagged(tp_ctx* ctx, bool topology);
tp_status tp_ensure_flagged(tp_ctx* ctx);
// refreshes soa/src/Fs after a positions-only upload, when a kernel first needs them
tp_status tp_ensure_sorted(tp_ctx* ctx);
tp_status tp_launch_fields(tp_ctx* ctx, const tp_params* prm, double* fw, double* fnu, double* fx);
tp_status tp_launch_conf_tri(tp_ctx* ctx);
tp_status tp_launch_expand_faces(tp_ctx* ctx);
tp_status tp_build_exclusion_bits(tp_ctx* ctx);
tp_status take_device_error(tp_ctx* ctx, const char* where);  // read and clear the device error word
tp_status tp_launch_mlp_tc(tp_ctx* ctx, const __nv_bfloat16* wb, const float* bias, const __nv_bfloat16* X,
                           int64_t rows, float* kf, int raw);
// The network on the listed far rows [w0, w1) with their input rows built in
// the kernel (features of nodeft[leaves[far_leaf[r]]] and nodeft[far_list[r]],
// normalised with mnorm): kf[r - w0] as tp_launch_mlp_tc with raw = 0.
struct tp_feat_src {
    const float* nodeft;
    const int32_t* far_list;
    const int32_t* far_leaf;
    const int32_t* leaves;
    const float* mnorm;
    int64_t nleaves, nnodes;  // bounds of the indices (checked in TP_DEBUG builds)
};
tp_status tp_launch_mlp_tc_feat(tp_ctx* ctx, const __nv_bfloat16* wb, const float* bias, const tp_feat_src& fs,
                                int64_t w0, int64_t w1, float* kf);
tp_status tp_launch_conf(tp_ctx* ctx, const tp_params* prm);
tp_status tp_launch_energy_scaled(tp_ctx* ctx, double mul, double* d_out);
tp_status tp_build_v2t(tp_ctx* ctx);
tp_status tp_count_excluded(tp_ctx* ctx);
// tp_direct.cu
tp_status tp_launch_direct_grad(tp_ctx* ctx, const tp_params* prm);
tp_status tp_launch_direct_energy(tp_ctx* ctx, const tp_params* prm, double* partials, int* nparts);
tp_status tp_launch_direct_f64(tp_ctx* ctx, const tp_params* prm, bool grad);
// unordered pairs of the direct gradient's timed launch (ev[0] / ev[1])
int64_t tp_direct_timed_pairs(const tp_ctx* ctx);
// compensated FP32 sums (TP_F32_KAHAN): per-target gather into ctx->acc
tp_status tp_launch_direct_kahan(tp_ctx* ctx, const tp_params* prm);
// Stable sort of n (32-bit key, 32-bit value) pairs by the low `bits` bits of
// the key (LSD radix, tp_sort.cu); inputs are left unchanged.
tp_status tp_sort_pairs_u32(tp_ctx* ctx, const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_out,
                            int32_t* vals_out, int64_t n, int bits);
tp_status tp_sort_pairs_u64(tp_ctx* ctx, const uint64_t* keys_in, const int32_t* vals_in, uint64_t* keys_out,
                            int32_t* vals_out, int64_t n, int bits);
// The entries >= 0 of in[0..n) in order to out, their number to *count_d (device).
tp_status tp_compact_nonneg(tp_ctx* ctx, const int32_t* in, int64_t n, int32_t* out, int32_t* count_d);
// Prefix sum of m counts (exclusive or inclusive, out may be in), total to *total_d if not null.
tp_status tp_scan_u32(tp_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t m, bool inclusive, int32_t* total_d);
// tp_adjoint.cu
// A node the Barnes-Hut traversal can reach: the root, or a child of a node
// with more than leaf_size members (a node of at most leaf_size members is
// never opened, tp_bh.cu).  Per-node records are written for these only.
__device__ __forceinline__ bool tp_node_reachable(const int32_t* __restrict__ parent,
                                                  const int32_t* __restrict__ first,
                                                  const int32_t* __restrict__ last, int64_t v, int leaf_size) {
    const int32_t p = parent[v];
    return p < 0 || last[p] - first[p] + 1 > leaf_size;
}

// Per-node passes cover TP_NODE_BLK consecutive nodes per block and first
// gather the reachable ones (under a tenth at leaf size 16) into shared
// memory, so that their FP64 work runs on dense lanes rather than on a few
// lanes of every warp.
constexpr int TP_NODE_THREADS = 256;
constexpr int TP_NODE_BLK = 1024;

// Compacts the reachable nodes of [v0, v0 + TP_NODE_BLK) into list (order
// unspecified) and returns their count; every thread of the block calls it.
__device__ __forceinline__ int tp_reachable_list(const int32_t* __restrict__ parent,
                                                 const int32_t* __restrict__ first,
                                                 const int32_t* __restrict__ last, int leaf_size, int64_t v0,
                                                 int64_t nn, int32_t* list, int* cnt) {
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < TP_NODE_BLK; j += blockDim.x) {
        const int64_t v = v0 + j;
        if (v < nn && tp_node_reachable(parent, first, last, v, leaf_size)) list[atomicAdd(cnt, 1)] = (int32_t)v;
    }
    __syncthreads();
    return *cnt;
}

tp_status tp_launch_adjoint(tp_ctx* ctx, const tp_params* prm, void* grad, int g_dtype);
tp_status tp_launch_energy_from_acc(tp_ctx* ctx, const tp_params* prm, double* d_out);
tp_status tp_launch_reduce_sum(tp_ctx* ctx, const double* in, int64_t n, double* d_out);
tp_status tp_launch_check_finite(tp_ctx* ctx);
// tp_lbvh.cu
tp_status tp_launch_tree_build(tp_ctx* ctx, int leaf_size, int morton_bits);
// tp_bh.cu
tp_status tp_launch_bh(tp_ctx* ctx, const tp_params* prm, bool learned);
// Barnes-Hut near-field kernel on runs of clusters apart from their leaf (tp_bh.cu)
tp_status tp_launch_near_runs(tp_ctx* ctx, int q, const int2* list, int64_t list_len, const tp_far_run* runs,
                              int64_t run_cap, unsigned long long* counters);
// cluster-cluster (dual-tree) form into ctx->acc (tp_dual.cu)
tp_status tp_launch_dual(tp_ctx* ctx, const tp_params* prm);
tp_status tp_dual_lists(tp_ctx* ctx, int64_t cap_front, int64_t cap_far, int64_t cap_near);
tp_status tp_dual_leaf_buffers(tp_ctx* ctx, int64_t nleaves, int64_t nn, int64_t entries, int64_t runs);
tp_status tp_launch_bh_sample(tp_ctx* ctx, double theta, uint32_t keep_u, uint64_t seed, int2* out, int64_t cap,
                              int32_t* counter);
// tp_mlp.cu
void tp_mlp_release(tp_ctx* ctx);
tp_status tp_mlp_node_features(tp_ctx* ctx);
tp_status tp_ensure_node_features(tp_ctx* ctx);
bool tp_mlp_ready(const tp_ctx* ctx);
const void* tp_mlp_weights(const tp_ctx* ctx);
const float* tp_mlp_bias(const tp_ctx* ctx);
const float* tp_mlp_norm(const tp_ctx* ctx);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ void tp_dev_error(unsigned* derr, unsigned bit) { atomicOr(derr, bit); }

// A bound inside the FP64 interval [lo, hi] whose FP32 outward roundings are
// olo = rd(lo), ohi = ru(hi): moving olo up (ohi down) by |x| 1.25e-7 + 1e-37
// passes at least one float spacing (|x| 2^-23 for normal x, below 1e-37
// otherwise), and the next float above rd(lo) is at least lo.  So
// tp_inward_lo(olo) >= lo and tp_inward_hi(ohi) <= hi: inward bounds, at most
// a few spacings tighter than the inward roundings, for a pre-test whose
// undecided cases go to FP64.
__device__ __forceinline__ float tp_inward_lo(float olo) { return fmaf(fabsf(olo), 1.25e-7f, olo) + 1e-37f; }
__device__ __forceinline__ float tp_inward_hi(float ohi) { return fmaf(-fabsf(ohi), 1.25e-7f, ohi) - 1e-37f; }

// The checked build's bounds check: in a TP_DEBUG build, false (with TP_DERR_BOUNDS
// recorded) when `ok` fails; always true in the release build.
__device__ __forceinline__ bool tp_dbg_ok(bool ok, unsigned* derr) {
#if TP_DEBUG
    if (!ok) {
        atomicOr(derr, TP_DERR_BOUNDS);
        return false;
    }
#else
    (void)ok;
    (void)derr;
#endif
    return true;
}

// Bulk copies (cp.async.bulk, completion counted in bytes on an mbarrier) and
// bounded mbarrier waits, shared by the pair kernels.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t tp_globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: true when the phase completed; false once limit_ns of
// wall-clock time has passed (the clock is read every 32 polls, and only
// after the first poll failed) or after TP_SPIN_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = TP_WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = tp_globaltimer_ns();
    for (uint32_t i = 1; i < TP_SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 31u) == 0u && tp_globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

