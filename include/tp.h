/*
 * tp.h - C ABI of the GB300 tangent-point energy library (libtp.so).
 *
 * The library evaluates the discrete tangent-point energy of a closed
 * triangulated surface and its gradient with respect to the vertex
 * positions (Porrmann, Bartels, Voigt, "Self-avoiding fluid deformable
 * surfaces"):
 *
 *   Phi(X) = scale * sum_{(T,S) ordered, T != S, T and S share no vertex}
 *                  w_T w_S |<nu_T, x_T - x_S>|^q / |x_T - x_S|^p
 *
 * x_T the centroid, nu_T the unit normal and w_T the area of flat triangle T.
 * This is Eq. (TP) of Sec. 2.2.2 with alpha = q, 2 alpha = p (the paper uses
 * alpha = 6, rho = 1e-4, i.e. scale = rho/alpha), discretised with one
 * quadrature point per triangle.  The gradient is the exact derivative of
 * this sum (the discrete counterpart of Eq. (dTP), Sec. 3.2).  The
 * Barnes-Hut mode clusters the inner sum only (Sec. 3.2).
 *
 * Conventions for every call:
 *  - Status codes are the only error channel; a failing call leaves the
 *    context usable and stores a message readable with tp_last_error().
 *  - All work is ordered on the CUDA stream given to tp_create().  Calls that
 *    return a host scalar synchronise that stream.
 *  - The library copies its inputs.  The caller owns every output buffer.
 *  - Pointers flagged TP_DEVICE_PTR are device addresses on the context's
 *    device; otherwise they are host addresses.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef TP_H
#define TP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tp_ctx tp_ctx;

typedef enum {
    TP_OK = 0,
    TP_E_ARG = 1,       /* invalid argument (null pointer, bad size, unsupported q/p ...) */
    TP_E_CUDA = 2,      /* a CUDA runtime call failed                                    */
    TP_E_STATE = 3,     /* no mesh uploaded, BH without a tree, LEARNED without a model  */
    TP_E_NONFINITE = 4, /* degenerate triangle, non-finite vertex or coincident admitted
                           centroids: the energy is +inf (finite only if embedded,
                           Sec. 2.2.2)                                                   */
    TP_E_TIMEOUT = 5,   /* a device-side bounded wait gave up (1 s)                      */
    TP_E_OOM = 6,       /* device allocation failed (the mesh must be uploaded again)    */
    TP_E_MODEL = 7      /* malformed far-field model file                                */
} tp_status;

/* TP_DIRECT: every admitted pair exactly.  TP_BH: the inner integral
 * clustered (Sec. 3.2), cluster monopoles per target.  TP_LEARNED: TP_BH with
 * the network's correction of the far terms.  TP_BH_DUAL: both integrals
 * clustered (the cluster-cluster scheme Sec. 3.2 compares with): node pairs
 * with vertex boxes apart and max(diag_A, diag_B) < theta |X_A - X_B| take
 * the monopole of both orderings, the gradient includes the derivatives
 * through the cluster moments.  The clustered forms need tp_tree_build. */
typedef enum { TP_DIRECT = 0, TP_BH = 1, TP_LEARNED = 2, TP_BH_DUAL = 3 } tp_mode;
typedef enum { TP_F32_F64ACC = 0, TP_F32_KAHAN = 1, TP_F64 = 2 } tp_prec;
enum { TP_DTYPE_F32 = 0, TP_DTYPE_F64 = 1 };

/* flags of tp_mesh_upload / tp_gradient */
#define TP_DEVICE_PTR 0x1u      /* pointers are device addresses                       */
#define TP_POSITIONS_ONLY 0x2u  /* re-upload V only; keep faces and derived topology   */
/* flags of tp_params */
#define TP_EXCLUDE_EDGE 0x4u    /* exclude only pairs sharing an edge (default: a vertex) */
#define TP_LEARNED_ENERGY 0x8u  /* TP_LEARNED: the network's factors correct the energy value only:
                                   every per-triangle derivative keeps the plain monopole (the gradient
                                   and tp_fields are TP_BH's) and the correction of the two energy
                                   channels is added to the returned energy */

typedef struct {
    int32_t q, p;   /* exponents: q even, p even; supported (6,12) and (8,16)       */
    double scale;   /* prefactor c (rho/alpha in Eq. TP); 1.0 for the bare sum      */
    int32_t mode;   /* tp_mode                                                      */
    double theta;   /* opening parameter of TP_BH / TP_LEARNED (Sec. 3.2)           */
    int32_t prec;   /* tp_prec                                                      */
    uint32_t flags; /* TP_EXCLUDE_EDGE, TP_LEARNED_ENERGY                           */
} tp_params;

/* Fill *p with the defaults: q=6, p=12, scale=1, DIRECT, theta=0.25, F32_F64ACC. */
void tp_params_default(tp_params* p);

/* Create a context on `device` whose work is ordered on `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL is the
 * legacy default stream).  *out receives the context; free with tp_destroy. */
tp_status tp_create(tp_ctx** out, int device, void* cuda_stream);
void tp_destroy(tp_ctx* ctx);

/* Message of the last failing call on ctx (owned by ctx, valid until the next call). */
const char* tp_last_error(const tp_ctx* ctx);

/* Upload a mesh.  V: nv*3 coordinates (v_dtype TP_DTYPE_F32 or _F64, row-major
 * [nv][3]); F: nt*3 int32 vertex indices, counter-clockwise seen from outside.
 * Flags: TP_DEVICE_PTR (V and F are device pointers), TP_POSITIONS_ONLY (F
 * is ignored and the previous connectivity is kept; nv must match).
 * Computes the per-triangle data (centroids, normals, areas; Sec. 3.2: the
 * data every quadrature point needs is cached contiguously) and orders the
 * triangles along a Morton curve.  Degenerate triangles or non-finite
 * coordinates give TP_E_NONFINITE.  Indices outside [0, nv) give TP_E_ARG. */
tp_status tp_mesh_upload(tp_ctx* ctx, const void* V, int64_t nv, int v_dtype, const int32_t* F, int64_t nt,
                         uint32_t flags);

/* Quadrature rule per triangle for the next full tp_mesh_upload (Sec. 3.1
 * and Sec. 3.2 integrate both integrals with a rule per element): npoints = 1
 * (the centroid, the default), 3 (degree 2: (2/3, 1/6, 1/6) and its
 * permutations) or 6 (degree 4, Strang and Fix).  Both integrals use the same
 * rule.  Every point becomes an element with its triangle's normal, the
 * weight om_q times the area, and its triangle's vertices, so pairs of points
 * of the same or of vertex-sharing triangles are left out.  With k > 1 points
 * the element count (tp_stats.nt, the tree, tp_fields) is k times the
 * triangle count, element i being point i % k of triangle i / k; the vertex
 * gradient is the exact chain rule through the points.  TP_E_ARG for other
 * counts.  The allocation-free entry point always uses the centroid. */
tp_status tp_set_quadrature(tp_ctx* ctx, int npoints);

/* Build the cluster tree used by TP_BH and TP_LEARNED from the current
 * positions: 30-bit Morton codes of the FP64 centroids (morton_bits must be
 * a multiple of 3, at most 30), radix tree of the sorted (code, index) keys,
 * cluster leaves of at most leaf_size triangles (1..32) and FP64 cluster
 * moments (area, area-weighted centroid, first and second normal moments,
 * vertex bounding box) - the "precomputed averages over a patch" of Sec. 3.2. */
tp_status tp_tree_build(tp_ctx* ctx, int leaf_size, int morton_bits);

/* Energy Phi of the uploaded mesh; *energy_out (host) receives it. */
tp_status tp_energy(tp_ctx* ctx, const tp_params* params, double* energy_out);

/* Energy (optional: energy_out may be NULL) and gradient dPhi/dV.  grad_out
 * receives nv*3 values of type g_dtype (TP_DTYPE_F32 / _F64), row-major like
 * V; it is a device pointer when flags has TP_DEVICE_PTR, else host memory. */
tp_status tp_gradient(tp_ctx* ctx, const tp_params* params, double* energy_out, void* grad_out, int g_dtype,
                      uint32_t flags);

/* Energy (energy_out may be NULL) and the per-triangle derivatives that the
 * vertex gradient is assembled from: for every triangle T, in the caller's
 * order, dPhi/dw_T (area) into fw[nt], dPhi/dnu_T (unit normal, taken as a
 * free vector) into fnu[nt][3] and dPhi/dx_T (centroid) into fx[nt][3], all
 * FP64 and including the prefactor c.  These are the one-point counterparts
 * of the fields f_K, f_nu and f of Eq. (dTP_reordered), Sec. 3.2, which the
 * surface finite-element assembly consumes.  Every mode (direct, Barnes-Hut,
 * learned) and precision of tp_gradient is supported.  The outputs are device
 * pointers when flags has TP_DEVICE_PTR, else host memory; any of them may be
 * NULL.  Errors as tp_gradient. */
tp_status tp_fields(tp_ctx* ctx, const tp_params* params, double* energy_out, double* fw, double* fnu, double* fx,
                    uint32_t flags);

/* Upload the fixed confining surface S_conf of the confinement energy,
 * Eq. (TPConf), Sec. 2.2 (Confinement): vertices V[nv][3] (v_dtype f32/f64)
 * and faces F[nt][3], host memory or device memory with TP_DEVICE_PTR; the
 * library copies them.  Only the centroids and areas of its triangles enter
 * (its normal never does, so orientation does not matter and the surface may
 * be non-smooth).  Face indices outside [0, nv) give TP_E_ARG, non-finite
 * coordinates TP_E_NONFINITE.  It stays until the next tp_conf_upload and is
 * independent of tp_mesh_upload. */
tp_status tp_conf_upload(tp_ctx* ctx, const void* V, int64_t nv, int v_dtype, const int32_t* F, int64_t nt,
                         uint32_t flags);

/* Confinement energy of the uploaded (evolving) mesh S against S_conf,
 *   Phi_conf = c sum_{T in S} sum_{K in S_conf} w_T a_K |nu_T.(x_T - y_K)|^q / |x_T - y_K|^p
 * (one centroid point per flat triangle on both surfaces; c = rho_conf/alpha is
 * params->scale), and optionally its gradient with respect to the vertices of
 * S (S_conf does not move): grad_out as in tp_gradient, or NULL for the energy
 * only.  params->mode must be TP_DIRECT; prec TP_F32_F64ACC (FP32 pair terms,
 * FP64 accumulation) or TP_F64.  Touching surfaces give TP_E_NONFINITE with
 * energy +inf; no confining surface gives TP_E_STATE. */
tp_status tp_conf_gradient(tp_ctx* ctx, const tp_params* params, double* energy_out, void* grad_out, int g_dtype,
                           uint32_t flags);

/* Load the far-field network used by TP_LEARNED from a file written by
 * tp_far_model_save: header {"TPFM", version 1, 24, 64, 7, nparam, theta,
 * q, p, step}, then the feature mean/std/min/max [4][24] f32 and the FP32
 * master parameters.  Malformed files give TP_E_MODEL. */
tp_status tp_far_model_load(tp_ctx* ctx, const char* path);

/* ------------------------------------------------------------------ */
/* Learned far field: a network 24 -> 64 -> 64 -> 64 -> 7 (tanh-form GELU,
 * BF16 weights on the tensor cores, FP32 accumulation) predicts, for an
 * admissible (target leaf, cluster) pair, log-factors correcting the
 * channels of the Barnes-Hut monopole far term (the paper has no network:
 * its clustered inner integral uses plain averages over the patch, Sec. 3.2).
 * Parameters: FP32, packed W1[64][24] b1 W2[64][64] b2 W3[64][64] b3 W4[7][64]
 * b4 (10,375 numbers).  All pointers below are host pointers. */

/* Fresh network with Xavier-uniform weights from a counter-based generator. */
tp_status tp_far_model_init(tp_ctx* ctx, uint64_t seed);
tp_status tp_far_model_save(tp_ctx* ctx, const char* path);
/* Set / read the FP32 parameters and (optional) feature normalisation [4][24]. */
tp_status tp_far_set_params(tp_ctx* ctx, const float* params, const float* norm);
tp_status tp_far_get_params(tp_ctx* ctx, float* params, float* norm);
/* Training set: sampled admissible pairs of the current tree with features
 * [24], labels [8] (7 used: log(exact member sum / monopole) per channel) and
 * masks [8]; the labels come from direct sums over the members.  Each
 * admissible pair at opening angle theta is kept with probability `keep`
 * (counter-based hash of the pair and seed), at most max_pairs are added;
 * max_pairs = 0 only counts the kept pairs into *n_added. */
tp_status tp_far_dataset_reset(tp_ctx* ctx);
tp_status tp_far_dataset_size(tp_ctx* ctx, int64_t* n);
tp_status tp_far_sample_pairs(tp_ctx* ctx, double theta, double keep, uint64_t seed, int64_t max_pairs,
                              int64_t* n_added);
tp_status tp_far_dataset_get(tp_ctx* ctx, int64_t i0, int64_t n, float* feat, float* lab, float* mask,
                             int32_t* pairs);
/* Feature mean/std and in-distribution ranges from the training set. */
tp_status tp_far_fit_normalisation(tp_ctx* ctx);
/* `steps` AdamW steps (b1 0.9, b2 0.999, eps 1e-8, decoupled decay wd) on
 * batches of `batch` rows; *last_loss: masked mean-square loss of the last batch. */
tp_status tp_far_train(tp_ctx* ctx, int64_t steps, int64_t batch, double lr, double wd, uint64_t seed,
                       double* last_loss);
/* Network on given rows X[n][24] (raw, or normalised if bit 0 of normalised
 * is set): outputs Y[n][7].  With targets or masks [n][8] the training kernel
 * runs and also returns the loss and the parameter gradient grad[10375]; with
 * neither, the inference network of TP_LEARNED evaluations runs (tcgen05 on
 * the tensor cores; with bit 1 of normalised set, the register-resident
 * mma.sync variant) and grad and loss are zeroed.  Each output may be NULL.
 * For tests. */
tp_status tp_far_eval(tp_ctx* ctx, const float* X, int64_t n, int normalised, const float* tgt, const float* mask,
                      float* Y, float* grad, double* loss);
/* One AdamW step with the given gradient [10375].  For tests. */
tp_status tp_far_adamw_step(tp_ctx* ctx, const float* grad, double lr, double wd);

/* ------------------------------------------------------------------ */
/* Inspection entry points (host outputs, for tests and benchmarks)   */

typedef struct {
    int64_t nt, nv;
    int64_t pairs_exact;   /* ordered pairs evaluated exactly in the last call        */
    int64_t far_terms;     /* (target, cluster) far-field terms in the last call      */
    int64_t far_pairs;     /* ordered pairs represented by those far terms            */
    int64_t learned_terms; /* far terms evaluated by the network                       */
    int64_t tile_pairs, tile_pairs_masked, tile_pairs_precise;
    float ms_kernel;       /* device time of the dominant kernel of the last call
                              (direct: the pair launch of the PRECISE and FAST items;
                              Barnes-Hut and learned: the near-field kernel)          */
    float ms_total;        /* device time of the whole last call                       */
    int64_t kernel_launches; /* library kernels launched by the last call (CUDA library
                                calls such as the radix sort are not counted)        */
    int64_t kernel_pairs;    /* pairs evaluated by the dominant kernel launch of the
                                last call, for throughput accounting: direct mode, the
                                unordered pairs of the PRECISE and FAST items;
                                Barnes-Hut and learned, the ordered (target, source)
                                pairs of the near-field kernel                        */
    int64_t far_rows;        /* (target leaf, cluster) far pairs of the last Barnes-Hut
                                or learned call: in the learned form, the rows the
                                network evaluated                                     */
} tp_stats;

tp_status tp_get_stats(const tp_ctx* ctx, tp_stats* out);

/* Per-triangle data in the library's (Morton) order: perm[nt] original index,
 * x[nt*3] f64 centroids, nu[nt*3] f64 normals, w[nt] f64 areas.  Any pointer may be NULL. */
tp_status tp_debug_tri_data(tp_ctx* ctx, int32_t* perm, double* x, double* nu, double* w);

/* Per-triangle derivatives of the last tp_gradient call, in ORIGINAL triangle
 * order (without scale): gw[nt] = dPhi/dw_T, gnu[nt*3], gx[nt*3]. */
tp_status tp_debug_accum(tp_ctx* ctx, double* gw, double* gnu, double* gx);

/* Rows of the learned far field processed at a time.  A TP_LEARNED
 * evaluation lists its (leaf, cluster) far pairs, then computes features,
 * runs the network and applies its factors in windows of at most `rows`
 * listed pairs; the network rows and factors take 100 B per row of the
 * window.  rows = 0 restores the default of 32 Mi rows (about 3.4 GB).
 * Windows end on the first row of a run of one leaf's pairs, so they may
 * hold up to 255 rows more, and no run is split: results do not depend on
 * the window beyond the order of the FP64 atomic sums.  An implementation
 * control with no counterpart in the paper.  TP_E_ARG for rows in 1..31. */
tp_status tp_set_learned_window(tp_ctx* ctx, int64_t rows);

/* The tree of the last tp_tree_build: codes[nt] (by original index),
 * perm[nt], left/right[nt-1], first/last[2nt-1], leaves[*nleaves] (capacity nt),
 * mom[(2nt-1)*13], box[(2nt-1)*6].  Any pointer may be NULL. */
tp_status tp_debug_tree(tp_ctx* ctx, uint32_t* codes, int32_t* perm, int32_t* left, int32_t* right,
                        int32_t* first, int32_t* last, int32_t* leaves, int64_t* nleaves, double* mom,
                        double* box);

/* Energy and gradient of the direct form for callers that cannot allocate
 * device memory - code recording a CUDA graph (allocation is not allowed
 * while a stream is being captured), plug-ins whose host application owns
 * all device memory through its own pool, loops that forbid allocation once
 * running.  The paper has no counterpart: this is a deployment variant of
 * tp_gradient in TP_DIRECT mode with the same arithmetic (FP32 pair terms,
 * FP64 accumulation).
 *   V [nv][3] f64, F [nt][3] i32: device inputs on the current device.
 *   energy_out (1 f64) and grad_out ([nv][3] f64): device outputs, caller-owned.
 *   params: q/p as tp_gradient, mode must be TP_DIRECT and prec
 *   TP_F32_F64ACC (other modes and precisions give TP_E_ARG); scale and
 *   TP_EXCLUDE_EDGE are honoured.  cuda_stream orders the work; the call
 *   does not synchronise.  errbuf (may be NULL) receives a message on failure.
 * All scratch is one fixed __device__ array sized for at most 65536
 * triangles (about 7 MB, kept by every GPU that loads the library until the
 * process exits); larger meshes give TP_E_ARG.  The first call on a device
 * looks up that array's address (cudaGetSymbolAddress) and keeps it for the
 * life of the process; make that first call before any stream capture.  The
 * kept address assumes the device's primary context is never reset
 * (cudaDeviceReset) and that callers use the primary context.  Calls share
 * the array: calls that overlap on the GPU race.
 * The inputs are not validated on the device, since the call does not
 * synchronise: a face index outside [0, nv) (the triangle is skipped by the
 * pull-back and its data set to NaN), a degenerate (zero-area) triangle and
 * coincident admitted centroids all show as NaN or inf in energy_out and
 * grad_out, with status TP_OK. */
tp_status tp_gradient_direct_noalloc(const double* V, int64_t nv, const int32_t* F, int64_t nt,
                                     const tp_params* params, double* energy_out, double* grad_out,
                                     void* cuda_stream, char* errbuf, int64_t errbuf_len);

/* One 128 x N x K tensor-core GEMM D = A B^T (A [128][K], B [N][K] BF16 as
 * raw 16-bit patterns, D [128][N] FP32; host arrays; K in {16, 32, 64},
 * N in {16, 64}) through the operand layout, descriptors and accumulator
 * read-back of the learned far field's network kernel.  Synchronises the
 * device.  TP_E_ARG on bad sizes.  For tests. */
tp_status tp_debug_tc_gemm(int device, const uint16_t* A, int K, const uint16_t* B, int N, float* D);

/* Failure paths, for tests (no GPU fault is involved in either):
 * tp_debug_wait_timeout launches one block that arms an mbarrier for bytes no
 * copy delivers and waits on it with the pair kernels' bounded wait, limited
 * to limit_ms (0 < limit_ms <= 1000); the wait gives up, the kernel sets the
 * device error word and returns, and the call reports TP_E_TIMEOUT (the
 * context stays usable).  tp_debug_fail_alloc makes the allocation after
 * `after` more successful ones fail once as if the device were out of memory
 * (after < 0 disarms it).  Any TP_E_OOM, simulated or real, releases the
 * mesh, tree, pair lists and confining surface of the context (the model,
 * stream and settings stay): upload the mesh again to continue. */
tp_status tp_debug_wait_timeout(tp_ctx* ctx, double limit_ms);
tp_status tp_debug_fail_alloc(tp_ctx* ctx, int64_t after);

/* The cluster-tree build's own stable key sort and compaction on a host
 * array, for tests: keys[n] are sorted by their low `bits` bits (1..32) with
 * ties in input order; keys_out receives the sorted keys and perm_out the
 * input position of each.  With compact_out and ncompact not NULL, the keys
 * read as int32 are also compacted: the entries >= 0, in order, to
 * compact_out (capacity n) and their number to *ncompact.  Host buffers;
 * synchronises the context stream; allocates and frees its own buffers. */
tp_status tp_debug_sort(tp_ctx* ctx, const uint32_t* keys, int64_t n, int bits, uint32_t* keys_out,
                        int32_t* perm_out, int32_t* compact_out, int32_t* ncompact);

/* Library version string. */
const char* tp_version(void);

/*
 * Measured FP32 throughput of this GPU: independent chains of FMAs, scalar
 * (packed = 0, FFMA) or FP32x2 (packed = 1, FFMA2), on every SM with
 * `warps_per_sm` resident warps (1..64) and `chains` (2, 4, 8 or 16)
 * independent accumulators per thread.  Writes the best of three timed
 * launches (after one warm-up) in TFLOP/s to *tflops_out (an FMA counts as
 * 2 flops).  It is the measured counterpart of the FP32 peak the pair kernels
 * are compared with (SMs x 128 lanes x 2 x clock).  Runs on `cuda_stream`
 * (NULL: the legacy default stream) and synchronises it; allocates and frees a
 * small output buffer.  TP_E_ARG on bad arguments, TP_E_CUDA on a CUDA error.
 */
tp_status tp_measure_fp32_peak(int device, void* cuda_stream, int packed, int warps_per_sm, int chains,
                               double* tflops_out);

#ifdef __cplusplus
}
#endif
#endif /* TP_H */
