/*
 * mlps.h -- C ABI of the GB300 (sm_103a) MLP-Splatting renderer.
 *
 * MLP-Splatting represents a scene by K primitives, each a unit-Mahalanobis ellipsoid (centre
 * mu, per-axis scale s, rotation quaternion q; Sec. 3.1) carrying its own small MLP that maps an
 * encoded (local position, view direction) input to colour and density (Sec. 3.1-3.2). A pixel
 * is rendered by intersecting its ray with the primitives, ordering the hit intervals by the
 * soft contact point t* of Eq. 2 (which is the chord midpoint), placing S midpoint samples in
 * each interval, evaluating the primitive's MLP at every sample, and compositing front to back
 * (Eq. 6 and its sampled form in App. D.1).
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers unless marked "host". All floats are FP32.
 *  - The caller owns every buffer. The library never allocates or frees device memory and keeps
 *    no state between calls (except the optional host-side profiler below). All work is
 *    enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is asynchronous.
 *  - Synchronous argument errors return a status immediately and enqueue nothing.
 *    Data-dependent errors found on the device (hit-capacity overflow, non-finite values,
 *    bounded waits that gave up) are recorded in a status word inside the `saved` or
 *    `scratch` region and returned by mlps_read_status(). No call traps, aborts or hangs.
 *  - Image layouts: rgb [V, H, W, 3], trans [V, H, W], feat [V, H, W, F], all row-major,
 *    V = n_views, F = feat_dim + slot_dim (the MLP's extra outputs, then the slot channels).
 *    Gradients dL/d* use the same layouts.
 *  - Primitive layouts: centers [K, 3], scales [K, 3] (linear, > 0), quats [K, 4] as
 *    (w, x, y, z) with any nonzero norm (normalised inside; gradients include the
 *    normalisation), weights in the canonical FP32 layout [K, P] described below.
 *  - Canonical FP32 weight layout (P = mlps_param_count floats per primitive): for each layer l
 *    in order, W_l as [out_l, in_l] row-major, then b_l as [out_l]. Layer 0 reads the encoded
 *    input, hidden layers have `hidden_width` outputs with ReLU, the last layer has
 *    4 + feat_dim linear outputs ordered (r, g, b, sigma, f_0 .. f_{F-1}); colour = sigmoid,
 *    density = softplus (Sec. 3.2), features are used as is. With slot_dim = C > 0 the four
 *    slot embeddings follow as [4, C] (Sec. 3.4).
 *  - Encoding (Eq. 5): per scalar p, (sin(2^0 pi p), cos(2^0 pi p), ..., sin(2^{L-1} pi p),
 *    cos(2^{L-1} pi p)), concatenated over the 3 components of the scale-normalised local
 *    position x' = S^-1 R^T (x - mu) (L = xyz_freqs; raw x' when 0), then over the 3 components
 *    of the unit world ray direction (L = dir_freqs; omitted when 0).
 *  - Camera: pinhole, pixel centres at +0.5, OpenCV axes. world_to_cam = [R | t] row-major;
 *    ray origin -R^T t, direction normalise(R^T ((x + .5 - cx)/fx, (y + .5 - cy)/fy, 1)).
 */
#ifndef MLPS_H
#define MLPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLPS_ABI_VERSION 7
#define MLPS_MAX_VIEWS 64

typedef int32_t mlps_status;
enum {
  MLPS_OK = 0,
  MLPS_ERR_INVALID_ARGUMENT = 1,   /* null pointer, bad size, non-finite config value */
  MLPS_ERR_UNSUPPORTED = 2,        /* valid but not implemented shape/precision combination */
  MLPS_ERR_WORKSPACE_TOO_SMALL = 3,/* saved/scratch smaller than mlps_workspace_size() */
  MLPS_ERR_CAPACITY_OVERFLOW = 4,  /* device: a ray had > max_hits_per_ray hits, or the total
                                      hit records exceeded the workspace capacity */
  MLPS_ERR_TIMEOUT = 5,            /* device: a bounded wait gave up */
  MLPS_ERR_NONFINITE = 6,          /* device: non-finite value met */
  MLPS_ERR_CUDA = 7                /* a CUDA runtime call failed */
};

typedef int32_t mlps_precision;
enum {
  MLPS_FP32 = 0,      /* MLP on FP32 FMA (no TF32) */
  MLPS_BF16 = 1,      /* MLP on tcgen05 tensor cores, BF16 operands, FP32 accumulation */
  MLPS_FP8_E4M3 = 2   /* MLP on tcgen05 tensor cores, E4M3 operands with per-primitive scales */
};

/* Renderer configuration. Zero-initialise, then set the fields; mlps_config_default() fills the
 * defaults for a model shape. */
typedef struct {
  int32_t xyz_freqs;            /* L of the local-position encoding (Eq. 5); 0 = raw x' */
  int32_t dir_freqs;            /* L of the view-direction encoding; 0 = no direction input */
  int32_t hidden_width;         /* hidden layer width: 32, 64 or 128 */
  int32_t hidden_layers;        /* number of hidden (ReLU) layers, 1..6 */
  int32_t feat_dim;             /* extra linear outputs composited like colour, 0..32 */
  int32_t samples;              /* S midpoint samples per hit interval, 1..128 */
  int32_t precision;            /* mlps_precision of the MLP contractions */
  int32_t max_hits_per_ray;     /* per-ray sorted hit capacity, 1..64 */
  float hit_capacity_per_ray;   /* hit-record capacity = ceil(rays * this), > 0 */
  float t_eps;                  /* early termination: stop compositing once T < t_eps (0: never) */
  int32_t tile;                 /* screen tile edge in pixels for binning: 16 (default) or 8 */
  int32_t mlp_groups;           /* chunks of 128 sample rows in flight per CTA in the forward
                                   tensor-core MLP (2..5 at width 64 in BF16, 2..6 in E4M3,
                                   3 with a feature head,
                                   2 at width 128); 0 = library default. mlps_autotune_batch
                                   picks it together with `tile`. */
  int32_t contact;              /* 0: S midpoint samples of the local position per hit interval;
                                   1: contact-point mode of Sec. 3.2 (Eq. 2-4): one sample per
                                   hit (samples must be 1) whose MLP input is gamma([d; delta]),
                                   d the unit ray direction and delta = mu - p* the offset from
                                   the contact point p* = o + max(0, t*) d to the centre (Eq. 3);
                                   the hit's alpha uses its chord length. The forward pass
                                   runs in every precision. The backward pass runs in FP32,
                                   and on the tensor cores (BF16 / E4M3 precisions) for the
                                   paper's model (xyz_freqs = dir_freqs = 6, hidden width 32
                                   or 64, at least two hidden layers, no feature head);
                                   mlps_render_backward returns MLPS_ERR_UNSUPPORTED for other
                                   contact models in those precisions. */
  int32_t slot_dim;             /* C of the feature slots of Sec. 3.4 (0 = none; a multiple of 4,
                                   <= 2048): every primitive also carries four slot embeddings
                                   e_k in R^C, stored after its MLP parameters (canonical weights
                                   [K, mlps_param_count] = MLP, then e_0..e_3). A hit's feature is
                                   f = sum_k g_k e_k with g = softmax_k(a_k . u),
                                   u = clip_[-1,1]^3(R^T (mu - p*) / s) and a_k the unit vertices
                                   (+-1, +-1, +-1)/sqrt(3) (even number of minus signs) of a
                                   regular tetrahedron; the rendered map
                                   F_slot = sum_i w_i f_i uses each hit's compositing weight w_i
                                   and is returned in the `feat` rows after the feat_dim MLP
                                   outputs (rows of feat_dim + slot_dim floats). */
  int32_t tile_sort;            /* 0: every ray composites its hits in its own order of
                                   max(0, t*) (Eq. 2, exact); 1: in the order of max(0, t*) along
                                   the virtual ray through the centre of its `tile` x `tile`
                                   screen tile (the approximate order of Sec. 3.3 and App. A.4),
                                   ties by primitive index. Hit intervals, samples and MLP inputs
                                   stay per ray. */
  int32_t early_stop_wave;      /* 0: the MLP forward evaluates every hit interval, and early
                                   termination (t_eps) only stops the composite. k > 0 (at most
                                   max_hits_per_ray): it runs in two depth waves, first the
                                   first k hits of every ray, then the later hits of the rays
                                   whose composite has not stopped within their first k, so
                                   that the intervals behind a ray's termination point are not
                                   evaluated (App. B.2). The outputs are the same as with 0.
                                   Not with feature slots (MLPS_ERR_UNSUPPORTED). */
} mlps_config;

typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float world_to_cam[12];       /* row-major [R | t] */
  float near_t;                 /* samples start at max(t0, near_t); >= 0 */
} mlps_camera;

/* One scene. Pointers are device pointers. `weights` is the packed blob produced by
 * mlps_pack_weights() for config->precision (mlps_weight_stride() bytes per primitive). */
typedef struct {
  int32_t K;
  const float* centers;         /* [K, 3] */
  const float* scales;          /* [K, 3] */
  const float* quats;           /* [K, 4] (w, x, y, z) */
  const void* weights;          /* [K, stride] packed, 256-byte aligned */
} mlps_scene;

/* ---------------------------------------------------------------------------------------- */
/* Introspection                                                                              */

/* ABI version (MLPS_ABI_VERSION of the build). */
int32_t mlps_abi_version(void);

/* Short English text for a status code; never NULL. */
const char* mlps_status_string(mlps_status s);

/* Fill *cfg with defaults: S = 32, FP32, max_hits_per_ray = 64, hit_capacity_per_ray = 8,
 * t_eps = 1e-6 (early termination of Sec. B.2; the paper does not give the threshold),
 * tile = 16. Shape fields are set from the arguments. Returns MLPS_ERR_INVALID_ARGUMENT on a
 * NULL cfg. */
mlps_status mlps_config_default(mlps_config* cfg, int32_t xyz_freqs, int32_t dir_freqs,
                                int32_t hidden_width, int32_t hidden_layers, int32_t feat_dim);

/* Input width of layer 0 after encoding: (xyz_freqs ? 6 xyz_freqs : 3) + 6 dir_freqs. */
int32_t mlps_input_dim(const mlps_config* cfg);

/* Floats per primitive in the canonical FP32 weight layout (P). 0 on invalid config. */
int64_t mlps_param_count(const mlps_config* cfg);

/* Bytes per primitive of the packed weight blob for cfg->precision. 0 on invalid config. */
int64_t mlps_weight_stride(const mlps_config* cfg);

/* Validates a config. MLPS_OK, or the reason it cannot be rendered. */
mlps_status mlps_check_config(const mlps_config* cfg);

/* ---------------------------------------------------------------------------------------- */
/* Weights                                                                                    */

/* Convert canonical FP32 weights [K, P] (device) into the packed blob for cfg->precision
 * (device, [K, mlps_weight_stride] bytes, 256-byte aligned). FP32: a copy re-laid for the SIMT
 * kernels; BF16: operand tiles in the tensor-core shared-memory layout plus FP32 biases;
 * FP8-E4M3: the same with per-(primitive, layer) power-of-two scales. Enqueued on `stream`. */
mlps_status mlps_pack_weights(const mlps_config* cfg, int32_t K, const float* weights_fp32,
                              void* packed, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Rendering                                                                                  */

/* Bytes of the two workspaces a render of n_views cameras (host array) needs.
 * `saved` carries the forward state to the backward pass; `scratch` is reused per call.
 * Both must be 256-byte aligned device memory. */
mlps_status mlps_workspace_size(const mlps_config* cfg, int32_t K, const mlps_camera* cams,
                                int32_t n_views, size_t* saved_bytes, size_t* scratch_bytes);

/* Forward render (Sec. 3.2-3.3). cams is a HOST array of n_views cameras (1..MLPS_MAX_VIEWS),
 * all of the same width and height. Writes rgb [V,H,W,3] and trans [V,H,W] (final
 * transmittance; background is black), and feat [V,H,W,feat_dim + slot_dim] when that is > 0
 * (NULL allowed when it is 0). Fills `saved` for mlps_render_backward. */
mlps_status mlps_render_forward(const mlps_config* cfg, const mlps_scene* scene,
                                const mlps_camera* cams, int32_t n_views, float* rgb,
                                float* trans, float* feat, void* saved, size_t saved_bytes,
                                void* scratch, size_t scratch_bytes, void* stream);

/* Backward of the forward call that filled `saved` (same cfg, scene and cams). Given dL/drgb
 * (required), dL/dtrans and dL/dfeat (either may be NULL = zero), OVERWRITES
 * d_weights [K, P] (canonical FP32 layout, slot embeddings included), d_centers [K,3],
 * d_scales [K,3], d_quats [K,4]. The slot features' gradient reaches the embeddings, the
 * compositing weights (and through them the MLP) and the pose (through u).
 * The MLP is recomputed, not stored. Hit sets and orders are piecewise constant and are not
 * differentiated.
 * Shapes the backward covers (others return MLPS_ERR_UNSUPPORTED before anything is enqueued;
 * the forward covers every valid configuration):
 *  - FP32: samples <= 64; hidden width 32 or 64 while both layouts of a primitive's weights fit
 *    in shared memory (up to three 64-wide hidden layers) and its weight gradient fits 1024 tiles
 *    of 4 x 4; hidden width 128 with input and output widths <= 64.
 *  - BF16 / E4M3 (the backward recomputes in BF16): hidden width 32 or 64 with up to six hidden
 *    layers, at most 12 feature outputs and the midpoint encodings (xyz_freqs 0 or 6), or the
 *    paper's contact-point model; hidden width 128 with up to four hidden layers on the tensor
 *    cores (xyz_freqs 6, dir_freqs 4, at most 16 feature outputs, a multiple of 4), other
 *    width-128 networks with samples <= 64 in an FP32-FMA kernel reading the BF16 weights. */
mlps_status mlps_render_backward(const mlps_config* cfg, const mlps_scene* scene,
                                 const mlps_camera* cams, int32_t n_views, const float* d_rgb,
                                 const float* d_trans, const float* d_feat, const void* saved,
                                 size_t saved_bytes, float* d_weights, float* d_centers,
                                 float* d_scales, float* d_quats, void* scratch,
                                 size_t scratch_bytes, void* stream);

/* Forward render like mlps_render_forward, for callers that cannot allocate device memory
 * (for example code whose device memory belongs to another allocator, or a frame loop that must
 * not call cudaMalloc / cudaFree because they can synchronise the device or fail mid-frame).
 * The paper has no counterpart; this is a convenience of this library.
 * Instead of caller-provided `saved` / `scratch` buffers it uses one fixed workspace of 32 MiB
 * held in a static device array of the library (every GPU that loads the library keeps it
 * until the process exits). Renders whose mlps_workspace_size() total (saved rounded up to 256
 * bytes, plus scratch) exceeds 32 MiB are rejected with MLPS_ERR_WORKSPACE_TOO_SMALL before
 * anything is enqueued. It calls no cudaMalloc / cudaFree and no allocating routine.
 * The first call on a device looks up the array's device address with that device current.
 * Under CUDA's lazy module loading (the default) that lookup is also what loads the array's
 * module on the device and reserves its 32 MiB there, so the first call can fail for lack of
 * device memory (MLPS_ERR_CUDA) and can synchronise: make it once, before the frame loop and
 * before any stream capture. Later calls reserve nothing. All calls share the one array and it
 * keeps the last call's contents (each call clears what it needs), so calls that overlap on the
 * GPU (other streams, other host threads) race; serialise them. There is no backward pass for
 * this variant. If `device_status` (device pointer, may be NULL) is given and the call returns
 * MLPS_OK, the call's device status word (MLPS_OK or the device-detected error, as
 * mlps_read_status would return) is copied there asynchronously on `stream` at the end of the
 * call; when the call returns any other status, `device_status` is not written. */
mlps_status mlps_render_forward_static(const mlps_config* cfg, const mlps_scene* scene,
                                       const mlps_camera* cams, int32_t n_views, float* rgb,
                                       float* trans, float* feat, int32_t* device_status,
                                       void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Batched rendering: many scenes (primitive sets) and resolutions in one call                */
/*
 * The renderer of Sec. 3.2-3.3 applied to a batch of independent items, each one view of one
 * scene. The scenes' primitives are passed as ONE set of scene arrays (mlps_scene with the
 * scenes' primitives concatenated, K = their total, weights packed with mlps_pack_weights);
 * item i renders primitives [prim_offset, prim_offset + prim_count) of those arrays through its
 * own camera at the camera's own resolution. Items may share primitives (several views of one
 * scene). Every stage runs as one launch over all items: the MLP stage is one persistent launch
 * over the chunks of every primitive of every scene. No call synchronises, allocates or reads
 * device memory on the host, so a batch (forward and backward) can be captured in a CUDA graph
 * and replayed; the item table is read on the host at call time and baked into the launches.
 *
 * Image layout: items are concatenated in order. Item i's pixels start at
 * P_i = sum_{j < i} width_j * height_j; rgb [P, 3], trans [P], feat [P, F] and their gradients,
 * each item row-major inside its block (pixel P_i + y * width_i + x). Gradients dL/dweights,
 * dL/dcenters, ... cover all K primitives (zero for primitives no item renders). At most
 * MLPS_MAX_VIEWS items. */
typedef struct {
  int32_t prim_offset;  /* first primitive of the item's scene in the batch's scene arrays */
  int32_t prim_count;   /* its primitives; prim_offset + prim_count <= K */
  mlps_camera cam;      /* the item's view (host struct), any resolution */
} mlps_batch_item;

/* Workspace of a batch (host items[n_items]); same meaning as mlps_workspace_size. */
mlps_status mlps_batch_workspace_size(const mlps_config* cfg, int32_t K, const mlps_batch_item* items,
                                      int32_t n_items, size_t* saved_bytes, size_t* scratch_bytes);

/* Forward render of a batch; arguments as mlps_render_forward with the batch image layout. */
mlps_status mlps_render_batch_forward(const mlps_config* cfg, const mlps_scene* scene,
                                      const mlps_batch_item* items, int32_t n_items, float* rgb,
                                      float* trans, float* feat, void* saved, size_t saved_bytes,
                                      void* scratch, size_t scratch_bytes, void* stream);

/* Backward of a batch (same items and `saved` as the forward call); as mlps_render_backward. */
mlps_status mlps_render_batch_backward(const mlps_config* cfg, const mlps_scene* scene,
                                       const mlps_batch_item* items, int32_t n_items, const float* d_rgb,
                                       const float* d_trans, const float* d_feat, const void* saved,
                                       size_t saved_bytes, float* d_weights, float* d_centers,
                                       float* d_scales, float* d_quats, void* scratch,
                                       size_t scratch_bytes, void* stream);

/* Autotuner (no counterpart in the paper): picks `tile` (16 or 8) and `mlp_groups` (samples per
 * CTA of the forward tensor-core MLP: 2 to 6 chunks of 128 rows, width-64 models without a
 * feature head; other shapes keep their default) for this batch by running every candidate
 * `reps` times (after one warm-up run) on the caller's arguments, as mlps_render_batch_forward
 * (+ mlps_render_batch_backward with dL/drgb = d_rgb when do_backward), timed with CUDA events
 * on `stream`. Candidates whose workspace exceeds saved_bytes / scratch_bytes are skipped.
 * Writes *tuned = *cfg with the fastest tile and mlp_groups and *best_ms (mean ms per run;
 * 0 when the decision came from the cache). Decisions are cached per batch shape (model, S,
 * precision, max hits, each item's primitive count and resolution, do_backward) for the life of
 * the process. Optional outputs (host, capacity 16, may be NULL): the candidates' tile, groups
 * and ms (negative = did not run). Synchronises `stream`; do not call it during stream capture.
 * The output and gradient buffers are overwritten. Returns MLPS_ERR_UNSUPPORTED if no
 * candidate ran. */
mlps_status mlps_autotune_batch(const mlps_config* cfg, const mlps_scene* scene, const mlps_batch_item* items,
                                int32_t n_items, int32_t do_backward, const float* d_rgb, float* rgb,
                                float* trans, float* feat, void* saved, size_t saved_bytes, void* scratch,
                                size_t scratch_bytes, float* d_weights, float* d_centers, float* d_scales,
                                float* d_quats, int32_t reps, mlps_config* tuned, float* best_ms,
                                int32_t* n_candidates, int32_t* cand_tile, int32_t* cand_groups,
                                float* cand_ms, void* stream);

/* Forget every cached autotuner decision. */
void mlps_autotune_clear(void);

/* ---------------------------------------------------------------------------------------- */
/* Batched rendering with a device-resident item table                                       */
/*
 * The batch renderer above, with the item table (primitive ranges and cameras, resolutions
 * included) read from DEVICE memory when the launches run, not from the host at call time.
 * A graph captured around these calls can therefore be replayed with new items (other
 * cameras, resolutions and primitive ranges within the caps) written into the same device
 * table between replays; nothing is baked in but n_items and the caps.
 *
 * caps (host struct): every item must satisfy width <= max_width, height <= max_height and
 * prim_count <= max_prim_count. The workspace is sized for n_items items at the caps
 * (mlps_batch_workspace_size_dev), and the image buffers for n_items * max_width * max_height
 * pixels. Items are concatenated at their actual sizes exactly as in the host-table calls
 * (item i's pixels start at P_i = sum_{j < i} width_j * height_j); pixels past the batch's
 * actual total are not written.
 *
 * dev_items: device array of n_items mlps_batch_item (1..MLPS_MAX_VIEWS), read by the first
 * kernel of each call (it may be written by the same stream just before). An item that breaks
 * the caps, names primitives outside [0, K) or has an invalid camera (the checks of
 * mlps_render_forward) is rendered as an empty view and sets the device status word to
 * MLPS_ERR_INVALID_ARGUMENT (mlps_read_status); the call itself returns MLPS_OK. Host-side
 * checks (null pointers, caps < 1, n_items out of range, workspace sizes) return their status
 * immediately. The backward call must use the same dev_items contents and saved region as the
 * forward call. */
typedef struct {
  int32_t max_width, max_height;  /* largest item resolution */
  int32_t max_prim_count;         /* largest item primitive range */
} mlps_batch_caps;

/* Workspace of a device-table batch of n_items items at the caps. */
mlps_status mlps_batch_workspace_size_dev(const mlps_config* cfg, int32_t K, int32_t n_items,
                                          const mlps_batch_caps* caps, size_t* saved_bytes,
                                          size_t* scratch_bytes);

/* Forward render of a device-table batch; other arguments as mlps_render_batch_forward. */
mlps_status mlps_render_batch_forward_dev(const mlps_config* cfg, const mlps_scene* scene,
                                          const mlps_batch_item* dev_items, int32_t n_items,
                                          const mlps_batch_caps* caps, float* rgb, float* trans,
                                          float* feat, void* saved, size_t saved_bytes, void* scratch,
                                          size_t scratch_bytes, void* stream);

/* Backward of a device-table batch (same items, caps and `saved` as the forward call). */
mlps_status mlps_render_batch_backward_dev(const mlps_config* cfg, const mlps_scene* scene,
                                           const mlps_batch_item* dev_items, int32_t n_items,
                                           const mlps_batch_caps* caps, const float* d_rgb,
                                           const float* d_trans, const float* d_feat, const void* saved,
                                           size_t saved_bytes, float* d_weights, float* d_centers,
                                           float* d_scales, float* d_quats, void* scratch,
                                           size_t scratch_bytes, void* stream);

/* Inspection of the last backward pass: *chunks = the MLP chunks of the forward pass (<= ipc
 * intervals of one primitive each), *live = those the backward pass walked (the chunks holding
 * an interval with a nonzero gradient: intervals behind a ray's early-termination point, and
 * rays with zero dL/dC, have none). Synchronises `stream`. */
mlps_status mlps_backward_chunk_counts(const void* saved, const void* scratch, int64_t* chunks,
                                       int64_t* live, void* stream);

/* Inspection of the last forward pass with depth waves (early_stop_wave > 0): *intervals = its
 * hit intervals, *evaluated = those the MLP evaluated over both waves (0 without waves, where
 * every interval is evaluated). Synchronises `stream`. */
mlps_status mlps_forward_wave_counts(const void* saved, const void* scratch, int64_t* intervals,
                                     int64_t* evaluated, void* stream);

/* Synchronise `stream`, return the device status word of a `saved` or `scratch` region
 * written by the calls above (MLPS_OK if none), and clear it. */
mlps_status mlps_read_status(const void* region, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Inspection of a forward pass (tests and tools)                                             */

/* Total hit records written by the forward pass in `saved` (host int64 out). Synchronises. */
mlps_status mlps_saved_hit_count(const void* saved, int64_t* n_hits, void* stream);

/* Dense copy of the per-ray sorted hit lists held in `saved`: for every ray r (global index
 * v*H*W + y*W + x), count[r] and, for j < min(count, max_out), prim[r*max_out + j],
 * t0/t1 (world units, near-clipped) and tmid (Eq. 2 before its max(0, .)). Device outputs. */
mlps_status mlps_export_hits(const mlps_config* cfg, const mlps_camera* cams, int32_t n_views,
                             const void* saved, int32_t max_out, int32_t* count, int32_t* prim,
                             float* t0, float* t1, float* tmid, void* stream);

/* Per-tile candidate lists of the last forward pass held in `scratch` (valid until the
 * scratch region is reused): count[v*n_tiles + t] and list[(v*n_tiles + t)*K + j], tiles in
 * row-major order of ceil(H/tile) x ceil(W/tile). Device outputs. */
mlps_status mlps_export_tiles(const mlps_config* cfg, int32_t K, const mlps_camera* cams,
                              int32_t n_views, const void* scratch, int32_t* count,
                              int32_t* list, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Optional host-side stage profiler (not thread-safe; off by default)                        */

/* Number of kernels this library has launched since the last reset (all entry points);
 * reset != 0 zeroes the counter after reading. */
int64_t mlps_kernel_launches(int32_t reset);

/* Self-test of the bounded waits (no counterpart in the paper). Every wait of the persistent
 * tensor-core kernels gives up after a wall-time limit and ends its kernel with MLPS_ERR_TIMEOUT
 * in the status word instead of hanging. This call runs that wait on a barrier nothing arrives
 * at, for limit_us microseconds (1 .. 1e6), and writes its outcome to the status word of
 * `scratch` (>= 256 bytes, 256-byte aligned): mlps_read_status(scratch) then returns
 * MLPS_ERR_TIMEOUT. Nothing faults; the device stays usable. */
mlps_status mlps_selftest_bounded_wait(int32_t limit_us, void* scratch, size_t scratch_bytes, void* stream);

/* Enable (1) or disable (0). When enabled every call records CUDA events around each kernel
 * stage on its stream. */
void mlps_profiler_enable(int32_t on);

/* Synchronise on the recorded events and return the number of stages; for i < max fill
 * names[i] (static strings) and ms[i] (summed over calls since the last reset) and
 * counts[i]. reset != 0 clears the table afterwards. */
int32_t mlps_profiler_read(const char** names, float* ms, int32_t* counts, int32_t max,
                           int32_t reset);

/* ---------------------------------------------------------------------------------------- */
/* Training objective and optimizer (Sec. 3.5, App. A.4)                                      */

/* A training step's images: rgb and its target [V, H, W, 3], optional feature rows
 * [V, H, W, feat_dim] and their targets. Only the selected `tile` x `tile` screen tiles enter
 * the loss (the paper's tile mini-batching): tile_mask [V, ceil(H/tile), ceil(W/tile)] bytes on
 * the device, nonzero = selected, NULL = every pixel. */
typedef struct {
  int32_t n_views, height, width;
  int32_t tile;                 /* edge of the mask tiles, >= 1 */
  const uint8_t* tile_mask;     /* device, or NULL */
  float lambda_ssim;            /* lambda of the photometric loss (Eq. 7), in [0, 1] */
  int32_t feat_dim;             /* feature channels (0: no feature loss) */
} mlps_loss_desc;

/* Workspace bytes of mlps_loss (9 floats per pixel and the loss sums); 0 for an invalid desc. */
size_t mlps_loss_workspace_size(const mlps_loss_desc* desc);

/* The loss of Eq. 7 (plus Eq. 8 when feat_dim > 0) over the N selected pixels:
 *   L = (1 - lambda) L1 + lambda (1 - SSIM) + L_f,
 *   L1 = sum_p sum_c |C - C*| / (3 N), SSIM = mean of the per-pixel, per-channel SSIM map (11 x 11
 *   Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2), L_f = sum |F - F*| / (F N),
 * and its gradient: OVERWRITES d_rgb [V, H, W, 3] (and d_feat when feat_dim > 0; may be NULL
 * otherwise), and loss_out (device, 5 floats) = {L, L1, SSIM, N, L_f}. `workspace` is
 * 256-byte aligned device memory of mlps_loss_workspace_size bytes. */
mlps_status mlps_loss(const mlps_loss_desc* desc, const float* rgb, const float* rgb_target,
                      const float* feat, const float* feat_target, float* d_rgb, float* d_feat,
                      float* loss_out, void* workspace, size_t workspace_bytes, void* stream);

/* One parameter group of an Adam step; all pointers are device memory of n floats. kind 0:
 * plain; kind 1: log-parameter (param holds log x, grad is dL/dx, aux holds x: the step uses
 * dL/dlog x = dL/dx * x and rewrites aux = exp(param)). m and v start at zero. */
typedef struct {
  float* param;
  const float* grad;
  float* m;
  float* v;
  float* aux;
  int64_t n;
  float lr;
  int32_t kind;
} mlps_adam_group;

#define MLPS_MAX_ADAM_GROUPS 8

/* One Adam step (Kingma and Ba) over n_groups <= MLPS_MAX_ADAM_GROUPS groups (HOST array),
 * step = 1, 2, ... (bias corrections 1 - beta^step). One kernel launch. */
mlps_status mlps_adam_step(const mlps_adam_group* groups, int32_t n_groups, float beta1, float beta2,
                           float eps, int32_t step, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLPS_H */
