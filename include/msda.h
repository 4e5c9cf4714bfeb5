/*
 * msda.h - C-ABI of the GB300 (sm_103a) Multi-Scale Deformable Aggregation
 * library (libmsda_gb300.so).
 *
 * The operator (arXiv 2601.10819, Sec. 3.1, Sec. 3.2 and Sec. 5.3): every
 * anchor's P keypoints are projected into each of Ncam cameras; each
 * projected location is bilinearly sampled from that camera's Nscale
 * feature maps, with zero padding outside a map; the samples are multiplied
 * by per-group attention weights and summed into one C-channel feature per
 * anchor.  For channel c in group g = c / (C/G):
 *
 *   out[b,a,c] = sum_{p,k,s} w[b,a,p,k,s,g] * S_{b,k,s}(loc[b,a,p,k])[c]
 *
 * S is the bilinear sample at x = u*W - 0.5, y = v*H - 0.5 of the map of
 * camera k at scale s (pixel (i, j) is centred at ((j+0.5)/W, (i+0.5)/H));
 * a corner outside [0,H) x [0,W) reads 0 and a point with x <= -1,
 * x >= W, y <= -1, y >= H, or a NaN coordinate, contributes nothing.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All tensor pointers are DEVICE pointers owned by the caller, row-major
 *   and densely packed.  The library never allocates, frees or synchronises
 *   inside msda_forward / msda_backward / msda_forward_batched; scratch
 *   memory is passed in by the caller.
 * - Layouts:
 *     feat               [B, sum_hw, C]           (feat_dtype)
 *     spatial_shape      [Ncam, Nscale, 2] int32  (H, W) of each map
 *     scale_start_index  [Ncam, Nscale]    int32  first row of each map
 *                        inside one batch element's sum_hw rows; the row of
 *                        pixel (i, j) is b*sum_hw + start[k,s] + i*W + j
 *     sampling_location  [B, A, P, Ncam, 2] float32, normalised (u, v)
 *     weights            [B, A, P, Ncam, Nscale, G] (weights_dtype)
 *     out                [B, A, C]              (out_dtype), overwritten
 * - Arithmetic: features and weights are widened to FP32 and every product
 *   and sum is FP32; a BF16/FP16 output is rounded once, to nearest even.
 * - Alignment: every tensor pointer must be 16-byte aligned, and
 *   (C/G) * sizeof(feat element) must be a multiple of 16 bytes.
 * - Channel split: a channel row is read by a team of lanes, each lane
 *   taking n 16-byte vectors (VEC = 16 / sizeof(feat element) channels per
 *   vector).  Some n in {1, 2, 4} must give C % (VEC*n) == 0,
 *   (C/G) % (VEC*n) == 0 and a team size C / (VEC*n) that is a power of two
 *   no larger than 32; otherwise the call returns MSDA_ERR_UNSUPPORTED.
 *   For example C=256 works for every G that divides it into groups of at
 *   least 16 bytes, while C=96 with G=2 (FP32), C=48 with G=3 (BF16) and FP32
 *   rows wider than 512 channels are rejected.
 * - Every map must satisfy H >= 1, W >= 1 and start + H*W <= sum_hw.  The
 *   shape tables live on the device, so they are checked by the kernels: a
 *   bad map is skipped (it contributes nothing) and the device status word
 *   is set to MSDA_ERR_OUT_OF_RANGE; read it with msda_get_device_status().
 * - Errors are returned, never printed; no entry point aborts.
 *   msda_last_error() gives a message for the last failing call of the
 *   calling thread.
 * - Streams: `stream` is a cudaStream_t (NULL = legacy default stream); all
 *   work is ordered on it.  The calls allocate nothing and do not
 *   synchronise, so they may be captured in a CUDA graph, except that the
 *   first call on a device looks up the device status word and reads
 *   device attributes, which should happen before any capture.  The
 *   deterministic msda_backward runs its cell-binned kernels on a second
 *   stream of the library's (one per device, made by the first such call
 *   outside a capture), forked from `stream` and joined back to it with
 *   events inside the call, so everything enqueued on `stream` afterwards
 *   sees the whole result and a capture of `stream` takes those kernels in
 *   as a parallel branch.
 */
#ifndef MSDA_GB300_H
#define MSDA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                      /* cudaStream_t == struct CUstream_st* */
typedef struct CUstream_st* msda_stream_t;

typedef enum {
    MSDA_OK = 0,
    MSDA_ERR_INVALID_ARG = 1,   /* null pointer, negative or inconsistent size  */
    MSDA_ERR_UNSUPPORTED = 2,   /* alignment / channel split this build rejects */
    MSDA_ERR_CUDA = 3,          /* a CUDA call or kernel launch failed          */
    MSDA_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up           */
    MSDA_ERR_OUT_OF_RANGE = 5,  /* a shape-table entry points outside feat      */
    MSDA_ERR_WORKSPACE = 6      /* workspace missing or smaller than required   */
} msda_status;

typedef enum { MSDA_F32 = 0, MSDA_BF16 = 1, MSDA_F16 = 2 } msda_dtype;

/* Launch mapping.  A NULL tuning pointer, or a zero field, picks the
 * built-in default for that field.  For a fixed tuning every entry point
 * except the atomic backward is bitwise reproducible run to run; two
 * different tunings may differ in the last bits, because the warps_per_block
 * split decides the order of the FP32 sums. */
typedef struct {
    int warps_per_block;   /* 1..8: warps per block (teams of lanes per block)   */
    int blocks_per_sm;     /* persistent batched kernel: resident blocks per SM  */
    int variant;           /* 0 = default; msda_forward: 1 = anchor-per-block
                              kernel even with a workspace, 3 = FP16
                              features and weights accumulated in half2 (the
                              paper's plugin arithmetic, Sec. 5.3; less
                              accurate), 4 = the single-stage anchor kernel
                              (every lane of a team locates its point-scales
                              itself; by default a block locates each
                              point-scale once into a shared list; also for
                              msda_forward_train and _oae);
                              msda_backward (deterministic):
                              2 = staged camera-group form,
                              5 = corner-slot form even where the
                              cell-binned form applies                       */
    int vectors_per_lane;  /* 16-byte feature vectors per lane and corner row
                              (1, 2 or 4): more work per lane, fewer lanes
                              per point; 0 = built-in default (2 when that
                              split is valid), else the smallest valid split */
    int flags;             /* MSDA_FLAG_* bits                                */
    int reserved[3];
} msda_tuning;

/* tuning->flags: the caller has already zeroed grad_feat (for example on a
 * side stream while the forward ran); the atomic backward then skips its
 * own clearing of grad_feat.  Ignored by the deterministic modes, which
 * write every row. */
#define MSDA_FLAG_GRAD_FEAT_ZEROED 1

/* ------------------------------------------------------------------------
 * msda_forward - the operator above (Sec. 3.2 multi-scale multi-view
 * feature extraction at projected keypoints; Sec. 5.3 MSDA).
 *   feat_dtype, weights_dtype: MSDA_F32, MSDA_BF16 or MSDA_F16.
 *   out_dtype: MSDA_F32 (default use), MSDA_BF16 or MSDA_F16.
 *   B, sum_hw, Ncam, Nscale, A, P >= 0 (zero-size problems are no-ops,
 *   except that out is still written when B*A > 0); C, G >= 1; C % G == 0;
 *   Nscale <= 16.
 *   workspace: NULL, or device memory of at least
 *     msda_forward_workspace_size(...) bytes (16-byte aligned).  With a
 *     workspace (and Nscale <= 4, (C/G)*sizeof(feat) in {16, 32, 64, 128})
 *     the staged camera-group kernels run: each (camera, group) stages its
 *     coarse maps in shared memory with TMA and writes per-camera partial
 *     sums, which are then added in camera order.  Without one, one block
 *     per anchor gathers every corner from L2/HBM.
 * Deterministic: the same inputs and launch choice give bitwise-identical
 * outputs (the two kernels differ in the last bits: different sum order).
 * ------------------------------------------------------------------------ */
size_t msda_forward_workspace_size(int B, int sum_hw, int C, int Ncam, int Nscale,
                                   int A, int P, int G);

msda_status msda_forward(const void* feat, msda_dtype feat_dtype,
                         const int32_t* spatial_shape, const int32_t* scale_start_index,
                         const float* sampling_location,
                         const void* weights, msda_dtype weights_dtype,
                         void* out, msda_dtype out_dtype,
                         int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                         void* workspace, size_t workspace_bytes,
                         const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * Forward of a training step: msda_forward (anchor-per-block kernel; the
 * tuning fields as for msda_forward) that also sets grad_feat
 * [B, sum_hw, C] (float32, 16-byte aligned; C a multiple of 4) to zero, for
 * an atomic msda_backward called afterwards with MSDA_FLAG_GRAD_FEAT_ZEROED.
 * The forward's blocks store the zeros in small pieces alongside their
 * gathers, on HBM write bandwidth the forward leaves unused, instead of a
 * separate memset before the backward.  With no anchors or no points the
 * clearing is a memset on `stream`.
 * ------------------------------------------------------------------------ */
msda_status msda_forward_train(const void* feat, msda_dtype feat_dtype,
                               const int32_t* spatial_shape, const int32_t* scale_start_index,
                               const float* sampling_location,
                               const void* weights, msda_dtype weights_dtype,
                               void* out, msda_dtype out_dtype, float* grad_feat,
                               int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                               const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * msda_forward_oae - the operator followed by the occlusion-aware
 * visibility-weighted fusion over cameras (Sec. 3.2, Eq. 2), fused:
 *   out[b,a,:] = sum_k vis[b,a,k] * g_k / sum_k vis[b,a,k]
 * where g_k is the operator above restricted to camera k.  Implemented by
 * scaling every weight of camera k by vis[b,a,k] / sum_j vis[b,a,j] inside
 * the anchor-per-block forward (cameras with zero visibility are skipped).
 * An anchor whose visibilities sum to 0 gets out = 0.
 *   visibility: [B, A, Ncam] float32, device, 16-byte aligned.
 * Other arguments and errors as msda_forward (no workspace).
 * ------------------------------------------------------------------------ */
msda_status msda_forward_oae(const void* feat, msda_dtype feat_dtype,
                             const int32_t* spatial_shape, const int32_t* scale_start_index,
                             const float* sampling_location,
                             const void* weights, msda_dtype weights_dtype,
                             const float* visibility,
                             void* out, msda_dtype out_dtype,
                             int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                             const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * msda_keypoints - the sampling locations the operator consumes (Sec. 3.1
 * and 3.2: anchor keypoints, motion compensation with the estimated
 * velocity, projection into every camera):
 *   q = R(yaw) (offset * (w, l, h)) + centre + velocity * dt
 *   (hx, hy, hz) = proj_k (q, 1)
 *   sampling_location[b,a,p,k] = (hx/hz/width_k, hy/hz/height_k),
 *                                or (-2, -2) when hz <= 1e-5.
 *   anchors [B, A, 11] = (x, y, z, w, l, h, sin yaw, cos yaw, vx, vy, vz)
 *   offsets [B, A, P, 3] keypoints in box units; dt [B];
 *   proj [B, Ncam, 3, 4] world -> homogeneous pixels; img_wh [Ncam, 2];
 *   sampling_location [B, A, P, Ncam, 2] written.  All float32, device,
 *   16-byte aligned.
 * ------------------------------------------------------------------------ */
msda_status msda_keypoints(const float* anchors, const float* offsets, const float* dt,
                           const float* proj, const float* img_wh, float* sampling_location,
                           int B, int A, int P, int Ncam, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * msda_backward - gradients of msda_forward for the upstream gradient
 * grad_out [B, A, C] (float32):
 *   grad_feat    [B, sum_hw, C]             float32, overwritten
 *   grad_loc     [B, A, P, Ncam, 2]          float32, overwritten
 *   grad_weights [B, A, P, Ncam, Nscale, G]  float32, overwritten
 * For each in-bound corner with bilinear weight omega:
 *   grad_feat[row, c] += w_g * omega * grad_out[c];
 *   grad_weights = sum over the group's channels of grad_out * S;
 *   grad_loc = (W * dS/dx, H * dS/dy) contracted with w_g * grad_out and
 *   summed over scales, using the bilinear patch selected by floor() at a
 *   grid line.
 * The paper's operator is forward-only (an inference plugin, Sec. 5.3);
 * this is its exact adjoint, for training.
 *
 *   deterministic = 0: the feature gradient is scattered with FP32 vector
 *     atomics (summation order varies run to run, values agree to rounding).
 *     With a workspace (256 bytes) the items are handed out from one
 *     counter strictly in camera order, which keeps the rows being
 *     accumulated in L2; with workspace = NULL a static stride is used.
 *   deterministic = 1: no floating-point atomics; bitwise reproducible.  By
 *     default (cell-binned form) each map's in-view point-scales are binned
 *     by bilinear cell in point order, and every feature row is summed over
 *     the bins of its four neighbouring cells in a fixed order, with
 *     grad_out of one channel group staged in shared memory.  It applies
 *     when the valid maps do not overlap, A*P <= 65535, C/G is 4 times a
 *     power of two up to 128, Ncam*Nscale <= 4096, A*(C/G)*4 bytes fit in a
 *     block's shared memory and every map's (H+1)*(W+1) cells fit the
 *     binning block; the map conditions are checked on the device.
 *     Otherwise (or with tuning->variant = 5) the corner-slot form runs:
 *     the corner contributions are grouped by feature row (a counting sort
 *     whose integer counters place them), each row's group is sorted by
 *     slot id, and each row is reduced in that order.  With
 *     tuning->variant = 2, when the staged kernels apply (Nscale <= 4, C/G a
 *     power of two in 4..128, at most 40960 bilinear cells per map, maps
 *     that do not overlap, A*(C/G)*4 bytes of grad_out per group fitting in
 *     shared memory): dw and dloc come from the camera-group gather, and the
 *     feature gradient from a stable per-map sort of the points by bilinear
 *     cell followed by one fixed-order gather per feature row; overlapping
 *     maps then raise MSDA_ERR_OUT_OF_RANGE in the status word.
 * grad_loc and grad_weights are computed without atomics in both modes.
 * workspace: device memory of at least msda_backward_workspace_size(...)
 * bytes, 16-byte aligned (may be NULL when that size is 0).
 * ------------------------------------------------------------------------ */
size_t msda_backward_workspace_size(int B, int sum_hw, int C, int Ncam, int Nscale,
                                    int A, int P, int G, int deterministic);

msda_status msda_backward(const void* feat, msda_dtype feat_dtype,
                          const int32_t* spatial_shape, const int32_t* scale_start_index,
                          const float* sampling_location,
                          const void* weights, msda_dtype weights_dtype,
                          const float* grad_out,
                          float* grad_feat, float* grad_loc, float* grad_weights,
                          int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                          int deterministic, void* workspace, size_t workspace_bytes,
                          const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched serving: many independent scenes (B = 1 each) with uneven camera
 * counts, map sizes and anchor counts, in ONE persistent launch (the
 * paper's many-camera-stream setting, Sec. 5.3 and App. C).  Scene i has
 * its own tensors, laid out as for msda_forward with B = 1.  All scenes
 * share C, G, P, Nscale and the dtypes.
 * ------------------------------------------------------------------------ */
typedef struct {
    const void* feat;                  /* [sum_hw, C]                        */
    const int32_t* spatial_shape;      /* [Ncam, Nscale, 2] (device)         */
    const int32_t* scale_start_index;  /* [Ncam, Nscale]    (device)         */
    const float* sampling_location;    /* [A, P, Ncam, 2]                    */
    const void* weights;               /* [A, P, Ncam, Nscale, G]            */
    void* out;                         /* [A, C], overwritten                */
    int32_t sum_hw;
    int32_t Ncam;
    int32_t A;
    int32_t unit_begin;                /* sum of A over the scenes before it */
} msda_scene;

/* Scratch needed by msda_forward_batched for num_scenes scenes. */
size_t msda_forward_batched_workspace_size(int num_scenes);

/* scenes: DEVICE array of num_scenes descriptors (unit_begin filled in by
 * the caller as the running sum of A).  total_anchors = sum of A.
 * max_ncam >= every scene's Ncam.  scene_done_ns (optional, device,
 * num_scenes + 1 entries): entry 0 receives the %globaltimer value when the
 * launch starts, entry i+1 the value when scene i's last anchor finished.
 * The workspace is re-initialised by every call (one cudaMemsetAsync), so a
 * captured graph can be replayed. */
msda_status msda_forward_batched(const msda_scene* scenes, int num_scenes, int total_anchors,
                                 int max_ncam, int Nscale, int C, int P, int G,
                                 msda_dtype feat_dtype, msda_dtype weights_dtype,
                                 msda_dtype out_dtype,
                                 void* workspace, size_t workspace_bytes,
                                 uint64_t* scene_done_ns,
                                 const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * msda_forward_batched_noalloc - msda_forward_batched without a workspace.
 * The paper has no counterpart; this exists for callers that cannot
 * allocate device memory where they launch work (a plugin's enqueue inside
 * an inference engine, a real-time loop with a fixed memory budget, a C host
 * program without a device allocator).  Same arguments and results as
 * msda_forward_batched minus the workspace: the scratch is a device array
 * built into the library, sized for at most
 * msda_forward_batched_noalloc_max_scenes() scenes (1024); more scenes are
 * rejected with MSDA_ERR_INVALID_ARG.  The call allocates nothing (no
 * cudaMalloc/cudaFree, no allocating library routine).  Every GPU that
 * loads the library keeps the array until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - All calls share the array and each call clears it first, so calls
 *     that overlap on the GPU (different streams, no ordering between them)
 *     race and give wrong results: order them on one stream or with events.
 * ------------------------------------------------------------------------ */
int msda_forward_batched_noalloc_max_scenes(void);

msda_status msda_forward_batched_noalloc(const msda_scene* scenes, int num_scenes, int total_anchors,
                                         int max_ncam, int Nscale, int C, int P, int G,
                                         msda_dtype feat_dtype, msda_dtype weights_dtype,
                                         msda_dtype out_dtype, uint64_t* scene_done_ns,
                                         const msda_tuning* tuning, msda_stream_t stream);

/* ------------------------------------------------------------------------
 * Status and diagnostics
 * ------------------------------------------------------------------------ */
/* Testing aid (no counterpart in the paper): the staged kernels (the
 * staged forward with a workspace, the staged and the cell-binned
 * deterministic backward) wait on an mbarrier for each set of bulk copies
 * they issue, polling at most a fixed number of times (about 2^26, seconds)
 * before they give up, set MSDA_ERR_TIMEOUT in the device status word and
 * skip the work that needed the copies.  This sets the poll limit of that
 * first wait on the current device: polls > 0 polls that many times,
 * polls = 0 gives up at once (so the next staged call reports
 * MSDA_ERR_TIMEOUT and computes wrong results), polls < 0 restores the
 * default.  After a give-up a second wait with the full limit lets the copies
 * in flight land before the block moves on.  Synchronous (a copy to a
 * device variable); not for use during stream capture. */
msda_status msda_debug_set_wait_limit(long long polls);

/* Synchronises `stream`, returns the device status word of the current
 * device (MSDA_OK if no kernel reported a problem since the last read) and
 * clears it. */
msda_status msda_get_device_status(msda_stream_t stream);

/* Message for the last failing call on this thread ("" if none). */
const char* msda_last_error(void);

/* Library version string. */
const char* msda_version(void);

/* ------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): streams `bytes` bytes of
 * `buf` (device, 16-byte aligned, bytes a multiple of 16) `reps` times with
 * 128-bit loads, in `blocks` blocks of 512 threads, and writes one word per
 * block to `sink` (device, >= blocks words) so the loads are not removed.
 * A buffer smaller than L2 measures L2 read bandwidth, a larger one HBM.
 * rows > 0 switches to random row gathers: each warp reads `rows`
 * pseudo-random 512-byte rows of buf per rep (the access pattern of the
 * operator's corner loads).
 * ------------------------------------------------------------------------ */
msda_status msda_probe_read(const void* buf, size_t bytes, int reps, int blocks, int rows,
                            uint32_t* sink, msda_stream_t stream);

/* Measurement aid: FP32 reduction throughput.  In `blocks` blocks of 512
 * threads, every warp adds 1.0 to `rows` pseudo-random 1 KB rows of `buf`
 * (device FP32, 16-byte aligned, bytes a multiple of 1024; its contents are
 * changed) per rep with 16-byte vector reductions, the scatter pattern of the
 * atomic backward.  A buffer smaller than L2 measures the L2's reduction
 * throughput, which bounds that backward. */
msda_status msda_probe_reduce(float* buf, size_t bytes, int reps, int blocks, int rows, msda_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MSDA_GB300_H */
