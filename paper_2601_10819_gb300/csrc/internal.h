// Host-side declarations shared by the translation units of libmsda_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "msda.h"

namespace msda {

// Validated description of one single-scene problem.
struct Problem {
    const void* feat;
    msda_dtype feat_t;
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    msda_dtype w_t;
    int B, sum_hw, C, Ncam, Nscale, A, P, G;
    int Cg;  // channels per group
    int nv;  // 16-byte chunks per lane (1, 2 or 4)
    int rt;  // lanes per channel row (power of two, <= 32)
};

struct DeviceInfo {
    int device;
    int sm_count;
    int max_smem_optin;  // bytes of dynamic shared memory a block may opt into
    int* status;         // device address of the status word
};

// Per-device constants, looked up on the first call on each device.
msda_status device_info(DeviceInfo* out);

// Record a message for msda_last_error() and return `code`.
msda_status fail(msda_status code, const char* fmt, ...);

// Translate a CUDA error (after a launch) into a status.
msda_status check_launch(const char* what);

// Raise the dynamic shared-memory limit of `func` to `bytes` if needed.
msda_status ensure_smem(const void* func, size_t bytes, const DeviceInfo& dev);

// Lanes-per-row / chunks-per-lane split for C channels of `t`, or false.
bool pick_split(int C, int G, msda_dtype t, int* nv, int* rt);
// As pick_split, but take `pref` vectors per lane when that split is valid.
bool pick_split_pref(int C, int G, msda_dtype t, int pref, int* nv, int* rt);

int dtype_size(msda_dtype t);

// Kernel launchers (validated inputs).  launch_backward_loc_w's `scatter`:
// 0 = no feature gradient, 1 = clear grad_feat then scatter, 2 = scatter
// into a grad_feat the caller already cleared.
msda_status launch_forward(const Problem& p, void* out, msda_dtype out_t, int warps,
                           cudaStream_t stream, const float* vis = nullptr, bool half_acc = false,
                           float* clear = nullptr, bool units = false);
msda_status launch_backward_atomic(const Problem& p, const float* grad_out, float* grad_feat,
                                   float* grad_loc, float* grad_w, void* ws, size_t ws_bytes, int warps,
                                   bool zeroed, cudaStream_t stream);
msda_status launch_backward_loc_w(const Problem& p, const float* grad_out, float* grad_feat,
                                  float* grad_loc, float* grad_w, int warps, int scatter,
                                  cudaStream_t stream, unsigned long long* counter = nullptr);
// dloc and dw only, one block per anchor (the deterministic modes; grad_feat is not touched).
msda_status launch_backward_locw(const Problem& p, const float* grad_out, float* grad_loc, float* grad_w, int warps,
                                 cudaStream_t stream);
size_t backward_det_workspace(const Problem& p);
// allow_cells: take the cell-binned feature gradient (cb.cu) where it applies; false forces the corner-slot
// path of det.cu.
msda_status launch_backward_det(const Problem& p, const float* grad_out, float* grad_feat,
                                float* grad_loc, float* grad_w, void* ws, size_t ws_bytes,
                                int warps, bool allow_cells, cudaStream_t stream);
// The cell-binned deterministic feature gradient (cb.cu).  cb_shape_ok: the sizes allow it on any device;
// cb_device_ok: and on the current one.  Its plan area (cb_plan_bytes) opens the workspace; its other arrays
// start at body_base.
bool cb_shape_ok(const Problem& p);
bool cb_device_ok(const Problem& p, const DeviceInfo& dev);
size_t cb_plan_bytes(const Problem& p);
size_t cb_workspace(const Problem& p, size_t body_base);
msda_status launch_backward_cb(const Problem& p, const float* grad_out, float* grad_feat, void* ws,
                               size_t body_base, cudaStream_t stream);
// Poll limit of the first wait of each staging step of the staged kernels (cg.cu, cb.cu); see
// msda_debug_set_wait_limit.
msda_status cg_set_wait_limit(long long polls);
msda_status cb_set_wait_limit(long long polls);
size_t batched_workspace(int num_scenes);
msda_status launch_forward_batched(const msda_scene* scenes, int num_scenes, int total_anchors,
                                   int max_ncam, int Nscale, int C, int P, int G, msda_dtype ft,
                                   msda_dtype wt, msda_dtype ot, void* ws, size_t ws_bytes,
                                   uint64_t* done_ns, int warps, int blocks_per_sm, int vec,
                                   cudaStream_t stream);
int batched_noalloc_max_scenes();
msda_status launch_forward_batched_noalloc(const msda_scene* scenes, int num_scenes, int total_anchors,
                                           int max_ncam, int Nscale, int C, int P, int G, msda_dtype ft,
                                           msda_dtype wt, msda_dtype ot, uint64_t* done_ns, int warps,
                                           int blocks_per_sm, int vec, cudaStream_t stream);
bool cg_supported(const Problem& p);
size_t cg_forward_workspace(const Problem& p);
size_t cg_backward_workspace(const Problem& p);
msda_status launch_forward_cg(const Problem& p, void* out, msda_dtype out_t, void* ws, size_t ws_bytes,
                              cudaStream_t stream);
msda_status launch_backward_cg(const Problem& p, const float* grad_out, float* grad_feat, float* grad_loc,
                               float* grad_w, void* ws, size_t ws_bytes, cudaStream_t stream);
msda_status launch_keypoints(const float* anchors, const float* offsets, const float* dt, const float* proj,
                             const float* img_wh, float* loc, int B, int A, int P, int Ncam, cudaStream_t stream);
msda_status launch_probe_reduce(float* buf, size_t bytes, int reps, int blocks, int rows, cudaStream_t stream);
msda_status launch_probe(const void* buf, size_t bytes, int reps, int blocks, int rows,
                         uint32_t* sink, cudaStream_t stream);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace msda
