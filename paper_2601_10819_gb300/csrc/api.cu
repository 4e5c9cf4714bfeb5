// C-ABI entry points of libmsda_gb300: argument validation, per-device
// constants, the device status word and error messages.  Every compute step
// is a kernel of fwd.cu, bwd.cu, det.cu, cg.cu, prologue.cu or probe.cu;
// nothing here touches tensor data.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace msda {

__device__ int g_status_word;  // first error code raised by any kernel

static thread_local char t_err[512];

msda_status fail(msda_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

msda_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MSDA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return MSDA_OK;
}

msda_status device_info(DeviceInfo* out) {
    static std::mutex mu;
    static DeviceInfo cache[128];
    static bool valid[128];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MSDA_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(MSDA_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!valid[dev]) {
        DeviceInfo d;
        d.device = dev;
        if ((e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
            (e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.status), g_status_word)) != cudaSuccess)
            return fail(MSDA_ERR_CUDA, "device set-up: %s", cudaGetErrorString(e));
        cache[dev] = d;
        valid[dev] = true;
    }
    *out = cache[dev];
    return MSDA_OK;
}

msda_status ensure_smem(const void* func, size_t bytes, const DeviceInfo& dev) {
    if (bytes > (size_t)dev.max_smem_optin)
        return fail(MSDA_ERR_UNSUPPORTED, "needs %zu bytes of shared memory per block (limit %d)", bytes,
                    dev.max_smem_optin);
    if (bytes <= 48 * 1024) return MSDA_OK;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return fail(MSDA_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return MSDA_OK;
}

int dtype_size(msda_dtype t) {
    switch (t) {
        case MSDA_F32: return 4;
        case MSDA_BF16: return 2;
        case MSDA_F16: return 2;
    }
    return 0;
}

static bool split_ok(int C, int G, msda_dtype t, int n, int* rt) {
    const int sz = dtype_size(t);
    if (sz == 0 || G <= 0 || C <= 0 || C % G || (n != 1 && n != 2 && n != 4)) return false;
    const int cpl = (16 / sz) * n;
    const int cg = C / G;
    if (C % cpl || cg % cpl) return false;
    const int r = C / cpl;
    if (r > 32 || (r & (r - 1))) return false;
    *rt = r;
    return true;
}

// Prefer `want` 16-byte vectors per lane (the tuning's, else `dflt`) when
// that split is valid; otherwise keep the smallest valid one.
static void prefer_split(const msda_tuning* t, Problem* p, int dflt) {
    const int want = (t && t->vectors_per_lane > 0) ? t->vectors_per_lane : dflt;
    int rt;
    if (want > 0 && split_ok(p->C, p->G, p->feat_t, want, &rt)) {
        p->nv = want;
        p->rt = rt;
    }
}

bool pick_split(int C, int G, msda_dtype t, int* nv, int* rt) {
    const int sz = dtype_size(t);
    if (sz == 0 || G <= 0 || C <= 0 || C % G) return false;
    const int vec = 16 / sz;
    const int cg = C / G;
    for (int n = 1; n <= 4; n *= 2) {
        const int cpl = vec * n;
        if (C % cpl || cg % cpl) continue;
        const int r = C / cpl;
        if (r > 32 || (r & (r - 1))) continue;
        *nv = n;
        *rt = r;
        return true;
    }
    return false;
}

bool pick_split_pref(int C, int G, msda_dtype t, int pref, int* nv, int* rt) {
    if (!pick_split(C, G, t, nv, rt)) return false;
    int r;
    if (pref > 0 && split_ok(C, G, t, pref, &r)) {
        *nv = pref;
        *rt = r;
    }
    return true;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int pick_warps(const msda_tuning* t, int dflt) {
    const int w = (t && t->warps_per_block > 0) ? t->warps_per_block : dflt;
    return w > 8 ? 8 : w;  // the kernels are built for at most 256 threads per block
}

// Shared validation of the single-scene entry points.
static msda_status validate(const char* fn, const void* feat, msda_dtype ft, const int32_t* shape,
                            const int32_t* start, const float* loc, const void* w, msda_dtype wt,
                            int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                            Problem* p) {
    if (B < 0 || sum_hw < 0 || Ncam < 0 || Nscale < 0 || A < 0 || P < 0)
        return fail(MSDA_ERR_INVALID_ARG, "%s: negative dimension", fn);
    if (C < 1 || G < 1 || C % G != 0)
        return fail(MSDA_ERR_INVALID_ARG, "%s: need C >= 1, G >= 1 and C %% G == 0 (C=%d G=%d)", fn, C, G);
    if (Nscale > kMaxScales) return fail(MSDA_ERR_UNSUPPORTED, "%s: Nscale %d > %d", fn, Nscale, kMaxScales);
    if (dtype_size(ft) == 0 || dtype_size(wt) == 0) return fail(MSDA_ERR_INVALID_ARG, "%s: unknown dtype", fn);
    if ((C / G) * dtype_size(ft) % 16 != 0)
        return fail(MSDA_ERR_UNSUPPORTED, "%s: (C/G)*sizeof(feat) = %d bytes is not a multiple of 16", fn,
                    (C / G) * dtype_size(ft));
    if (!pick_split(C, G, ft, &p->nv, &p->rt))
        return fail(MSDA_ERR_UNSUPPORTED, "%s: no lane split for C=%d G=%d", fn, C, G);
    const bool any_pts = (long long)B * A * P * Ncam > 0;
    if (((long long)B * sum_hw > 0 || any_pts) && !feat) return fail(MSDA_ERR_INVALID_ARG, "%s: feat is NULL", fn);
    if ((long long)Ncam * Nscale > 0 && (!shape || !start))
        return fail(MSDA_ERR_INVALID_ARG, "%s: spatial_shape/scale_start_index is NULL", fn);
    if (any_pts && (!loc || (Nscale > 0 && !w)))
        return fail(MSDA_ERR_INVALID_ARG, "%s: sampling_location/weights is NULL", fn);
    if (!aligned16(feat) || !aligned16(loc) || !aligned16(w) || !aligned16(shape) || !aligned16(start))
        return fail(MSDA_ERR_UNSUPPORTED, "%s: tensor pointers must be 16-byte aligned", fn);
    if ((long long)P * Ncam > (1ll << 24) || (long long)Ncam * Nscale > (1ll << 20))
        return fail(MSDA_ERR_UNSUPPORTED, "%s: P*Ncam or Ncam*Nscale too large", fn);
    p->feat = feat; p->feat_t = ft; p->shape = shape; p->start = start; p->loc = loc; p->w = w; p->w_t = wt;
    p->B = B; p->sum_hw = sum_hw; p->C = C; p->Ncam = Ncam; p->Nscale = Nscale; p->A = A; p->P = P; p->G = G;
    p->Cg = C / G;
    return MSDA_OK;
}

}  // namespace msda

using namespace msda;

extern "C" {

const char* msda_last_error(void) { return t_err; }

const char* msda_version(void) { return "msda_gb300 1.0 (sm_103a)"; }

size_t msda_forward_workspace_size(int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G) {
    if (B < 0 || sum_hw < 0 || C < 1 || Ncam < 0 || Nscale < 0 || A < 0 || P < 0 || G < 1) return 0;
    Problem p;
    p.B = B; p.sum_hw = sum_hw; p.C = C; p.Ncam = Ncam; p.Nscale = Nscale; p.A = A; p.P = P; p.G = G;
    return cg_forward_workspace(p);
}

msda_status msda_forward(const void* feat, msda_dtype feat_dtype, const int32_t* spatial_shape,
                         const int32_t* scale_start_index, const float* sampling_location,
                         const void* weights, msda_dtype weights_dtype, void* out, msda_dtype out_dtype,
                         int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                         void* workspace, size_t workspace_bytes,
                         const msda_tuning* tuning, msda_stream_t stream) {
    t_err[0] = 0;
    Problem p;
    msda_status st = validate("msda_forward", feat, feat_dtype, spatial_shape, scale_start_index,
                              sampling_location, weights, weights_dtype, B, sum_hw, C, Ncam, Nscale, A, P, G, &p);
    if (st != MSDA_OK) return st;
    if (dtype_size(out_dtype) == 0) return fail(MSDA_ERR_INVALID_ARG, "msda_forward: unknown out dtype");
    if ((long long)B * A > 0 && !out) return fail(MSDA_ERR_INVALID_ARG, "msda_forward: out is NULL");
    if (!aligned16(out)) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward: out must be 16-byte aligned");
    prefer_split(tuning, &p, 2);
    const bool half_acc = tuning && tuning->variant == 3;  // paper-faithful half2 accumulation
    const bool direct = tuning && (tuning->variant == 1 || tuning->variant == 4 || half_acc);  // anchor kernel
    if (workspace && !direct && cg_supported(p)) {
        if (!aligned16(workspace)) return fail(MSDA_ERR_WORKSPACE, "msda_forward: workspace must be 16-byte aligned");
        return launch_forward_cg(p, out, out_dtype, workspace, workspace_bytes, (cudaStream_t)stream);
    }
    const bool units = !(tuning && tuning->variant == 4);  // variant 4: the single-stage anchor kernel
    return launch_forward(p, out, out_dtype, pick_warps(tuning, 8), (cudaStream_t)stream, nullptr, half_acc, nullptr,
                          units);
}

msda_status msda_forward_train(const void* feat, msda_dtype feat_dtype, const int32_t* spatial_shape,
                               const int32_t* scale_start_index, const float* sampling_location,
                               const void* weights, msda_dtype weights_dtype, void* out, msda_dtype out_dtype,
                               float* grad_feat, int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P,
                               int G, const msda_tuning* tuning, msda_stream_t stream) {
    t_err[0] = 0;
    Problem p;
    msda_status st = validate("msda_forward_train", feat, feat_dtype, spatial_shape, scale_start_index,
                              sampling_location, weights, weights_dtype, B, sum_hw, C, Ncam, Nscale, A, P, G, &p);
    if (st != MSDA_OK) return st;
    if (dtype_size(out_dtype) == 0) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_train: unknown out dtype");
    if ((long long)B * A > 0 && !out) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_train: out is NULL");
    if ((long long)B * sum_hw > 0 && !grad_feat)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_train: grad_feat is NULL");
    if (!aligned16(out) || !aligned16(grad_feat))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_train: out and grad_feat must be 16-byte aligned");
    if (C % 4 != 0) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_train: C must be a multiple of 4");
    prefer_split(tuning, &p, 2);
    const bool half_acc = tuning && tuning->variant == 3;
    const bool units = !(tuning && tuning->variant == 4);
    return launch_forward(p, out, out_dtype, pick_warps(tuning, 8), (cudaStream_t)stream, nullptr, half_acc,
                          grad_feat, units);
}

msda_status msda_forward_oae(const void* feat, msda_dtype feat_dtype, const int32_t* spatial_shape,
                             const int32_t* scale_start_index, const float* sampling_location,
                             const void* weights, msda_dtype weights_dtype, const float* visibility, void* out,
                             msda_dtype out_dtype, int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P,
                             int G, const msda_tuning* tuning, msda_stream_t stream) {
    t_err[0] = 0;
    Problem p;
    msda_status st = validate("msda_forward_oae", feat, feat_dtype, spatial_shape, scale_start_index,
                              sampling_location, weights, weights_dtype, B, sum_hw, C, Ncam, Nscale, A, P, G, &p);
    if (st != MSDA_OK) return st;
    if (dtype_size(out_dtype) == 0) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_oae: unknown out dtype");
    if ((long long)B * A > 0 && !out) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_oae: out is NULL");
    if ((long long)B * A * Ncam > 0 && !visibility)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_oae: visibility is NULL");
    if (!aligned16(out) || !aligned16(visibility))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_oae: out and visibility must be 16-byte aligned");
    prefer_split(tuning, &p, 2);
    const bool units = !(tuning && tuning->variant == 4);
    return launch_forward(p, out, out_dtype, pick_warps(tuning, 8), (cudaStream_t)stream,
                          visibility ? visibility : nullptr, false, nullptr, units);
}

size_t msda_backward_workspace_size(int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                                    int deterministic) {
    if (B < 0 || sum_hw < 0 || C < 1 || Ncam < 0 || Nscale < 0 || A < 0 || P < 0 || G < 1) return 0;
    if (!deterministic) return 256;  // the work counter of the dynamic item order
    Problem p;
    p.B = B; p.sum_hw = sum_hw; p.C = C; p.Ncam = Ncam; p.Nscale = Nscale; p.A = A; p.P = P; p.G = G;
    p.Cg = C / G;
    const size_t a = backward_det_workspace(p), b = cg_backward_workspace(p);
    return a > b ? a : b;
}

msda_status msda_backward(const void* feat, msda_dtype feat_dtype, const int32_t* spatial_shape,
                          const int32_t* scale_start_index, const float* sampling_location,
                          const void* weights, msda_dtype weights_dtype, const float* grad_out,
                          float* grad_feat, float* grad_loc, float* grad_weights,
                          int B, int sum_hw, int C, int Ncam, int Nscale, int A, int P, int G,
                          int deterministic, void* workspace, size_t workspace_bytes,
                          const msda_tuning* tuning, msda_stream_t stream) {
    t_err[0] = 0;
    Problem p;
    msda_status st = validate("msda_backward", feat, feat_dtype, spatial_shape, scale_start_index,
                              sampling_location, weights, weights_dtype, B, sum_hw, C, Ncam, Nscale, A, P, G, &p);
    if (st != MSDA_OK) return st;
    const bool any_pts = (long long)B * A * P * Ncam > 0;
    if ((long long)B * A > 0 && !grad_out) return fail(MSDA_ERR_INVALID_ARG, "msda_backward: grad_out is NULL");
    if ((long long)B * sum_hw > 0 && !grad_feat) return fail(MSDA_ERR_INVALID_ARG, "msda_backward: grad_feat is NULL");
    if (any_pts && (!grad_loc || (Nscale > 0 && !grad_weights)))
        return fail(MSDA_ERR_INVALID_ARG, "msda_backward: grad_loc/grad_weights is NULL");
    if (!aligned16(grad_out) || !aligned16(grad_feat) || !aligned16(grad_loc) || !aligned16(grad_weights))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: gradient pointers must be 16-byte aligned");
    if (p.C % 4 != 0) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: C must be a multiple of 4");
    prefer_split(tuning, &p, 2);
    const int warps = pick_warps(tuning, 4);
    if (deterministic) {
        if (workspace && !aligned16(workspace))
            return fail(MSDA_ERR_WORKSPACE, "msda_backward: workspace must be 256-byte aligned");
        const bool staged = tuning && tuning->variant == 2;  // the staged camera-group form
        if (staged && cg_supported(p))
            return launch_backward_cg(p, grad_out, grad_feat, grad_loc, grad_weights, workspace, workspace_bytes,
                                      (cudaStream_t)stream);
        const bool cells = !(tuning && tuning->variant == 5);  // variant 5: the corner-slot form
        return launch_backward_det(p, grad_out, grad_feat, grad_loc, grad_weights, workspace, workspace_bytes,
                                   warps, cells, (cudaStream_t)stream);
    }
    if (workspace && !aligned16(workspace))
        return fail(MSDA_ERR_WORKSPACE, "msda_backward: workspace must be 16-byte aligned");
    const bool zeroed = tuning && (tuning->flags & MSDA_FLAG_GRAD_FEAT_ZEROED);
    return launch_backward_atomic(p, grad_out, grad_feat, grad_loc, grad_weights, workspace, workspace_bytes, warps,
                                  zeroed, (cudaStream_t)stream);
}

size_t msda_forward_batched_workspace_size(int num_scenes) {
    return num_scenes < 0 ? 0 : batched_workspace(num_scenes);
}

msda_status msda_forward_batched(const msda_scene* scenes, int num_scenes, int total_anchors, int max_ncam,
                                 int Nscale, int C, int P, int G, msda_dtype feat_dtype,
                                 msda_dtype weights_dtype, msda_dtype out_dtype, void* workspace,
                                 size_t workspace_bytes, uint64_t* scene_done_ns, const msda_tuning* tuning,
                                 msda_stream_t stream) {
    t_err[0] = 0;
    if (num_scenes < 0 || total_anchors < 0 || max_ncam < 0 || Nscale < 0 || P < 0)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched: negative dimension");
    if (C < 1 || G < 1 || C % G) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched: need C %% G == 0");
    if (Nscale > kMaxScales) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: Nscale too large");
    if (dtype_size(feat_dtype) == 0 || dtype_size(weights_dtype) == 0 || dtype_size(out_dtype) == 0)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched: unknown dtype");
    if ((C / G) * dtype_size(feat_dtype) % 16 != 0)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: (C/G)*sizeof(feat) not a multiple of 16");
    if (num_scenes > 0 && !scenes) return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched: scenes is NULL");
    if (num_scenes == 0 && total_anchors > 0)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched: anchors without scenes");
    if (!aligned16(scenes) || !aligned16(scene_done_ns) || !aligned16(workspace))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: pointers must be 16-byte aligned");
    return launch_forward_batched(scenes, num_scenes, total_anchors, max_ncam, Nscale, C, P, G, feat_dtype,
                                  weights_dtype, out_dtype, workspace, workspace_bytes, scene_done_ns,
                                  pick_warps(tuning, 8), tuning ? tuning->blocks_per_sm : 0,
                                  tuning && tuning->vectors_per_lane > 0 ? tuning->vectors_per_lane : 2,
                                  (cudaStream_t)stream);
}

int msda_forward_batched_noalloc_max_scenes(void) { return batched_noalloc_max_scenes(); }

msda_status msda_forward_batched_noalloc(const msda_scene* scenes, int num_scenes, int total_anchors,
                                         int max_ncam, int Nscale, int C, int P, int G, msda_dtype feat_dtype,
                                         msda_dtype weights_dtype, msda_dtype out_dtype, uint64_t* scene_done_ns,
                                         const msda_tuning* tuning, msda_stream_t stream) {
    t_err[0] = 0;
    const char* fn = "msda_forward_batched_noalloc";
    if (num_scenes < 0 || total_anchors < 0 || max_ncam < 0 || Nscale < 0 || P < 0)
        return fail(MSDA_ERR_INVALID_ARG, "%s: negative dimension", fn);
    if (num_scenes > batched_noalloc_max_scenes())
        return fail(MSDA_ERR_INVALID_ARG, "%s: %d scenes exceed the built-in limit of %d", fn, num_scenes,
                    batched_noalloc_max_scenes());
    if (C < 1 || G < 1 || C % G) return fail(MSDA_ERR_INVALID_ARG, "%s: need C %% G == 0", fn);
    if (Nscale > kMaxScales) return fail(MSDA_ERR_UNSUPPORTED, "%s: Nscale too large", fn);
    if (dtype_size(feat_dtype) == 0 || dtype_size(weights_dtype) == 0 || dtype_size(out_dtype) == 0)
        return fail(MSDA_ERR_INVALID_ARG, "%s: unknown dtype", fn);
    if ((C / G) * dtype_size(feat_dtype) % 16 != 0)
        return fail(MSDA_ERR_UNSUPPORTED, "%s: (C/G)*sizeof(feat) not a multiple of 16", fn);
    if (num_scenes > 0 && !scenes) return fail(MSDA_ERR_INVALID_ARG, "%s: scenes is NULL", fn);
    if (num_scenes == 0 && total_anchors > 0) return fail(MSDA_ERR_INVALID_ARG, "%s: anchors without scenes", fn);
    if (!aligned16(scenes) || !aligned16(scene_done_ns))
        return fail(MSDA_ERR_UNSUPPORTED, "%s: pointers must be 16-byte aligned", fn);
    return launch_forward_batched_noalloc(scenes, num_scenes, total_anchors, max_ncam, Nscale, C, P, G, feat_dtype,
                                          weights_dtype, out_dtype, scene_done_ns, pick_warps(tuning, 8),
                                          tuning ? tuning->blocks_per_sm : 0,
                                          tuning && tuning->vectors_per_lane > 0 ? tuning->vectors_per_lane : 2,
                                          (cudaStream_t)stream);
}

msda_status msda_keypoints(const float* anchors, const float* offsets, const float* dt, const float* proj,
                           const float* img_wh, float* sampling_location, int B, int A, int P, int Ncam,
                           msda_stream_t stream) {
    t_err[0] = 0;
    if (B < 0 || A < 0 || P < 0 || Ncam < 0) return fail(MSDA_ERR_INVALID_ARG, "msda_keypoints: negative dimension");
    const long long n = (long long)B * A * P * Ncam;
    if (n > 0 && (!anchors || !offsets || !dt || !proj || !img_wh || !sampling_location))
        return fail(MSDA_ERR_INVALID_ARG, "msda_keypoints: NULL pointer");
    if (!aligned16(anchors) || !aligned16(offsets) || !aligned16(dt) || !aligned16(proj) || !aligned16(img_wh) ||
        !aligned16(sampling_location))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_keypoints: pointers must be 16-byte aligned");
    return launch_keypoints(anchors, offsets, dt, proj, img_wh, sampling_location, B, A, P, Ncam,
                            (cudaStream_t)stream);
}

msda_status msda_debug_set_wait_limit(long long polls) {
    t_err[0] = 0;
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    if ((st = cg_set_wait_limit(polls)) != MSDA_OK) return st;
    return cb_set_wait_limit(polls);
}

msda_status msda_get_device_status(msda_stream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    int v = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&v, dev.status, sizeof(int), cudaMemcpyDeviceToHost);
    const int zero = 0;
    if (e == cudaSuccess) e = cudaMemcpy(dev.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(MSDA_ERR_CUDA, "msda_get_device_status: %s", cudaGetErrorString(e));
    return (msda_status)v;
}

msda_status msda_probe_read(const void* buf, size_t bytes, int reps, int blocks, int rows, uint32_t* sink,
                            msda_stream_t stream) {
    t_err[0] = 0;
    if (!buf || !sink || reps < 1 || blocks < 1 || rows < 0 || bytes < 512 || bytes % 16)
        return fail(MSDA_ERR_INVALID_ARG, "msda_probe_read: bad arguments");
    if (!aligned16(buf) || !aligned16(sink)) return fail(MSDA_ERR_UNSUPPORTED, "msda_probe_read: alignment");
    return launch_probe(buf, bytes, reps, blocks, rows, sink, (cudaStream_t)stream);
}

msda_status msda_probe_reduce(float* buf, size_t bytes, int reps, int blocks, int rows, msda_stream_t stream) {
    t_err[0] = 0;
    if (!buf || reps < 1 || blocks < 1 || rows < 1 || bytes < 1024 || bytes % 1024)
        return fail(MSDA_ERR_INVALID_ARG, "msda_probe_reduce: bad arguments");
    if (!aligned16(buf)) return fail(MSDA_ERR_UNSUPPORTED, "msda_probe_reduce: alignment");
    return launch_probe_reduce(buf, bytes, reps, blocks, rows, (cudaStream_t)stream);
}

}  // extern "C"
