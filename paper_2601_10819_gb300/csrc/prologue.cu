// Keypoint prologue (sm_103a): the sampling locations the operator consumes.
//
// Sec. 3.1 and 3.2 of the paper: each anchor box carries fixed geometric and
// learned keypoints; the keypoints are moved by the object's estimated
// velocity (motion compensation) and projected into every camera with its
// intrinsic and extrinsic parameters.  Here, for keypoint p of anchor a in
// camera k:
//   q   = R(yaw) (offset_p * (w, l, h)) + centre + velocity * dt
//   h   = M_k (q, 1)             (M_k: 3x4 world -> homogeneous pixels)
//   loc = (h_x / h_z / width_k, h_y / h_z / height_k), or (-2, -2) when
//         h_z <= 1e-5 (behind the camera: a location the operator drops).
// One thread per (b, a, p, k), camera fastest, so consecutive threads write
// consecutive 8-byte locations; the anchor, its offsets and the 64 camera
// matrices stay in L1.
#include "common.cuh"
#include "internal.h"

namespace msda {

__global__ void __launch_bounds__(256) keypoints_kernel(const float* __restrict__ anchors,
                                                        const float* __restrict__ offsets,
                                                        const float* __restrict__ dt,
                                                        const float* __restrict__ proj,
                                                        const float* __restrict__ img_wh, float2* __restrict__ loc,
                                                        long long n, int A, int P, int Ncam) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % Ncam);
        const long long t = i / Ncam;
        const int p = (int)(t % P);
        const long long ba = t / P;
        const long long b = ba / A;
        const float* an = anchors + ba * 11;
        const float* of = offsets + (ba * P + p) * 3;
        const float bx = __ldg(of + 0) * __ldg(an + 3);
        const float by = __ldg(of + 1) * __ldg(an + 4);
        const float bz = __ldg(of + 2) * __ldg(an + 5);
        const float sy = __ldg(an + 6), cy = __ldg(an + 7), d = __ldg(dt + b);
        const float qx = fmaf(cy, bx, -sy * by) + __ldg(an + 0) + __ldg(an + 8) * d;
        const float qy = fmaf(sy, bx, cy * by) + __ldg(an + 1) + __ldg(an + 9) * d;
        const float qz = bz + __ldg(an + 2) + __ldg(an + 10) * d;
        const float* M = proj + (b * Ncam + k) * 12;
        float h[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            h[r] = fmaf(__ldg(M + 4 * r), qx, fmaf(__ldg(M + 4 * r + 1), qy, fmaf(__ldg(M + 4 * r + 2), qz, __ldg(M + 4 * r + 3))));
        float2 o;
        if (h[2] <= 1e-5f) {
            o = make_float2(-2.0f, -2.0f);
        } else {
            o = make_float2(h[0] / h[2] / __ldg(img_wh + 2 * k), h[1] / h[2] / __ldg(img_wh + 2 * k + 1));
        }
        loc[i] = o;
    }
}

msda_status launch_keypoints(const float* anchors, const float* offsets, const float* dt, const float* proj,
                             const float* img_wh, float* loc, int B, int A, int P, int Ncam, cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    const long long n = (long long)B * A * P * Ncam;
    if (n == 0) return MSDA_OK;
    long long grid = (n + 255) / 256;
    if (grid > (long long)dev.sm_count * 32) grid = (long long)dev.sm_count * 32;
    keypoints_kernel<<<(unsigned)grid, 256, 0, stream>>>(anchors, offsets, dt, proj, img_wh,
                                                         reinterpret_cast<float2*>(loc), n, A, P, Ncam);
    return check_launch("msda_keypoints");
}

}  // namespace msda
