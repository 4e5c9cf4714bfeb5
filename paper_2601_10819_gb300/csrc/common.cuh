// Device helpers shared by the MSDA kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "msda.h"

namespace msda {

constexpr int kMaxScales = 16;  // Nscale limit of the single-scene kernels
constexpr int kScaleChunk = 4;  // scales whose corner loads are issued together

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// Feature element traits: one 16-byte load carries VEC channels.
// ---------------------------------------------------------------------------
template <typename T> struct Elem;
template <> struct Elem<float> {
    static constexpr int VEC = 4;
    static constexpr msda_dtype id = MSDA_F32;
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr int VEC = 8;
    static constexpr msda_dtype id = MSDA_BF16;
};
template <> struct Elem<__half> {
    static constexpr int VEC = 8;
    static constexpr msda_dtype id = MSDA_F16;
};

// 16-byte read-only load (L1-cached, non-coherent path).
__device__ __forceinline__ uint4 ld16(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// 32 bytes (p 32-byte aligned) in one 256-bit read-only load (ld.global.nc.v8.b32, sm_100 and later).
__device__ __forceinline__ void ld32(const void* p, uint4& lo, uint4& hi) {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
                 : "l"(p));
}

// Widen the VEC channels of one 16-byte chunk to FP32.
__device__ __forceinline__ void widen(const uint4& v, float* f, float) {
    f[0] = __uint_as_float(v.x); f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z); f[3] = __uint_as_float(v.w);
}
__device__ __forceinline__ void widen(const uint4& v, float* f, __nv_bfloat16) {
    // BF16 -> FP32 is exact: the 16 bits become the upper half of the word.
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i + 0] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}
__device__ __forceinline__ void widen(const uint4& v, float* f, __half) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
        float2 t = __half22float2(h);
        f[2 * i + 0] = t.x;
        f[2 * i + 1] = t.y;
    }
}

// Widen 16 bytes into VEC/2 channel pairs (for packed FP32 math).
__device__ __forceinline__ void widen2(const uint4& v, float2* f, float) {
    f[0] = make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
    f[1] = make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
}
__device__ __forceinline__ void widen2(const uint4& v, float2* f, __nv_bfloat16) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = make_float2(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
}
__device__ __forceinline__ void widen2(const uint4& v, float2* f, __half) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
}

// Scalar weight load widened to FP32.
__device__ __forceinline__ float ldw(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldw(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldw(const __half* p) { return __half2float(__ldg(p)); }

// Store n consecutive FP32 values, narrowed to the output type (RNE).
__device__ __forceinline__ void store_out(float* o, float v) { *o = v; }
__device__ __forceinline__ void store_out(__nv_bfloat16* o, float v) { *o = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_out(__half* o, float v) { *o = __float2half_rn(v); }

// ---------------------------------------------------------------------------
// Projected location -> bilinear cell.
//
// x = u*W - 0.5 and y = v*H - 0.5 (pixel (i, j) centred at ((j+0.5)/W,
// (i+0.5)/H)).  The product u*W is split into its rounded value px and its
// exact rounding error ex (one FMA); xh = px - 0.5 is exact, so the exact
// coordinate is the pair x = xh + ex.  Every discrete decision (dropped or
// not, which cell) is taken on that exact pair, so it matches the exact
// real-number decision, and the fraction inside the cell carries ~2^-24
// absolute error instead of half an ulp of x (4e-6 px at W = 120).  This
// matters for the location gradient, which jumps across cell borders.  The
// intrinsics keep the compiler from fusing the product into the subtraction.
//
// Returns false when the point is dropped: x <= -1, x >= W, y <= -1,
// y >= H, or a NaN coordinate (every comparison with NaN is false).
// ---------------------------------------------------------------------------
struct Cell {
    int x0, y0;
    float fx, fy;
};

// In (-1, n) for the exact value xh + e (|e| below half an ulp of xh).
__device__ __forceinline__ bool in_open_range(float xh, float e, float n) {
    return (xh > -1.0f || (xh == -1.0f && e > 0.0f)) && (xh < n || (xh == n && e < 0.0f));
}

// floor and fraction of the exact value xh + e.
__device__ __forceinline__ void split_cell(float xh, float e, int& i0, float& f) {
    float fl = floorf(xh);
    f = __fadd_rn(__fsub_rn(xh, fl), e);
    if (f < 0.0f) {  // xh is an integer and the exact value lies just below it
        fl -= 1.0f;
        f = __fadd_rn(f, 1.0f);
    }
    i0 = (int)fl;
}

__device__ __forceinline__ bool locate(float u, float v, int H, int W, Cell& c) {
    const float Wf = (float)W, Hf = (float)H;
    const float px = __fmul_rn(u, Wf), py = __fmul_rn(v, Hf);
    const float ex = __fmaf_rn(u, Wf, -px), ey = __fmaf_rn(v, Hf, -py);
    const float xh = __fadd_rn(px, -0.5f), yh = __fadd_rn(py, -0.5f);
    if (!(in_open_range(xh, ex, Wf) && in_open_range(yh, ey, Hf))) return false;
    split_cell(xh, ex, c.x0, c.fx);
    split_cell(yh, ey, c.y0, c.fy);
    return true;
}

// Device status word: first non-zero code wins until the host reads it.
__device__ __forceinline__ void raise_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Per-map metadata staged in shared memory: H, W and the first row of the
// map inside one batch element.  A map that violates H >= 1, W >= 1,
// start >= 0, start + H*W <= sum_hw is stored with W = 0 (skipped) and
// reported through the status word.
struct MapInfo {
    int H, W, start;
};

__device__ __forceinline__ MapInfo load_map(const int32_t* shape, const int32_t* start, int idx,
                                            int sum_hw, int* status) {
    MapInfo m;
    m.H = __ldg(shape + 2 * idx + 0);
    m.W = __ldg(shape + 2 * idx + 1);
    m.start = __ldg(start + idx);
    const long long end = (long long)m.start + (long long)m.H * (long long)m.W;
    if (m.H < 1 || m.W < 1 || m.start < 0 || end > (long long)sum_hw) {
        raise_status(status, MSDA_ERR_OUT_OF_RANGE);
        m.H = 0;
        m.W = 0;
        m.start = 0;
    }
    return m;
}

// Normalised box outside of which a point is dropped at every scale of a
// camera: a point is kept at scale s iff u in (-0.5/W_s, 1 + 0.5/W_s) and
// v in (-0.5/H_s, 1 + 0.5/H_s), so the union over scales is the box of the
// smallest W and H.  The box is widened by a relative 1e-3 so rounding can
// only keep extra points (each scale still runs the exact test).
// Returns (u_lo, u_hi, v_lo, v_hi); an empty box if no map is valid.
__device__ __forceinline__ float4 camera_box(const MapInfo* maps, int Nscale) {
    int wmin = 0, hmin = 0;
    for (int s = 0; s < Nscale; ++s) {
        if (maps[s].W == 0) continue;
        if (wmin == 0 || maps[s].W < wmin) wmin = maps[s].W;
        if (hmin == 0 || maps[s].H < hmin) hmin = maps[s].H;
    }
    if (wmin == 0) return make_float4(1.0f, 0.0f, 1.0f, 0.0f);
    const float mu = 0.5f / (float)wmin * 1.001f + 1e-6f, mv = 0.5f / (float)hmin * 1.001f + 1e-6f;
    return make_float4(-mu, 1.0f + mu, -mv, 1.0f + mv);
}

__device__ __forceinline__ bool in_box(float2 uv, float4 b) {
    return uv.x > b.x && uv.x < b.y && uv.y > b.z && uv.y < b.w;  // false for NaN
}

}  // namespace msda
