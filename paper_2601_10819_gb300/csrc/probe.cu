// Bandwidth probes (a measurement aid; no counterpart in the paper).
//
// The operator is a gather: it reads each feature row about ten times, so
// its speed is set by how fast the SMs can pull 16-byte chunks of random
// 512-byte rows out of L2, not only by HBM.  These kernels measure the two
// roofs on the running GPU:
//   * streaming: every thread reads consecutive 16-byte chunks of `buf`
//     `reps` times (L2-only loads, ld.global.cg); a buffer smaller than L2
//     gives the L2 read bandwidth, a larger one the HBM bandwidth;
//   * gather: every warp reads `rows` pseudo-random 512-byte rows of `buf`
//     per rep, one 16-byte chunk per lane, like the operator's corner loads.
// The XOR of everything read decides a store that never happens in
// practice, so the compiler cannot drop the loads.
#include "common.cuh"
#include "internal.h"

namespace msda {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // 32-bit integer finaliser (xorshift-multiply rounds)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(512) probe_stream_kernel(const uint4* __restrict__ buf, size_t n16, int reps,
                                                           uint32_t* __restrict__ sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(512) probe_gather_kernel(const uint4* __restrict__ buf, uint32_t nrows, int reps,
                                                           int rows, uint32_t* __restrict__ sink) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r) {
        for (int j = 0; j < rows; j += 8) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t row = mix32(gw * 0x9e3779b9u + (uint32_t)(r * rows + j + u)) % nrows;
                v[u] = __ldcg(buf + (size_t)row * 32 + lane);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
    }
    if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

// Reduction probe: every warp adds 1.0 to `rows` pseudo-random 1 KB rows of FP32 per rep with 16-byte vector
// reductions (red.global.add.v4.f32, two per lane and row), the scatter pattern of the atomic backward.  With
// a buffer that fits in L2 it measures the L2's FP32 reduction throughput.
__global__ void __launch_bounds__(512) probe_reduce_kernel(float* __restrict__ buf, uint32_t nrows, int reps,
                                                           int rows) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < reps; ++r) {
        for (int j = 0; j < rows; ++j) {
            const uint32_t row = mix32(gw * 0x9e3779b9u + (uint32_t)(r * rows + j)) % nrows;
            float* base = buf + (size_t)row * 256 + 4 * lane;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                             :: "l"(__cvta_generic_to_global(base + 128 * h)), "f"(1.0f), "f"(1.0f), "f"(1.0f),
                                "f"(1.0f));
        }
    }
}

msda_status launch_probe_reduce(float* buf, size_t bytes, int reps, int blocks, int rows, cudaStream_t stream) {
    const size_t nrows = bytes / 1024;
    if (nrows == 0 || nrows > 0xffffffffull) return fail(MSDA_ERR_INVALID_ARG, "msda_probe_reduce: rows");
    probe_reduce_kernel<<<blocks, 512, 0, stream>>>(buf, (uint32_t)nrows, reps, rows);
    return check_launch("msda_probe_reduce");
}

msda_status launch_probe(const void* buf, size_t bytes, int reps, int blocks, int rows, uint32_t* sink,
                         cudaStream_t stream) {
    if (rows > 0) {
        const size_t nrows = bytes / 512;
        if (nrows == 0 || nrows > 0xffffffffull) return fail(MSDA_ERR_INVALID_ARG, "msda_probe_read: rows");
        probe_gather_kernel<<<blocks, 512, 0, stream>>>(reinterpret_cast<const uint4*>(buf), (uint32_t)nrows,
                                                        reps, (rows + 7) / 8 * 8, sink);
    } else {
        probe_stream_kernel<<<blocks, 512, 0, stream>>>(reinterpret_cast<const uint4*>(buf), bytes / 16, reps,
                                                        sink);
    }
    return check_launch("msda_probe_read");
}

}  // namespace msda
