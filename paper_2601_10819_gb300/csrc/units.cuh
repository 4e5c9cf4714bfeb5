// Point-scale lists of the two-stage anchor kernels (sm_103a).
//
// A block that owns one anchor takes the anchor's point-scales (camera k,
// keypoint p, scale s), flattened camera-major as u = (k * P + p) * Nscale + s,
// in chunks of kUnitsPerThread per thread.  Stage A (build_unit_list) culls
// each point-scale of the chunk (camera box, visibility factor, map range)
// and locates its bilinear cell once, into a record in shared memory, and
// lists the in-view ones in increasing u with a block scan.  Stage B (in the
// kernels) deals the list round-robin to the block's teams, which only load
// the corner rows and do their arithmetic; a team meets its records in
// increasing u, so its sums run in a fixed order.  The forward kernels
// (fwd.cu) write the same stage A out inline, between their zero stores:
// built through build_unit_list, the training forward ran 24 us slower on the
// 64-camera workload.
#pragma once

#include "common.cuh"

namespace msda {

constexpr int kUnitsPerThread = 4;

struct UnitRec {
    int row00;   // feature row of corner (y0, x0) inside the batch element (may be off the map: see the flags)
    int W;       // map width: rows between y0 and y0 + 1
    float fx, fy;
    int wf;      // (index of the point-scale's weights) << 4 | vx0 | vx1 << 1 | vy0 << 2 | vy1 << 3
    float scale; // camera factor of the fused occlusion-aware form, else 1
};

// Bytes of the record array, its 2-byte list and the scan scratch for `units` entries.
__host__ __device__ constexpr size_t unit_list_bytes(size_t units) {
    return units ? ((26 * units + 15) & ~size_t(15)) + 64 : 0;
}

// Exclusive block-wide prefix sum (blockDim.x a multiple of 32); *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int v, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < nw; ++w) {
            const int t = wsum[w];
            wsum[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const int r = x - v + wsum[warp];
    __syncthreads();  // wsum is reused by the next call
    return r;
}

// The list area: records, then their indices, then the scan scratch.
struct UnitList {
    UnitRec* rec;
    short* list;
    int* scan;
    __device__ __forceinline__ UnitList(unsigned char* area, int units) {
        rec = reinterpret_cast<UnitRec*>(area);
        list = reinterpret_cast<short*>(area + 24 * (size_t)units);
        scan = reinterpret_cast<int*>(area + ((26 * (size_t)units + 15) & ~size_t(15)));
    }
};

// Stage A for the chunk starting at u0: returns the number of listed point-scales (the same in every thread).
// dropped(pp, k, s) is called, by the thread that owns it, for each point-scale of the chunk that is not
// listed.  Ends with a block barrier, so the list is ready for stage B.
template <typename Dropped>
__device__ __forceinline__ int build_unit_list(int u0, int nunits, int P, int Ncam, int Nscale,
                                               const MapInfo* __restrict__ smap, const float4* __restrict__ sbox,
                                               const float2* __restrict__ sloc, const float* __restrict__ svn,
                                               const UnitList& ul, Dropped dropped) {
    const int per_cam = P * Nscale;
    const int mine = (int)threadIdx.x * kUnitsPerThread;
    unsigned vmask = 0u;
#pragma unroll
    for (int i = 0; i < kUnitsPerThread; ++i) {
        const int u = u0 + mine + i;
        if (u < nunits) {
            const int k = u / per_cam;
            const int rem = u - k * per_cam;
            const int pp = rem / Nscale;
            const int sc = rem - pp * Nscale;
            const float2 uv = sloc[pp * Ncam + k];
            const float cs = svn ? svn[k] : 1.0f;
            const MapInfo m = smap[k * Nscale + sc];
            Cell c;
            if (cs != 0.0f && in_box(uv, sbox[k]) && m.W != 0 && locate(uv.x, uv.y, m.H, m.W, c)) {
                UnitRec r;
                r.row00 = m.start + c.y0 * m.W + c.x0;
                r.W = m.W;
                r.fx = c.fx;
                r.fy = c.fy;
                r.wf = ((((pp * Ncam + k) * Nscale) + sc) << 4) | (c.x0 >= 0 ? 1 : 0) | (c.x0 + 1 < m.W ? 2 : 0) |
                       (c.y0 >= 0 ? 4 : 0) | (c.y0 + 1 < m.H ? 8 : 0);
                r.scale = cs;
                ul.rec[mine + i] = r;
                vmask |= 1u << i;
            } else {
                dropped(pp, k, sc);
            }
        }
    }
    int off = block_excl_scan(__popc(vmask), ul.scan, ul.scan + 8);
#pragma unroll
    for (int i = 0; i < kUnitsPerThread; ++i)
        if (vmask & (1u << i)) ul.list[off++] = (short)(mine + i);
    __syncthreads();
    return ul.scan[8];
}

}  // namespace msda
