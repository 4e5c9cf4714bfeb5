// MSDA backward, atomic mode (sm_103a).
//
// Gradients of the forward of fwd.cu for the upstream gradient go[b, a, :]:
//   dfeat[row, c] += w_g * omega * go[c]          for every in-bound corner
//   dw[b,a,p,k,s,g] = sum_{c in g} go[c] * S[c]
//   du = sum_s W_s * w_g * sum_c go[c] ((1-fy)(F01-F00) + fy(F11-F10))
//   dv = sum_s H_s * w_g * sum_c go[c] ((1-fx)(F10-F00) + fx(F11-F01))
// (the paper's operator is an inference plugin, Sec. 5.3; this is the
// exact adjoint of the forward).
//
// Mapping: a persistent grid whose teams (rt lanes, each owning CPL
// contiguous channels) walk ONE global list of (camera, anchor, keypoint)
// items in camera-major order: team j of the whole grid takes items j,
// j + teams, ...  At any moment every team works inside the same fraction of
// one camera, so that camera's features and its FP32 feature-gradient rows
// stay in L2 while they are hit, and the work is balanced to one item.  One
// pass over an item reads its four corners per scale, reduces dw over the
// group's lanes and du/dv over the team with shuffles (fixed trees, no
// atomics: those two gradients are bitwise reproducible and independent of
// the launch shape), and scatters the feature gradient with 16-byte FP32
// vector atomics (red.global.add.v4.f32) in an interleaved lane layout, so
// each warp-wide atomic covers whole 32-byte sectors.
#include "common.cuh"
#include "internal.h"

namespace msda {

struct BwdArgs {
    const void* feat;
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* go;
    float* gfeat;
    float* gloc;
    float* gw;
    int B, sum_hw, C, Ncam, Nscale, A, P, G, Cg;
    int rt;
    int scatter;  // 0: skip the feature-gradient atomics (deterministic mode); 1, 2: scatter
    int wide;     // a lane's two 16-byte chunks are 32-byte aligned: one 256-bit load
    unsigned long long* counter;  // next unhanded item (dynamic order) or NULL (static stride)
    int* status;
};

constexpr int kItemsPerGrab = 4;  // items per team taken from the counter at once

// addr[0..3] += a * v as one 16-byte FP32 vector reduction in global memory with no return value
// (red.global.add.v4.f32, sm_90 and later).  Written out because atomicAdd(float4*) may be compiled as a
// generic-space atomic that returns the old values, which doubles the L2<->SM traffic of the scatter.
__device__ __forceinline__ void red_add_v4(float* addr, float a, const float4& v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "l"(__cvta_generic_to_global(addr)), "f"(a * v.x), "f"(a * v.y), "f"(a * v.z), "f"(a * v.w));
}

__device__ __forceinline__ float team_sum(float v, unsigned mask, int width) {
    for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// SCATTER = false builds the form without the feature-gradient reductions (dloc and dw of the deterministic
// modes for anchors too large for bwdlw.cu), which needs fewer registers.
template <typename FT, typename WT, int NV, bool SCATTER>
__global__ void __launch_bounds__(256) bwd_atomic_kernel(const BwdArgs p) {
    constexpr int VEC = Elem<FT>::VEC;
    constexpr int CPL = VEC * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nmaps = p.Ncam * p.Nscale;
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem);
    float4* sbox = reinterpret_cast<float4*>(smem + align16(sizeof(MapInfo) * (size_t)nmaps));
    for (int i = threadIdx.x; i < nmaps; i += blockDim.x)
        smap[i] = load_map(p.shape, p.start, i, p.sum_hw, p.status);
    __syncthreads();
    for (int k = threadIdx.x; k < p.Ncam; k += blockDim.x) sbox[k] = camera_box(smap + k * p.Nscale, p.Nscale);
    __syncthreads();

    const int tpw = 32 / p.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const int lane = threadIdx.x & 31;
    const int tiw = lane / p.rt;
    const int team = (threadIdx.x >> 5) * tpw + tiw;
    const int tl = lane & (p.rt - 1);
    const unsigned tmask = (p.rt == 32) ? 0xffffffffu : (((1u << p.rt) - 1u) << (tiw * p.rt));
    const int c0 = tl * CPL;          // contiguous channels of this lane (loads, dw, dloc)
    const int g = c0 / p.Cg;
    const int lg = p.Cg / CPL;        // lanes per group (power of two)
    const int ci = 4 * tl;            // interleaved channels of this lane (scatter): ci + j*4*rt
    const int cstride = 4 * p.rt;

    const long long BA = (long long)p.B * p.A;
    const long long per_cam = BA * p.P;
    const long long nitems = (long long)p.Ncam * per_cam;
    const long long total_teams = (long long)gridDim.x * nteams;
    // Global item list ordered (camera, anchor, keypoint); all teams walk it together.
    auto process = [&](long long item) {
        const int k = (int)(item / per_cam);
        const long long r = item - (long long)k * per_cam;
        const long long ba = r / p.P;
        const int pp = (int)(r - ba * p.P);
        const int b = (int)(ba / p.A);
        const long long pk = (ba * p.P + pp) * p.Ncam + k;
        const float2 uv = __ldg(reinterpret_cast<const float2*>(p.loc) + pk);
        float* gwrow = p.gw + pk * p.Nscale * p.G + g;
        if (!in_box(uv, sbox[k])) {
            // dropped at every scale: zero gradients for the point
            if ((tl & (lg - 1)) == 0)
                for (int s = 0; s < p.Nscale; ++s) gwrow[(long long)s * p.G] = 0.0f;
            if (tl == 0) reinterpret_cast<float2*>(p.gloc)[pk] = make_float2(0.0f, 0.0f);
            return;
        }
        const float* gorow = p.go + ba * p.C;
        float2 go[CPL / 2];
#pragma unroll
        for (int j = 0; j < CPL / 4; ++j) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(gorow + c0) + j);
            go[2 * j] = make_float2(t.x, t.y);
            go[2 * j + 1] = make_float2(t.z, t.w);
        }
        const FT* fb = reinterpret_cast<const FT*>(p.feat) + (long long)b * p.sum_hw * p.C + c0;
        float* gfb = p.gfeat + (long long)b * p.sum_hw * p.C + ci;
        const WT* wpt = reinterpret_cast<const WT*>(p.w) + pk * p.Nscale * p.G;  // weights of this point
        const WT* wrow = wpt + g;
        const MapInfo* mrow = smap + k * p.Nscale;
        float du = 0.0f, dv = 0.0f;
        for (int s = 0; s < p.Nscale; ++s) {
            const MapInfo m = mrow[s];
            Cell c;
            const bool in = (m.W != 0) && locate(uv.x, uv.y, m.H, m.W, c);  // uniform over the team
            float dwp = 0.0f;
            if (in) {
                const float wvs = ldw(wrow + (long long)s * p.G);
                const bool vx0 = c.x0 >= 0, vx1 = c.x0 + 1 < m.W;
                const bool vy0 = c.y0 >= 0, vy1 = c.y0 + 1 < m.H;
                const long long r00 = (long long)(m.start + c.y0 * m.W + c.x0) * p.C;
                const long long rW = (long long)m.W * p.C;
                const FT* p00 = fb + r00;
                uint4 q[4][NV];
                if (NV == 2 && p.wide && vx0 && vx1 && vy0 && vy1) {
                    ld32(p00, q[0][0], q[0][NV - 1]);
                    ld32(p00 + p.C, q[1][0], q[1][NV - 1]);
                    ld32(p00 + rW, q[2][0], q[2][NV - 1]);
                    ld32(p00 + rW + p.C, q[3][0], q[3][NV - 1]);
                } else if (vx0 && vx1 && vy0 && vy1) {
#pragma unroll
                    for (int n = 0; n < NV; ++n) {
                        q[0][n] = ld16(p00 + n * VEC);
                        q[1][n] = ld16(p00 + p.C + n * VEC);
                        q[2][n] = ld16(p00 + rW + n * VEC);
                        q[3][n] = ld16(p00 + rW + p.C + n * VEC);
                    }
                } else {
                    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int n = 0; n < NV; ++n) {
                        q[0][n] = (vy0 && vx0) ? ld16(p00 + n * VEC) : z;
                        q[1][n] = (vy0 && vx1) ? ld16(p00 + p.C + n * VEC) : z;
                        q[2][n] = (vy1 && vx0) ? ld16(p00 + rW + n * VEC) : z;
                        q[3][n] = (vy1 && vx1) ? ld16(p00 + rW + p.C + n * VEC) : z;
                    }
                }
                // d[q] = sum over this lane's channels of go * F_q (packed pairs)
                float2 d2[4];
#pragma unroll
                for (int cq = 0; cq < 4; ++cq) d2[cq] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int n = 0; n < NV; ++n) {
#pragma unroll
                    for (int cq = 0; cq < 4; ++cq) {
                        float2 f[VEC / 2];
                        widen2(q[cq][n], f, FT());
#pragma unroll
                        for (int j = 0; j < VEC / 2; ++j) d2[cq] = __ffma2_rn(go[n * (VEC / 2) + j], f[j], d2[cq]);
                    }
                }
                const float d00 = d2[0].x + d2[0].y, d01 = d2[1].x + d2[1].y;
                const float d10 = d2[2].x + d2[2].y, d11 = d2[3].x + d2[3].y;
                const float ax = 1.0f - c.fx, ay = 1.0f - c.fy;
                const float o00 = ax * ay, o01 = c.fx * ay, o10 = ax * c.fy, o11 = c.fx * c.fy;
                dwp = o00 * d00 + o01 * d01 + o10 * d10 + o11 * d11;
                du = fmaf((float)m.W * wvs, ay * (d01 - d00) + c.fy * (d11 - d10), du);
                dv = fmaf((float)m.H * wvs, ax * (d10 - d00) + c.fx * (d11 - d01), dv);
                if (SCATTER && p.scatter) {
                    // feature gradient w * omega * go, in the interleaved layout: each warp-wide
                    // 16-byte vector atomic covers 4*rt contiguous channels (whole sectors);
                    // an interleaved chunk belongs to its own group, with its own weight
                    float* g00 = gfb + r00;
#pragma unroll
                    for (int j = 0; j < CPL / 4; ++j) {
                        const float wj = ldw(wpt + (long long)s * p.G + (ci + j * cstride) / p.Cg);
                        const float c00 = wj * o00, c01 = wj * o01, c10 = wj * o10, c11 = wj * o11;
                        const float4 gv = __ldg(reinterpret_cast<const float4*>(gorow + ci + j * cstride));
                        float* qq = g00 + j * cstride;
                        if (vy0 && vx0) red_add_v4(qq, c00, gv);
                        if (vy0 && vx1) red_add_v4(qq + p.C, c01, gv);
                        if (vy1 && vx0) red_add_v4(qq + rW, c10, gv);
                        if (vy1 && vx1) red_add_v4(qq + rW + p.C, c11, gv);
                    }
                }
            }
            // weight gradient of group g at this scale: reduce over the group's lanes
            const float dw = team_sum(dwp, tmask, lg);
            if ((tl & (lg - 1)) == 0) gwrow[(long long)s * p.G] = dw;
        }
        du = team_sum(du, tmask, p.rt);
        dv = team_sum(dv, tmask, p.rt);
        if (tl == 0) reinterpret_cast<float2*>(p.gloc)[pk] = make_float2(du, dv);
        };
    if (p.counter) {
        // dynamic order: each block takes the next kItemsPerGrab items per team from one counter, so
        // items are handed out strictly in camera order and no team runs ahead of the others
        __shared__ unsigned long long s_base;
        const unsigned long long chunk = (unsigned long long)nteams * kItemsPerGrab;
        for (;;) {
            if (threadIdx.x == 0) s_base = atomicAdd(p.counter, chunk);
            __syncthreads();
            const unsigned long long base = s_base;
            __syncthreads();
            if (base >= (unsigned long long)nitems) break;
            for (int j = 0; j < kItemsPerGrab; ++j) {
                const long long item = (long long)base + (long long)j * nteams + team;
                if (item < nitems) process(item);
            }
        }
    } else {
        for (long long item = (long long)blockIdx.x * nteams + team; item < nitems; item += total_teams) process(item);
    }
}

using BwdKernel = void (*)(const BwdArgs);

template <typename FT, typename WT, bool SCATTER>
static BwdKernel bwd_pick_nv(int nv) {
    switch (nv) {
        case 1: return bwd_atomic_kernel<FT, WT, 1, SCATTER>;
        case 2: return bwd_atomic_kernel<FT, WT, 2, SCATTER>;
        case 4: return bwd_atomic_kernel<FT, WT, 4, SCATTER>;
    }
    return nullptr;
}

template <bool SCATTER>
static BwdKernel bwd_kernel_for(msda_dtype ft, msda_dtype wt, int nv) {
    if (ft == MSDA_F32 && wt == MSDA_F32) return bwd_pick_nv<float, float, SCATTER>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_BF16) return bwd_pick_nv<__nv_bfloat16, __nv_bfloat16, SCATTER>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_F32) return bwd_pick_nv<__nv_bfloat16, float, SCATTER>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F16) return bwd_pick_nv<__half, __half, SCATTER>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F32) return bwd_pick_nv<__half, float, SCATTER>(nv);
    return nullptr;
}

size_t bwd_smem_bytes(const Problem& p) {
    return align16(sizeof(MapInfo) * (size_t)p.Ncam * p.Nscale) + sizeof(float4) * (size_t)p.Ncam;
}

msda_status launch_backward_atomic(const Problem& p, const float* grad_out, float* grad_feat,
                                   float* grad_loc, float* grad_w, void* ws, size_t ws_bytes, int warps,
                                   bool zeroed, cudaStream_t stream) {
    unsigned long long* counter = (ws && ws_bytes >= sizeof(unsigned long long))
                                      ? reinterpret_cast<unsigned long long*>(ws) : nullptr;
    return launch_backward_loc_w(p, grad_out, grad_feat, grad_loc, grad_w, warps, zeroed ? 2 : 1, stream, counter);
}

msda_status launch_backward_loc_w(const Problem& p, const float* grad_out, float* grad_feat,
                                  float* grad_loc, float* grad_w, int warps, int scatter,
                                  cudaStream_t stream, unsigned long long* counter) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    BwdKernel k = scatter ? bwd_kernel_for<true>(p.feat_t, p.w_t, p.nv) : bwd_kernel_for<false>(p.feat_t, p.w_t, p.nv);
    if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: unsupported feature/weight dtype pair");
    const size_t feat_bytes = sizeof(float) * (size_t)p.B * p.sum_hw * p.C;
    if (scatter == 1 && feat_bytes && cudaMemsetAsync(grad_feat, 0, feat_bytes, stream) != cudaSuccess)
        return check_launch("msda_backward memset");
    const long long nblocks = (long long)p.B * p.A;
    if (nblocks == 0) return MSDA_OK;
    const size_t smem = bwd_smem_bytes(p);
    st = ensure_smem((const void*)k, smem, dev);
    if (st != MSDA_OK) return st;
    BwdArgs a;
    a.feat = p.feat; a.shape = p.shape; a.start = p.start; a.loc = p.loc; a.w = p.w;
    a.go = grad_out; a.gfeat = grad_feat; a.gloc = grad_loc; a.gw = grad_w;
    a.B = p.B; a.sum_hw = p.sum_hw; a.C = p.C; a.Ncam = p.Ncam; a.Nscale = p.Nscale;
    a.A = p.A; a.P = p.P; a.G = p.G; a.Cg = p.Cg; a.rt = p.rt; a.scatter = scatter; a.status = dev.status;
    a.counter = counter;
    {
        const size_t esz = (size_t)dtype_size(p.feat_t);
        a.wide = (p.nv == 2 && ((uintptr_t)p.feat % 32) == 0 && ((size_t)p.C * esz) % 32 == 0 &&
                  ((size_t)p.sum_hw * p.C * esz) % 32 == 0) ? 1 : 0;
    }
    if (counter && cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream) != cudaSuccess)
        return check_launch("msda_backward counter");
    // persistent grid: as many blocks as fit at once, all walking one camera-major item list
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, warps * 32, smem) != cudaSuccess || occ < 1)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: kernel does not fit on an SM");
    const long long items = (long long)p.Ncam * nblocks * p.P;
    const int nteams = warps * (32 / p.rt);
    long long grid = (long long)occ * dev.sm_count;
    const long long needed = (items + nteams - 1) / nteams;
    if (grid > needed) grid = needed;
    if (grid < 1) grid = 1;
    k<<<(unsigned)grid, warps * 32, smem, stream>>>(a);
    return check_launch("msda_backward");
}

}  // namespace msda
