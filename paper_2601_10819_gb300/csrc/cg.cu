// Camera-group (CG) kernels (sm_103a): the shared-memory-staged form of the
// MSDA forward and of its deterministic backward.
//
// Why.  The operator reads every feature row about ten times (each map is
// sampled by all anchors' keypoints), so the direct form moves ~10x the
// unique bytes through L2 and is bound by the L2 gather rate, not by HBM.
// Here one CTA owns a (batch element b, camera k, channel group g, anchor
// range) unit.  It stages the camera's coarse scales for its group into
// shared memory with TMA (cp.async.bulk.tensor, one elected thread, one
// mbarrier; the paper's asynchronous global->shared prefetch of feature
// tiles, Sec. 5.3), so only the finest scale is gathered from L2, and every
// staged row serves all of the unit's anchors.
//
// Mapping inside a unit.  A team of 2*LPC lanes owns one anchor at a time:
// lanes [0, LPC) read the left column (x0) and lanes [LPC, 2*LPC) the right
// column (x0+1) of a point's bilinear cell, each lane one 16-byte chunk of
// the group's Cg channels, top and bottom rows.  A quarter warp therefore
// reads two adjacent rows, which fall in different shared-memory bank
// halves (no conflicts).  The two columns are combined with one shuffle per
// anchor.  Everything is accumulated in FP32 in a fixed order.
//
// Forward: the unit writes its per-camera partial sums; a second kernel sums
// the cameras in order (deterministic).  Backward: the same gather computes
// dw (per group, written directly) and the group's share of dloc (summed over
// groups in order by a second kernel).  The feature gradient is computed as
// a gather too: every map's in-view points are sorted by bilinear cell with
// a stable counting sort, and one team per feature row sums the
// contributions of the four cells that touch the row, in sorted order, with
// grad_out staged in shared memory.  No atomics reach global memory, every
// row is written once, and the result is bitwise reproducible.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace msda {

constexpr int kCgMaxScales = 4;      // scales handled by the CG kernels
constexpr int kCgBoxRows = 32;       // rows per TMA box
constexpr int kCgMaxCells = 40960;   // bilinear cells per map in the cell sort
constexpr int kCgBlock = 512;                // threads of the gather kernels
constexpr int kCgStageBytes = 200 * 1024;    // upper bound of the staging area

// ---------------------------------------------------------------------------
// PTX helpers: TMA tensor copies (the mbarrier helpers are in tma.cuh)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint4 lds16(const void* p) {
    return *reinterpret_cast<const uint4*>(p);
}

// ---------------------------------------------------------------------------
// Unit description shared by the forward and backward gathers
// ---------------------------------------------------------------------------
struct CgArgs {
    const void* feat;
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* go;       // backward: grad_out [B, A, C]
    float* part;           // forward: [B][Ncam][A][C]; backward: dloc partials [G][B*A*P*Ncam] float2
    float* gw;             // backward: grad_weights
    int B, sum_hw, C, Ncam, Nscale, A, P, G, Cg;
    int apu, n_ar;         // anchors per unit, anchor ranges
    long long nunits;
    int stage_bytes;       // shared-memory staging budget
    int* status;
};

struct UnitInfo {
    int b, k, g, a0, a1;
};

__device__ __forceinline__ UnitInfo decode_unit(long long u, const CgArgs& p) {
    UnitInfo r;
    r.g = (int)(u % p.G);
    long long t = u / p.G;
    const int ar = (int)(t % p.n_ar);
    t /= p.n_ar;
    r.k = (int)(t % p.Ncam);
    r.b = (int)(t / p.Ncam);
    r.a0 = ar * p.apu;
    r.a1 = min(p.A, r.a0 + p.apu);
    return r;
}

// Stage the coarse scales of (b, k, g) that fit into the budget (smallest
// maps first).  Called by all threads; thread 0 issues the TMA copies and
// waits; returns false (and raises MSDA_ERR_TIMEOUT) if the copies did not
// land within the spin limit.
template <typename FT>
__device__ bool stage_unit(const CUtensorMap* tmap, const CgArgs& p, const UnitInfo& u, unsigned char* stage,
                           uint64_t* bar, uint32_t& phase, MapInfo* smap, int* soff, int* sflag) {
    const int rowbytes = p.Cg * (int)sizeof(FT);
    if (threadIdx.x < p.Nscale) smap[threadIdx.x] = load_map(p.shape, p.start, u.k * p.Nscale + threadIdx.x, p.sum_hw, p.status);
    __syncthreads();
    if (threadIdx.x == 0) {
        // greedy: smallest maps first while they fit
        int order[kCgMaxScales];
        for (int s = 0; s < p.Nscale; ++s) order[s] = s;
        for (int i = 1; i < p.Nscale; ++i)
            for (int j = i; j > 0; --j) {
                const long long aj = (long long)smap[order[j]].H * smap[order[j]].W;
                const long long ai = (long long)smap[order[j - 1]].H * smap[order[j - 1]].W;
                if (aj < ai) { const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t; }
            }
        int used = 0;  // rows
        for (int s = 0; s < p.Nscale; ++s) soff[s] = -1;
        for (int i = 0; i < p.Nscale; ++i) {
            const int s = order[i];
            const MapInfo m = smap[s];
            if (m.W == 0) continue;
            const int rows = (m.H * m.W + kCgBoxRows - 1) / kCgBoxRows * kCgBoxRows;
            if ((long long)(used + rows) * rowbytes > p.stage_bytes) break;
            soff[s] = used;
            used += rows;
        }
        const uint32_t bytes = (uint32_t)used * (uint32_t)rowbytes;
        mbar_arrive_expect_tx(bar, bytes);
        const int x = u.g * p.Cg;
        for (int s = 0; s < p.Nscale; ++s) {
            if (soff[s] < 0) continue;
            const MapInfo m = smap[s];
            const int nbox = (m.H * m.W + kCgBoxRows - 1) / kCgBoxRows;
            const int y0 = u.b * p.sum_hw + m.start;
            for (int i = 0; i < nbox; ++i)
                tma_load_2d(stage + (size_t)(soff[s] + i * kCgBoxRows) * rowbytes, tmap, x, y0 + i * kCgBoxRows, bar);
        }
        const bool ok = mbar_wait_first(bar, phase);
        if (!ok) {
            raise_status(p.status, MSDA_ERR_TIMEOUT);
            mbar_wait_drain(bar, phase);  // the copies in flight land before the CTA goes on
        }
        *sflag = ok ? 1 : 0;
    }
    __syncthreads();
    phase ^= 1u;
    return *sflag != 0;
}

// Lane view of one point-scale: which rows of this lane's column exist.
struct Corner2 {
    bool in;        // the point-scale is in view
    bool vt, vb;    // top / bottom row of this lane's column inside the map
    int r;          // row of the top corner inside the map
    float fx, fy;
};

__device__ __forceinline__ Corner2 corner2(float2 uv, const MapInfo& m, int col) {
    Corner2 c2;
    Cell c;
    c2.in = (m.W != 0) && locate(uv.x, uv.y, m.H, m.W, c);
    c2.vt = c2.vb = false;
    c2.r = 0;
    c2.fx = c2.fy = 0.0f;
    if (!c2.in) return c2;
    const int xc = c.x0 + col;
    const bool vx = xc >= 0 && xc < m.W;
    c2.vt = vx && c.y0 >= 0;
    c2.vb = vx && c.y0 + 1 < m.H;
    c2.r = c.y0 * m.W + xc;
    c2.fx = c.fx;
    c2.fy = c.fy;
    return c2;
}

__device__ __forceinline__ float team_sum_w(float v, unsigned mask, int width) {
    for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

constexpr int kPB = 4;   // points of one anchor whose global loads are issued together
constexpr int kNG = 2;   // non-staged scales whose rows are held in registers per point

// MODE 0: forward partial sums.  MODE 1: backward dw and group dloc.
//
// Per anchor the team first has the anchor's P locations in shared memory
// (loaded while the previous anchor was being processed).  Points are then
// taken kPB at a time: phase 1 issues every global load of the batch (the
// weights of all scales and the two rows of up to kNG non-staged scales);
// phase 2 reads the staged scales from shared memory and accumulates.
template <typename FT, typename WT, int LPC, int MODE>
__global__ void __launch_bounds__(512, 1) cg_gather_kernel(const __grid_constant__ CUtensorMap tmap, const CgArgs p) {
    constexpr int VEC = Elem<FT>::VEC;
    constexpr int TEAM = 2 * LPC;
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ MapInfo smap[kCgMaxScales];
    __shared__ int soff[kCgMaxScales];
    __shared__ int sflag;

    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / TEAM;
    const int nteams = blockDim.x / TEAM;
    const int tl = lane % TEAM;
    const int col = tl / LPC;
    const int q = tl % LPC;
    const unsigned tmask = (TEAM == 32) ? 0xffffffffu : (((1u << TEAM) - 1u) << ((lane / TEAM) * TEAM));
    const int rowbytes = p.Cg * (int)sizeof(FT);
    // per-team location slot after the staging area
    float2* sloc = reinterpret_cast<float2*>(stage + p.stage_bytes) + (size_t)team * p.P;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const WT* wbase = reinterpret_cast<const WT*>(p.w);
    const float2* gloc = reinterpret_cast<const float2*>(p.loc);

    for (long long unit = blockIdx.x; unit < p.nunits; unit += gridDim.x) {
        const UnitInfo u = decode_unit(unit, p);
        const bool ok = stage_unit<FT>(&tmap, p, u, stage, &bar, phase, smap, soff, &sflag);
        if (!ok) break;  // copies did not land: the status word says so; every thread leaves
        // global-scale slots: which scales are read from global memory, in order
        int gsc[kCgMaxScales];
        int ng = 0;
#pragma unroll
        for (int s = 0; s < kCgMaxScales; ++s) {
            gsc[s] = -1;
            if (s < p.Nscale && soff[s] < 0 && smap[s].W != 0) gsc[s] = ng++;
        }
        const FT* fb = reinterpret_cast<const FT*>(p.feat) + (long long)u.b * p.sum_hw * p.C + u.g * p.Cg + q * VEC;

        // locations of the team's first anchor
        int a = u.a0 + team;
        float2 pre[2];
        auto fetch_locs = [&](int an) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int i = tl + j * TEAM;
                pre[j] = make_float2(0.f, 0.f);
                if (an < u.a1 && i < p.P)
                    pre[j] = __ldg(gloc + (((long long)u.b * p.A + an) * p.P + i) * p.Ncam + u.k);
            }
        };
        auto store_locs = [&]() {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int i = tl + j * TEAM;
                if (i < p.P) sloc[i] = pre[j];
            }
        };
        fetch_locs(a);
        store_locs();
        __syncwarp(tmask);
        // locations beyond 2*TEAM per anchor are read directly
        for (; a < u.a1; a += nteams) {
            fetch_locs(a + nteams);  // next anchor's locations, consumed after this one
            const long long ba = (long long)u.b * p.A + a;
            float acc[VEC];
            float go[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j) acc[j] = 0.0f;
            if (MODE == 1) {
                const float4* gsrc = reinterpret_cast<const float4*>(p.go + ba * p.C + u.g * p.Cg + q * VEC);
#pragma unroll
                for (int j = 0; j < VEC / 4; ++j) {
                    const float4 t = __ldg(gsrc + j);
                    go[4 * j] = t.x; go[4 * j + 1] = t.y; go[4 * j + 2] = t.z; go[4 * j + 3] = t.w;
                }
            }
            for (int p0 = 0; p0 < p.P; p0 += kPB) {
                // phase 1: global loads of the batch
                float wv[kPB][kCgMaxScales];
                uint4 gt[kPB][kNG], gbm[kPB][kNG];
#pragma unroll
                for (int pb = 0; pb < kPB; ++pb) {
                    const int pp = p0 + pb;
                    const bool vp = pp < p.P;
                    const float2 uv = vp ? (pp < 2 * TEAM ? sloc[pp]
                                                          : __ldg(gloc + (ba * p.P + pp) * p.Ncam + u.k))
                                         : make_float2(0.f, 0.f);
                    const long long pk = (ba * p.P + (vp ? pp : 0)) * p.Ncam + u.k;
#pragma unroll
                    for (int s = 0; s < kCgMaxScales; ++s) {
                        wv[pb][s] = 0.0f;
                        if (s >= p.Nscale || !vp) continue;
                        const Corner2 c2 = corner2(uv, smap[s], col);
                        if (!c2.in) continue;
                        wv[pb][s] = ldw(wbase + (pk * p.Nscale + s) * p.G + u.g);
                        const int gi = gsc[s];
                        if (gi >= 0 && gi < kNG) {
                            const FT* base = fb + ((long long)smap[s].start + c2.r) * p.C;
#pragma unroll
                            for (int j = 0; j < kNG; ++j) {
                                if (j != gi) continue;
                                gt[pb][j] = c2.vt ? ld16(base) : make_uint4(0u, 0u, 0u, 0u);
                                gbm[pb][j] = c2.vb ? ld16(base + (long long)smap[s].W * p.C) : make_uint4(0u, 0u, 0u, 0u);
                            }
                        }
                    }
                }
                // phase 2: staged scales from shared memory, accumulate
#pragma unroll
                for (int pb = 0; pb < kPB; ++pb) {
                    const int pp = p0 + pb;
                    if (pp >= p.P) break;
                    const float2 uv = pp < 2 * TEAM ? sloc[pp] : __ldg(gloc + (ba * p.P + pp) * p.Ncam + u.k);
                    const long long pk = (ba * p.P + pp) * p.Ncam + u.k;
                    float du = 0.0f, dv = 0.0f;
#pragma unroll
                    for (int s = 0; s < kCgMaxScales; ++s) {
                        if (s >= p.Nscale) break;
                        const MapInfo m = smap[s];
                        const Corner2 c2 = corner2(uv, m, col);
                        float dwp = 0.0f;
                        if (c2.in) {
                            uint4 rt = make_uint4(0u, 0u, 0u, 0u), rb = rt;
                            const int gi = gsc[s];
                            if (soff[s] >= 0) {
                                const unsigned char* sb = stage + (long long)(soff[s] + c2.r) * rowbytes + q * 16;
                                if (c2.vt) rt = lds16(sb);
                                if (c2.vb) rb = lds16(sb + (long long)m.W * rowbytes);
                            } else if (gi < kNG) {
#pragma unroll
                                for (int j = 0; j < kNG; ++j)
                                    if (j == gi) { rt = gt[pb][j]; rb = gbm[pb][j]; }
                            } else {
                                const FT* base = fb + ((long long)m.start + c2.r) * p.C;
                                if (c2.vt) rt = ld16(base);
                                if (c2.vb) rb = ld16(base + (long long)m.W * p.C);
                            }
                            float ft[VEC], fbv[VEC];
                            widen(rt, ft, FT());
                            widen(rb, fbv, FT());
                            const float wx = col ? c2.fx : 1.0f - c2.fx;
                            const float wt = wx * (1.0f - c2.fy), wbt = wx * c2.fy;
                            const float w = wv[pb][s];
                            if (MODE == 0) {
                                const float ct = w * wt, cb = w * wbt;
#pragma unroll
                                for (int j = 0; j < VEC; ++j) acc[j] = fmaf(cb, fbv[j], fmaf(ct, ft[j], acc[j]));
                            } else {
                                float gxp = 0.0f, gyp = 0.0f;
                                const float ay = 1.0f - c2.fy;
#pragma unroll
                                for (int j = 0; j < VEC; ++j) {
                                    dwp = fmaf(go[j], wt * ft[j] + wbt * fbv[j], dwp);
                                    gxp = fmaf(go[j], ay * ft[j] + c2.fy * fbv[j], gxp);
                                    gyp = fmaf(go[j], fbv[j] - ft[j], gyp);
                                }
                                du = fmaf((float)m.W * w, col ? gxp : -gxp, du);
                                dv = fmaf((float)m.H * w, wx * gyp, dv);
                            }
                        }
                        if (MODE == 1) {
                            const float dw = team_sum_w(dwp, tmask, TEAM);
                            if (tl == 0) p.gw[(pk * p.Nscale + s) * p.G + u.g] = dw;
                        }
                    }
                    if (MODE == 1) {
                        du = team_sum_w(du, tmask, TEAM);
                        dv = team_sum_w(dv, tmask, TEAM);
                        if (tl == 0) {
                            const long long npk = (long long)p.B * p.A * p.P * p.Ncam;
                            reinterpret_cast<float2*>(p.part)[(long long)u.g * npk + pk] = make_float2(du, dv);
                        }
                    }
                }
            }
            if (MODE == 0) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) acc[j] += __shfl_xor_sync(tmask, acc[j], LPC);
                if (col == 0) {
                    float* dst = p.part + (((long long)u.b * p.Ncam + u.k) * p.A + a) * p.C + u.g * p.Cg + q * VEC;
#pragma unroll
                    for (int j = 0; j < VEC; j += 4)
                        *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
                }
            }
            __syncwarp(tmask);  // everyone is done with this anchor's locations
            store_locs();
            __syncwarp(tmask);
        }
        __syncthreads();  // the next unit overwrites the staged rows
        if (threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
}

// out[b, a, c] = sum over cameras k (in order) of part[b][k][a][c]
__global__ void __launch_bounds__(256) cg_reduce_cams_kernel(const float* __restrict__ part, void* out, int out_t,
                                                             int B, int Ncam, int A, int C) {
    const long long n4 = (long long)B * A * C / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const long long e = i * 4;
        const long long b = e / ((long long)A * C);
        const long long rem = e - b * A * C;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < Ncam; ++k) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(part + ((b * Ncam + k) * A) * C + rem));
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
        if (out_t == MSDA_F32) {
            *reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + e) = s;
        } else if (out_t == MSDA_BF16) {
            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + e;
            o[0] = __float2bfloat16_rn(s.x); o[1] = __float2bfloat16_rn(s.y);
            o[2] = __float2bfloat16_rn(s.z); o[3] = __float2bfloat16_rn(s.w);
        } else {
            __half* o = reinterpret_cast<__half*>(out) + e;
            o[0] = __float2half_rn(s.x); o[1] = __float2half_rn(s.y);
            o[2] = __float2half_rn(s.z); o[3] = __float2half_rn(s.w);
        }
    }
}

// grad_loc = sum over groups g (in order) of the group partials
__global__ void __launch_bounds__(256) cg_reduce_groups_kernel(const float2* __restrict__ part, float2* __restrict__ gl,
                                                               long long npk, int G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npk; i += (long long)gridDim.x * blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < G; ++g) {
            const float2 v = __ldg(part + (long long)g * npk + i);
            s.x += v.x;
            s.y += v.y;
        }
        gl[i] = s;
    }
}

// ---------------------------------------------------------------------------
// Deterministic feature gradient: cell sort (per map) + row gather (per unit)
// ---------------------------------------------------------------------------
struct SortArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    int w_t;
    int B, sum_hw, Ncam, Nscale, A, P, G;
    int* cell_base;       // [B*Ncam*Nscale + 1] first cell of each map (exclusive prefix)
    int* cell_off;        // [total cells + maps] record offsets per cell (per map: cells + 1 entries)
    int* scratch_cell;    // [maps][A*P] cell id of each point (-1 if out of view)
    int* scratch_pos;     // [maps][A*P] record slot
    int4* rec_hdr;        // [maps][A*P] {point, fx bits, fy bits, 0}
    float* rec_w;         // [G][maps*A*P] FP32 weights of each record
    long long cells_cap;
    int* status;
};

// One block: per-map cell counts (H+1)*(W+1) and their exclusive prefix.
__global__ void __launch_bounds__(1024) cell_base_kernel(const SortArgs a) {
    __shared__ long long carry_s;
    __shared__ int ws[32];
    const int nmaps = a.B * a.Ncam * a.Nscale;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nmaps; base += blockDim.x) {
        const int m = base + threadIdx.x;
        int cells = 0;
        if (m < nmaps) {
            const int km = m % (a.Ncam * a.Nscale);
            const MapInfo mi = load_map(a.shape, a.start, km, a.sum_hw, a.status);
            cells = (mi.W == 0) ? 0 : (mi.H + 1) * (mi.W + 1);
            if (cells > kCgMaxCells) {
                raise_status(a.status, MSDA_ERR_UNSUPPORTED);
                cells = 0;
            }
        }
        // block inclusive scan of `cells`
        int v = cells;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) ws[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int s = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const long long incl = carry_s + v + (warp > 0 ? ws[warp - 1] : 0);
        if (m < nmaps) a.cell_base[m] = (int)(incl - cells);
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry_s + nmaps > a.cells_cap) raise_status(a.status, MSDA_ERR_UNSUPPORTED);
        a.cell_base[nmaps] = (int)carry_s;
    }
}

// One block per map (b, k, s): stable counting sort of its in-view points by cell.
__global__ void __launch_bounds__(256) cell_sort_kernel(const SortArgs a) {
    extern __shared__ int cnt[];  // cells + 1
    __shared__ int ws[32];
    __shared__ int carry_s;
    const int map = blockIdx.x;
    const int km = map % (a.Ncam * a.Nscale);
    const int b = map / (a.Ncam * a.Nscale);
    const int k = km / a.Nscale, s = km % a.Nscale;
    const MapInfo m = load_map(a.shape, a.start, km, a.sum_hw, nullptr);
    const long long npts = (long long)a.A * a.P;
    int cells = (m.W == 0) ? 0 : (m.H + 1) * (m.W + 1);
    // the table of this map must match what cell_base_kernel reserved and fit the capacity;
    // otherwise the map is skipped (its points count as out of view, its rows get no contribution)
    const bool tab_ok = cells > 0 && cells <= kCgMaxCells && a.cell_base[map + 1] - a.cell_base[map] == cells &&
                        (long long)a.cell_base[map] + map + cells + 1 <= a.cells_cap;
    if (!tab_ok) cells = 0;
    int* coff = a.cell_off + a.cell_base[map] + map;  // cells + 1 entries (only touched when tab_ok)
    int* sc = a.scratch_cell + (long long)map * npts;
    int* spos = a.scratch_pos + (long long)map * npts;
    for (int i = threadIdx.x; i <= cells; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    // 1. cells and counts
    for (long long i = threadIdx.x; i < npts; i += blockDim.x) {
        const long long ba = (long long)b * a.A + i / a.P;
        const int pp = (int)(i % a.P);
        const float2 uv = __ldg(reinterpret_cast<const float2*>(a.loc) + (ba * a.P + pp) * a.Ncam + k);
        Cell c;
        int cell = -1;
        if (cells > 0 && locate(uv.x, uv.y, m.H, m.W, c)) {
            cell = (c.y0 + 1) * (m.W + 1) + (c.x0 + 1);
            atomicAdd(&cnt[cell], 1);
        }
        sc[i] = cell;
    }
    __syncthreads();
    // 2. exclusive prefix over cells (also the final total at cnt[cells])
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base <= cells; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int cv = (i < cells) ? cnt[i] : 0;
        int v = cv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) ws[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int sv = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += t;
            }
            ws[lane] = sv;
        }
        __syncthreads();
        const int excl = carry_s + v - cv + (warp > 0 ? ws[warp - 1] : 0);
        if (i <= cells) {
            cnt[i] = excl;   // becomes the running cursor
            if (tab_ok) coff[i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = excl + cv;
        __syncthreads();
    }
    // 3. stable slots: one warp walks the points in order
    if (warp == 0) {
        const unsigned lt = (1u << lane) - 1u;
        for (long long base = 0; base < npts; base += 32) {
            const long long i = base + lane;
            const int cell = (i < npts) ? sc[i] : -1;
            const unsigned act = __ballot_sync(0xffffffffu, cell >= 0);
            const unsigned peers = __match_any_sync(0xffffffffu, cell) & act;
            int pos = -1;
            if (cell >= 0) pos = cnt[cell] + __popc(peers & lt);
            __syncwarp();
            if (cell >= 0 && lane == __ffs(peers) - 1) cnt[cell] += __popc(peers);
            __syncwarp();
            if (i < npts) spos[i] = pos;
        }
    }
    __syncthreads();
    // 4. records
    const long long rbase = (long long)map * npts;
    const long long nrec_all = (long long)a.B * a.Ncam * a.Nscale * npts;
    for (long long i = threadIdx.x; i < npts; i += blockDim.x) {
        const int pos = spos[i];
        if (pos < 0) continue;
        const long long ba = (long long)b * a.A + i / a.P;
        const int pp = (int)(i % a.P);
        const long long pk = (ba * a.P + pp) * a.Ncam + k;
        const float2 uv = __ldg(reinterpret_cast<const float2*>(a.loc) + pk);
        Cell c;
        locate(uv.x, uv.y, m.H, m.W, c);
        a.rec_hdr[rbase + pos] = make_int4((int)i, __float_as_int(c.fx), __float_as_int(c.fy), 0);
        const long long wi = (pk * a.Nscale + s) * a.G;
        for (int g = 0; g < a.G; ++g) {
            float wv;
            if (a.w_t == MSDA_F32) wv = ldw(reinterpret_cast<const float*>(a.w) + wi + g);
            else if (a.w_t == MSDA_BF16) wv = ldw(reinterpret_cast<const __nv_bfloat16*>(a.w) + wi + g);
            else wv = ldw(reinterpret_cast<const __half*>(a.w) + wi + g);
            a.rec_w[(long long)g * nrec_all + rbase + pos] = wv;
        }
    }
}

// Rows of grad_feat that no map covers are zeroed; rows covered twice are reported.
__global__ void __launch_bounds__(256) cover_kernel(const int32_t* shape, const int32_t* start, int sum_hw,
                                                    int nmaps_per_b, unsigned int* cov) {
    const int map = blockIdx.x;
    const int b = map / nmaps_per_b, km = map % nmaps_per_b;
    const MapInfo m = load_map(shape, start, km, sum_hw, nullptr);
    const long long hw = (long long)m.H * m.W;
    for (long long r = threadIdx.x; r < hw; r += blockDim.x) atomicAdd(cov + (long long)b * sum_hw + m.start + r, 1u);
}

__global__ void __launch_bounds__(256) fill_uncovered_kernel(const unsigned int* __restrict__ cov, float* gfeat,
                                                             long long nrows, int C, int* status) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows; r += (long long)gridDim.x * blockDim.x) {
        const unsigned int c = cov[r];
        if (c == 0u) {
            float4* dst = reinterpret_cast<float4*>(gfeat + r * C);
            for (int j = 0; j < C / 4; ++j) dst[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (c > 1u) {
            raise_status(status, MSDA_ERR_OUT_OF_RANGE);  // overlapping maps
        }
    }
}

struct RowArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* go;
    const int* cell_base;
    const int* cell_off;
    const int4* rec_hdr;
    const float* rec_w;
    float* gfeat;
    int B, sum_hw, C, Ncam, Nscale, A, P, G, Cg;
    int n_rr;            // row ranges per (b, k, g)
    long long nunits;
    long long cells_cap;
    int* status;
};

// One unit = (b, k, g, row range): grad_out[b, :, g] staged in shared memory;
// one team of Cg/4 lanes per feature row sums the row's contributions.
__global__ void __launch_bounds__(512, 1) row_gather_kernel(const RowArgs a) {
    extern __shared__ __align__(16) float gos[];  // [A][Cg]
    __shared__ MapInfo smap[kCgMaxScales];
    __shared__ int srows[kCgMaxScales + 1];
    const int TEAM = a.Cg / 4;  // lanes per row (<= 32, power of two)
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / TEAM;
    const int nteams = blockDim.x / TEAM;
    const int tl = lane % TEAM;
    const long long npts = (long long)a.A * a.P;
    const long long nrec_all = (long long)a.B * a.Ncam * a.Nscale * npts;
    for (long long unit = blockIdx.x; unit < a.nunits; unit += gridDim.x) {
        const int g = (int)(unit % a.G);
        long long t = unit / a.G;
        const int rr = (int)(t % a.n_rr);
        t /= a.n_rr;
        const int k = (int)(t % a.Ncam);
        const int b = (int)(t / a.Ncam);
        if (threadIdx.x < a.Nscale) smap[threadIdx.x] = load_map(a.shape, a.start, k * a.Nscale + threadIdx.x, a.sum_hw, nullptr);
        // stage grad_out[b, :, g*Cg:(g+1)*Cg]
        const int c4 = a.Cg / 4;
        for (int i = threadIdx.x; i < a.A * c4; i += blockDim.x) {
            const int an = i / c4, j = i % c4;
            reinterpret_cast<float4*>(gos)[i] =
                __ldg(reinterpret_cast<const float4*>(a.go + ((long long)b * a.A + an) * a.C + g * a.Cg) + j);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            srows[0] = 0;
            for (int s = 0; s < a.Nscale; ++s) srows[s + 1] = srows[s] + smap[s].H * smap[s].W;
        }
        __syncthreads();
        const int total_rows = srows[a.Nscale];
        const int per = (total_rows + a.n_rr - 1) / a.n_rr;
        const int r0 = rr * per, r1 = min(total_rows, r0 + per);
        for (int row = r0 + team; row < r1; row += nteams) {
            int s = 0;
            while (s + 1 < a.Nscale && row >= srows[s + 1]) ++s;
            const MapInfo m = smap[s];
            const int r = row - srows[s];
            const int i = r / m.W, j = r - (r / m.W) * m.W;
            const int map = (b * a.Ncam + k) * a.Nscale + s;
            const int cb = a.cell_base[map];
            const int* coff = a.cell_off + cb + map;
            const long long rbase = (long long)map * npts;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            // a map whose cell table was rejected (too many cells) contributes nothing
            const bool table_ok = (a.cell_base[map + 1] - cb == (m.H + 1) * (m.W + 1)) &&
                                  ((long long)cb + map + (m.H + 1) * (m.W + 1) + 1 <= a.cells_cap);
#pragma unroll
            for (int nb = 0; nb < 4; ++nb) {
                if (!table_ok) break;
                const int dy = 1 - (nb >> 1), dx = 1 - (nb & 1);  // this row is corner (dy, dx) of cell (i-dy, j-dx)
                const int cell = (i - dy + 1) * (m.W + 1) + (j - dx + 1);
                const int e0 = coff[cell], e1 = coff[cell + 1];
                for (int e = e0; e < e1; ++e) {
                    const int4 h = __ldg(a.rec_hdr + rbase + e);
                    const float fx = __int_as_float(h.y), fy = __int_as_float(h.z);
                    const float om = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy);
                    const float coef = __ldg(a.rec_w + (long long)g * nrec_all + rbase + e) * om;
                    const int an = (int)(h.x / a.P);
                    const float4 gv = reinterpret_cast<const float4*>(gos)[an * c4 + tl];
                    acc.x = fmaf(coef, gv.x, acc.x);
                    acc.y = fmaf(coef, gv.y, acc.y);
                    acc.z = fmaf(coef, gv.z, acc.z);
                    acc.w = fmaf(coef, gv.w, acc.w);
                }
            }
            float* dst = a.gfeat + ((long long)b * a.sum_hw + m.start + r) * a.C + g * a.Cg + 4 * tl;
            *reinterpret_cast<float4*>(dst) = acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static bool make_tmap(CUtensorMap* map, const Problem& p) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = p.feat_t == MSDA_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : p.feat_t == MSDA_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const int es = dtype_size(p.feat_t);
    cuuint64_t dims[2] = {(cuuint64_t)p.C, (cuuint64_t)p.B * (cuuint64_t)p.sum_hw};
    cuuint64_t strides[1] = {(cuuint64_t)p.C * es};
    cuuint32_t box[2] = {(cuuint32_t)p.Cg, (cuuint32_t)kCgBoxRows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, dt, 2, const_cast<void*>(p.feat), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The CG kernels handle: Nscale <= 4, a group row of 16..128 bytes split into
// LPC 16-byte chunks with LPC in {1, 2, 4, 8}, rows addressable with int32.
static int cg_lpc(const Problem& p) {
    const int rowbytes = p.Cg * dtype_size(p.feat_t);
    if (rowbytes % 16) return 0;
    const int lpc = rowbytes / 16;
    return (lpc == 1 || lpc == 2 || lpc == 4 || lpc == 8) ? lpc : 0;
}

bool cg_supported(const Problem& p) {
    return p.Nscale >= 1 && p.Nscale <= kCgMaxScales && cg_lpc(p) > 0 && p.Cg <= 256 && p.P <= 64 &&
           (long long)p.B * p.sum_hw < (1ll << 30) && encode_fn() != nullptr;
}

using CgKernel = void (*)(const CUtensorMap, const CgArgs);

template <typename FT, typename WT, int MODE>
static CgKernel cg_pick_lpc(int lpc) {
    switch (lpc) {
        case 1: return cg_gather_kernel<FT, WT, 1, MODE>;
        case 2: return cg_gather_kernel<FT, WT, 2, MODE>;
        case 4: return cg_gather_kernel<FT, WT, 4, MODE>;
        case 8: return cg_gather_kernel<FT, WT, 8, MODE>;
    }
    return nullptr;
}

template <int MODE>
static CgKernel cg_kernel_for(msda_dtype ft, msda_dtype wt, int lpc) {
    if (ft == MSDA_F32 && wt == MSDA_F32) return cg_pick_lpc<float, float, MODE>(lpc);
    if (ft == MSDA_BF16 && wt == MSDA_BF16) return cg_pick_lpc<__nv_bfloat16, __nv_bfloat16, MODE>(lpc);
    if (ft == MSDA_BF16 && wt == MSDA_F32) return cg_pick_lpc<__nv_bfloat16, float, MODE>(lpc);
    if (ft == MSDA_F16 && wt == MSDA_F16) return cg_pick_lpc<__half, __half, MODE>(lpc);
    if (ft == MSDA_F16 && wt == MSDA_F32) return cg_pick_lpc<__half, float, MODE>(lpc);
    return nullptr;
}


// Anchor ranges per (b, k, g): keep the wave tail short.
static int pick_ranges(long long base_units, int A, int sms) {
    int best = 1;
    double best_eff = 0.0;
    for (int n = 1; n <= 8; ++n) {
        if (n > A) break;
        const long long units = base_units * n;
        const double waves = (double)units / sms;
        const double eff = waves / std::ceil(waves) - 0.01 * (n - 1);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = n; }
    }
    return best;
}

static size_t cg_loc_bytes(const Problem& p) {
    return sizeof(float2) * (size_t)(kCgBlock / 2) * (size_t)p.P;  // nteams <= kCgBlock / 2
}

static msda_status launch_cg(const Problem& p, CgKernel k, const CgArgs& a0, const DeviceInfo& dev,
                             cudaStream_t stream) {
    CUtensorMap map;
    if (!make_tmap(&map, p)) return fail(MSDA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    const size_t smem = (size_t)a0.stage_bytes + cg_loc_bytes(p);
    msda_status st = ensure_smem((const void*)k, smem, dev);
    if (st != MSDA_OK) return st;
    long long grid = a0.nunits;
    if (grid > (long long)dev.sm_count * 64) grid = (long long)dev.sm_count * 64;
    if (grid < 1) return MSDA_OK;
    k<<<(unsigned)grid, kCgBlock, smem, stream>>>(map, a0);
    return check_launch("cg gather");
}

static CgArgs cg_args(const Problem& p, const DeviceInfo& dev) {
    CgArgs a;
    a.feat = p.feat; a.shape = p.shape; a.start = p.start; a.loc = p.loc; a.w = p.w;
    a.go = nullptr; a.part = nullptr; a.gw = nullptr;
    a.B = p.B; a.sum_hw = p.sum_hw; a.C = p.C; a.Ncam = p.Ncam; a.Nscale = p.Nscale;
    a.A = p.A; a.P = p.P; a.G = p.G; a.Cg = p.Cg;
    const long long base = (long long)p.B * p.Ncam * p.G;
    a.n_ar = pick_ranges(base, p.A, dev.sm_count);
    a.apu = (p.A + a.n_ar - 1) / a.n_ar;
    a.nunits = base * a.n_ar;
    // the staging area takes what the location slots and the static shared memory leave
    long long room = (long long)dev.max_smem_optin - 1024 - (long long)cg_loc_bytes(p);
    if (room > kCgStageBytes) room = kCgStageBytes;
    a.stage_bytes = room > 0 ? (int)(room / 128 * 128) : 0;
    a.status = dev.status;
    return a;
}

size_t cg_forward_workspace(const Problem& p) {
    return align_up(sizeof(float) * (size_t)p.B * p.Ncam * p.A * p.C, 256);
}

msda_status launch_forward_cg(const Problem& p, void* out, msda_dtype out_t, void* ws, size_t ws_bytes,
                              cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    const size_t need = cg_forward_workspace(p);
    if (!ws || ws_bytes < need) return fail(MSDA_ERR_WORKSPACE, "msda_forward: workspace needs %zu bytes", need);
    CgKernel k = cg_kernel_for<0>(p.feat_t, p.w_t, cg_lpc(p));
    if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward: no staged kernel for this dtype pair");
    if ((long long)p.B * p.A == 0) return MSDA_OK;
    CgArgs a = cg_args(p, dev);
    a.part = reinterpret_cast<float*>(ws);
    if (p.Ncam > 0 && p.Nscale > 0 && p.P > 0) {
        st = launch_cg(p, k, a, dev, stream);
        if (st != MSDA_OK) return st;
    } else if (need && cudaMemsetAsync(ws, 0, need, stream) != cudaSuccess) {  // nothing is sampled
        return check_launch("msda_forward memset");
    }
    const long long n4 = (long long)p.B * p.A * p.C / 4;
    long long grid = (n4 + 255) / 256;
    if (grid > (long long)dev.sm_count * 16) grid = (long long)dev.sm_count * 16;
    cg_reduce_cams_kernel<<<(unsigned)grid, 256, 0, stream>>>(reinterpret_cast<float*>(ws), out, out_t, p.B, p.Ncam,
                                                              p.A, p.C);
    return check_launch("msda_forward reduce");
}

// Deterministic backward workspace layout.
struct CgBwdLayout {
    size_t dloc, cell_base, cell_off, sc, spos, hdr, recw, cov, total;
    long long cells_cap;
};

static CgBwdLayout cg_bwd_layout(const Problem& p) {
    CgBwdLayout L;
    const long long nmaps = (long long)p.B * p.Ncam * p.Nscale;
    const long long npts = (long long)p.A * p.P;
    const long long nrec = nmaps * npts;
    // cells per map <= 2*H*W + 2 <= 2*sum_hw + 2 summed over non-overlapping maps, plus one per map
    L.cells_cap = 2ll * p.B * p.sum_hw + 4 * nmaps + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.dloc = take(sizeof(float2) * (size_t)p.G * p.B * p.A * p.P * p.Ncam);
    L.cell_base = take(sizeof(int) * (size_t)(nmaps + 1));
    L.cell_off = take(sizeof(int) * (size_t)L.cells_cap);
    L.sc = take(sizeof(int) * (size_t)nrec);
    L.spos = take(sizeof(int) * (size_t)nrec);
    L.hdr = take(sizeof(int4) * (size_t)nrec);
    L.recw = take(sizeof(float) * (size_t)nrec * p.G);
    L.cov = take(sizeof(unsigned int) * (size_t)p.B * p.sum_hw);
    L.total = off;
    return L;
}

size_t cg_backward_workspace(const Problem& p) { return cg_bwd_layout(p).total; }

msda_status launch_backward_cg(const Problem& p, const float* grad_out, float* grad_feat, float* grad_loc,
                               float* grad_w, void* ws, size_t ws_bytes, cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    const CgBwdLayout L = cg_bwd_layout(p);
    if (!ws || ws_bytes < L.total)
        return fail(MSDA_ERR_WORKSPACE, "msda_backward: deterministic mode needs %zu workspace bytes", L.total);
    if (p.Cg % 4 || p.Cg / 4 > 32 || ((p.Cg / 4) & (p.Cg / 4 - 1)))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: deterministic mode needs C/G in {4, 8, ..., 128}");
    const long long nrec = (long long)p.B * p.Ncam * p.Nscale * p.A * p.P;
    if (nrec >= (1ll << 31) || (long long)p.A * p.P >= (1ll << 31))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: too many points for deterministic mode");
    unsigned char* base = reinterpret_cast<unsigned char*>(ws);
    const long long npk = (long long)p.B * p.A * p.P * p.Ncam;
    const long long nrows = (long long)p.B * p.sum_hw;

    // 1. dw and per-group dloc by the staged gather, then dloc summed over groups
    if (npk > 0) {
        CgKernel k = cg_kernel_for<1>(p.feat_t, p.w_t, cg_lpc(p));
        if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: no staged kernel for this dtype pair");
        CgArgs a = cg_args(p, dev);
        a.go = grad_out;
        a.part = reinterpret_cast<float*>(base + L.dloc);
        a.gw = grad_w;
        if (p.Nscale > 0) {
            st = launch_cg(p, k, a, dev, stream);
            if (st != MSDA_OK) return st;
            long long grid = (npk + 255) / 256;
            if (grid > (long long)dev.sm_count * 16) grid = (long long)dev.sm_count * 16;
            cg_reduce_groups_kernel<<<(unsigned)grid, 256, 0, stream>>>(
                reinterpret_cast<const float2*>(base + L.dloc), reinterpret_cast<float2*>(grad_loc), npk, p.G);
            if ((st = check_launch("msda_backward dloc")) != MSDA_OK) return st;
        } else if (cudaMemsetAsync(grad_loc, 0, sizeof(float2) * npk, stream) != cudaSuccess) {
            return check_launch("msda_backward memset");
        }
    }
    if (nrows == 0) return MSDA_OK;

    // 2. rows no map covers are zero; overlapping maps are reported
    unsigned int* cov = reinterpret_cast<unsigned int*>(base + L.cov);
    if (cudaMemsetAsync(cov, 0, sizeof(unsigned int) * nrows, stream) != cudaSuccess) return check_launch("memset");
    const int nmaps_b = p.Ncam * p.Nscale;
    if (nmaps_b > 0) {
        cover_kernel<<<(unsigned)(p.B * nmaps_b), 256, 0, stream>>>(p.shape, p.start, p.sum_hw, nmaps_b, cov);
    }
    {
        long long grid = (nrows + 255) / 256;
        if (grid > (long long)dev.sm_count * 16) grid = (long long)dev.sm_count * 16;
        fill_uncovered_kernel<<<(unsigned)grid, 256, 0, stream>>>(cov, grad_feat, nrows, p.C, dev.status);
        if ((st = check_launch("msda_backward cover")) != MSDA_OK) return st;
    }
    if (nmaps_b == 0 || p.A * p.P == 0) {
        // no points: every covered row is zero
        if (nmaps_b > 0 && cudaMemsetAsync(grad_feat, 0, sizeof(float) * nrows * p.C, stream) != cudaSuccess)
            return check_launch("memset");
        return MSDA_OK;
    }

    // 3. cell sort of every map's points
    SortArgs sa;
    sa.shape = p.shape; sa.start = p.start; sa.loc = p.loc; sa.w = p.w; sa.w_t = p.w_t;
    sa.B = p.B; sa.sum_hw = p.sum_hw; sa.Ncam = p.Ncam; sa.Nscale = p.Nscale; sa.A = p.A; sa.P = p.P; sa.G = p.G;
    sa.cell_base = reinterpret_cast<int*>(base + L.cell_base);
    sa.cell_off = reinterpret_cast<int*>(base + L.cell_off);
    sa.scratch_cell = reinterpret_cast<int*>(base + L.sc);
    sa.scratch_pos = reinterpret_cast<int*>(base + L.spos);
    sa.rec_hdr = reinterpret_cast<int4*>(base + L.hdr);
    sa.rec_w = reinterpret_cast<float*>(base + L.recw);
    sa.cells_cap = L.cells_cap;
    sa.status = dev.status;
    cell_base_kernel<<<1, 1024, 0, stream>>>(sa);
    const size_t sort_smem = sizeof(int) * (kCgMaxCells + 1);
    if ((st = ensure_smem((const void*)cell_sort_kernel, sort_smem, dev)) != MSDA_OK) return st;
    cell_sort_kernel<<<(unsigned)(p.B * nmaps_b), 256, sort_smem, stream>>>(sa);
    if ((st = check_launch("msda_backward cell sort")) != MSDA_OK) return st;

    // 4. row gather
    RowArgs ra;
    ra.shape = p.shape; ra.start = p.start; ra.go = grad_out; ra.cell_base = sa.cell_base; ra.cell_off = sa.cell_off;
    ra.rec_hdr = sa.rec_hdr; ra.rec_w = sa.rec_w; ra.gfeat = grad_feat;
    ra.B = p.B; ra.sum_hw = p.sum_hw; ra.C = p.C; ra.Ncam = p.Ncam; ra.Nscale = p.Nscale; ra.A = p.A; ra.P = p.P;
    ra.G = p.G; ra.Cg = p.Cg; ra.cells_cap = L.cells_cap; ra.status = dev.status;
    const long long base_units = (long long)p.B * p.Ncam * p.G;
    ra.n_rr = pick_ranges(base_units, 1 << 20, dev.sm_count);
    ra.nunits = base_units * ra.n_rr;
    const size_t gsmem = sizeof(float) * (size_t)p.A * p.Cg;
    if ((st = ensure_smem((const void*)row_gather_kernel, gsmem, dev)) != MSDA_OK) return st;
    long long grid = ra.nunits;
    if (grid > (long long)dev.sm_count * 64) grid = (long long)dev.sm_count * 64;
    row_gather_kernel<<<(unsigned)grid, 512, gsmem, stream>>>(ra);
    return check_launch("msda_backward row gather");
}

// The first-wait poll limit of this file's staged kernels (msda_debug_set_wait_limit).
msda_status cg_set_wait_limit(long long polls) {
    if (polls < 0) polls = kSpinLimit;
    const cudaError_t e = cudaMemcpyToSymbol(g_first_wait_limit, &polls, sizeof(polls));
    return e == cudaSuccess ? MSDA_OK : fail(MSDA_ERR_CUDA, "msda_debug_set_wait_limit: %s", cudaGetErrorString(e));
}

}  // namespace msda
