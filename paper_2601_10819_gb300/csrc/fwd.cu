// MSDA forward kernels (sm_103a).
//
// The operator (arXiv 2601.10819, Sec. 3.2 and Sec. 5.3): for every anchor,
// keypoint p, camera k and scale s, bilinearly sample the projected
// location from the camera's map (zero padding), weight the sample by the
// per-group attention weight and sum everything into out[b, a, :].
//
// Mapping.  One block owns one anchor (b, a).  Its threads form "teams" of
// rt lanes; a team covers the anchor's whole channel row, each lane owning
// CPL = VEC * NV contiguous channels (VEC = 16 bytes of features), so every
// corner read is one 256-bit load (NV = 2, aligned) or NV 16-byte loads per
// lane and a team reads a whole feature row with coalesced, sector-aligned
// loads.  By default the block works in two stages per chunk of the anchor's
// point-scales (camera, keypoint, scale) in camera-major order: the threads
// cull and locate each point-scale once into a record in shared memory and
// list the in-view ones in order; the teams then take the list round-robin
// and only load and accumulate (accumulate_anchor_units).  The single-stage
// form (accumulate_anchor, tuning variant 4) deals (camera, keypoint) items
// to the teams and lets every lane locate the point itself.  Because all
// resident blocks walk the cameras in the same order, the maps being read at
// any moment belong to a few cameras, which keeps them in L2 (the operator
// reads each feature row about ten times).  The sampling locations of the
// anchor and the map table are staged in shared memory first; the weights
// are read only for points that are in view (a point whose bilinear
// footprint misses the map costs no weight or feature traffic).
//
// Accumulation is FP32 in registers in a fixed order; the teams' partial
// rows are summed in team order through shared memory, so a given launch
// configuration is bitwise reproducible.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "units.cuh"

namespace msda {

struct FwdArgs {
    const void* feat;
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* vis;  // visibility [B, A, Ncam] for the fused occlusion-aware form, or NULL
    void* out;
    int out_t;
    int B, sum_hw, C, Ncam, Nscale, A, P, G, Cg;
    int rt;
    int* status;
    uint4* zero;                   // msda_forward_train: grad_feat to clear (16-byte units), or NULL
    unsigned long long zero_n16;
    int wide;                      // a lane's two 16-byte chunks are 32-byte aligned: one 256-bit load
};

// Shared-memory carve-up of a forward block.
// units: entries of the two-stage form's point-scale list (0 for the other forms).
struct FwdSmem {
    size_t maps, box, vn, loc, part, list, total;
    __host__ __device__ FwdSmem(int nmaps, int P, int Ncam, int nteams, int C, int units = 0) {
        maps = 0;
        box = align16(sizeof(MapInfo) * (size_t)nmaps);
        vn = box + sizeof(float4) * (size_t)Ncam;
        loc = vn + align16(sizeof(float) * (size_t)Ncam);
        part = loc + align16(sizeof(float2) * (size_t)P * Ncam);
        list = part + align16(sizeof(float) * (size_t)nteams * C);
        total = list + unit_list_bytes((size_t)units);
    }
};

// Accumulate the items of one anchor dealt to this team.
//   fb: feat of batch element b, offset to the lane's first channel
//   wb: weights of the anchor, offset to the lane's group
// Items outside the camera's box are skipped with one test.  Per scale, the
// four corner rows are loaded (NV 16-byte chunks each; unpredicated when the
// cell is inside the map) and accumulated with packed FP32 FMAs.
// svn (optional): per-camera factor applied to every weight of the camera
// (the normalised visibility of the fused occlusion-aware form); a camera
// with factor 0 is skipped.
// Clearing a slice of another buffer alongside (training forward): the team
// handling item i also zeroes piece i of the block's slice [zlo, zhi) of
// `zero` (16-byte units, zchunk per item, lanes tl of rt), so the stores
// are spread evenly over the block's life.
struct ZeroSlice {
    uint4* ptr;
    unsigned long long lo, hi, chunk;
};

template <typename FT, typename WT, int NV>
__device__ __forceinline__ void accumulate_anchor(const FT* __restrict__ fb, const WT* __restrict__ wb,
                                                  const MapInfo* __restrict__ smap, const float4* __restrict__ sbox,
                                                  const float2* __restrict__ sloc, int C, int Ncam,
                                                  int Nscale, int P, int G, int team, int nteams,
                                                  float2* acc, const float* __restrict__ svn = nullptr,
                                                  const ZeroSlice* zs = nullptr, int tl = 0, int rt = 1) {
    constexpr int VEC = Elem<FT>::VEC;
    const int nitems = Ncam * P;
    for (int item = team; item < nitems; item += nteams) {
        if (zs) {
            const unsigned long long z0 = zs->lo + (unsigned long long)item * zs->chunk;
            const unsigned long long z1 = min(z0 + zs->chunk, zs->hi);
            for (unsigned long long j = z0 + tl; j < z1; j += rt) __stcs(zs->ptr + j, make_uint4(0u, 0u, 0u, 0u));
        }
        const int k = item / P;
        const int pp = item - k * P;
        const float2 uv = sloc[pp * Ncam + k];
        if (!in_box(uv, sbox[k])) continue;
        const float cam_scale = svn ? svn[k] : 1.0f;
        if (cam_scale == 0.0f) continue;
        const WT* wrow = wb + ((long long)pp * Ncam + k) * Nscale * G;
        const MapInfo* mrow = smap + k * Nscale;
        for (int s = 0; s < Nscale; ++s) {
            const MapInfo m = mrow[s];
            Cell c;
            if (m.W == 0 || !locate(uv.x, uv.y, m.H, m.W, c)) continue;
            const float wv = ldw(wrow + (long long)s * G) * cam_scale;
            const float ax = 1.0f - c.fx, ay = 1.0f - c.fy;
            const float2 w00 = make_float2(wv * (ax * ay), wv * (ax * ay));
            const float2 w01 = make_float2(wv * (c.fx * ay), wv * (c.fx * ay));
            const float2 w10 = make_float2(wv * (ax * c.fy), wv * (ax * c.fy));
            const float2 w11 = make_float2(wv * (c.fx * c.fy), wv * (c.fx * c.fy));
            const FT* p00 = fb + (long long)(m.start + c.y0 * m.W + c.x0) * C;
            const FT* p10 = p00 + (long long)m.W * C;
            uint4 q[4][NV];
            if (c.x0 >= 0 && c.x0 + 1 < m.W && c.y0 >= 0 && c.y0 + 1 < m.H) {
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    q[0][n] = ld16(p00 + n * VEC);
                    q[1][n] = ld16(p00 + C + n * VEC);
                    q[2][n] = ld16(p10 + n * VEC);
                    q[3][n] = ld16(p10 + C + n * VEC);
                }
            } else {
                const bool vx0 = c.x0 >= 0, vx1 = c.x0 + 1 < m.W;
                const bool vy0 = c.y0 >= 0, vy1 = c.y0 + 1 < m.H;
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    q[0][n] = (vy0 && vx0) ? ld16(p00 + n * VEC) : z;
                    q[1][n] = (vy0 && vx1) ? ld16(p00 + C + n * VEC) : z;
                    q[2][n] = (vy1 && vx0) ? ld16(p10 + n * VEC) : z;
                    q[3][n] = (vy1 && vx1) ? ld16(p10 + C + n * VEC) : z;
                }
            }
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                float2 f[4][VEC / 2];
#pragma unroll
                for (int cq = 0; cq < 4; ++cq) widen2(q[cq][n], f[cq], FT());
#pragma unroll
                for (int j = 0; j < VEC / 2; ++j) {
                    float2 a = acc[n * (VEC / 2) + j];
                    a = __ffma2_rn(w00, f[0][j], a);
                    a = __ffma2_rn(w01, f[1][j], a);
                    a = __ffma2_rn(w10, f[2][j], a);
                    a = __ffma2_rn(w11, f[3][j], a);
                    acc[n * (VEC / 2) + j] = a;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Two-stage form of accumulate_anchor (the default; variant 4 is the other).
// The anchor's point-scales (camera, keypoint, scale) are taken in chunks of
// kUnitsPerThread per thread: stage A culls each one and locates its cell
// once (instead of once in each of a team's lanes) and compacts the in-view
// ones, in order, into a list in shared memory; stage B deals the list
// round-robin to the teams, which only load and accumulate.  A team's sums run
// in increasing point-scale order, so the result is deterministic; the
// teams' shares differ from accumulate_anchor's, so the rounding does too.
// ---------------------------------------------------------------------------
template <typename FT, typename WT, int NV>
__device__ __forceinline__ void accumulate_anchor_units(const FT* __restrict__ fb, const WT* __restrict__ wb,
                                                        const MapInfo* __restrict__ smap,
                                                        const float4* __restrict__ sbox,
                                                        const float2* __restrict__ sloc, int C, int Ncam,
                                                        int Nscale, int P, int G, int team, int nteams,
                                                        float2* acc, const float* __restrict__ svn,
                                                        UnitRec* srec, short* slist, int* sscan,
                                                        const ZeroSlice* zs, bool wide = false) {
    constexpr int VEC = Elem<FT>::VEC;
    const int per_cam = P * Nscale;
    const int nunits = Ncam * per_cam;
    const int chunk = blockDim.x * kUnitsPerThread;
    const int nchunks = (nunits + chunk - 1) / chunk;
    unsigned long long zpiece = 0;
    if (zs) {
        if (nchunks == 0) {  // nothing to carry the clearing: do it at once
            for (unsigned long long j = zs->lo + threadIdx.x; j < zs->hi; j += blockDim.x)
                __stcs(zs->ptr + j, make_uint4(0u, 0u, 0u, 0u));
        } else {
            zpiece = (zs->hi - zs->lo + nchunks - 1) / nchunks;
        }
    }
    for (int ci = 0; ci < nchunks; ++ci) {
        const int u0 = ci * chunk;
        if (zs) {
            const unsigned long long z0 = min(zs->lo + (unsigned long long)ci * zpiece, zs->hi);
            const unsigned long long z1 = min(z0 + zpiece, zs->hi);
            for (unsigned long long j = z0 + threadIdx.x; j < z1; j += blockDim.x)
                __stcs(zs->ptr + j, make_uint4(0u, 0u, 0u, 0u));
        }
        // stage A: cull and locate this thread's kUnitsPerThread consecutive point-scales into its own entries
        // of the record array, then list the in-view ones, in order, by index
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
                    r.wf = ((((pp * Ncam + k) * Nscale) + sc) << 4) | (c.x0 >= 0 ? 1 : 0) |
                           (c.x0 + 1 < m.W ? 2 : 0) | (c.y0 >= 0 ? 4 : 0) | (c.y0 + 1 < m.H ? 8 : 0);
                    r.scale = cs;
                    srec[mine + i] = r;
                    vmask |= 1u << i;
                }
            }
        }
        int off = block_excl_scan(__popc(vmask), sscan, sscan + 8);
#pragma unroll
        for (int i = 0; i < kUnitsPerThread; ++i)
            if (vmask & (1u << i)) slist[off++] = (short)(mine + i);
        __syncthreads();
        const int total = sscan[8];
        // stage B: the teams take the list round-robin
        for (int q = team; q < total; q += nteams) {
            const UnitRec r = srec[slist[q]];
            const float wv = ldw(wb + (long long)(r.wf >> 4) * G) * r.scale;
            const float ax = 1.0f - r.fx, ay = 1.0f - r.fy;
            const float2 w00 = make_float2(wv * (ax * ay), wv * (ax * ay));
            const float2 w01 = make_float2(wv * (r.fx * ay), wv * (r.fx * ay));
            const float2 w10 = make_float2(wv * (ax * r.fy), wv * (ax * r.fy));
            const float2 w11 = make_float2(wv * (r.fx * r.fy), wv * (r.fx * r.fy));
            const FT* p00 = fb + (long long)r.row00 * C;
            const FT* p10 = p00 + (long long)r.W * C;
            uint4 q4[4][NV];
            if (NV == 2 && wide && (r.wf & 15) == 15) {
                ld32(p00, q4[0][0], q4[0][NV - 1]);
                ld32(p00 + C, q4[1][0], q4[1][NV - 1]);
                ld32(p10, q4[2][0], q4[2][NV - 1]);
                ld32(p10 + C, q4[3][0], q4[3][NV - 1]);
            } else if ((r.wf & 15) == 15) {
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    q4[0][n] = ld16(p00 + n * VEC);
                    q4[1][n] = ld16(p00 + C + n * VEC);
                    q4[2][n] = ld16(p10 + n * VEC);
                    q4[3][n] = ld16(p10 + C + n * VEC);
                }
            } else {
                const bool vx0 = r.wf & 1, vx1 = r.wf & 2, vy0 = r.wf & 4, vy1 = r.wf & 8;
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    q4[0][n] = (vy0 && vx0) ? ld16(p00 + n * VEC) : z;
                    q4[1][n] = (vy0 && vx1) ? ld16(p00 + C + n * VEC) : z;
                    q4[2][n] = (vy1 && vx0) ? ld16(p10 + n * VEC) : z;
                    q4[3][n] = (vy1 && vx1) ? ld16(p10 + C + n * VEC) : z;
                }
            }
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                float2 f[4][VEC / 2];
#pragma unroll
                for (int cq = 0; cq < 4; ++cq) widen2(q4[cq][n], f[cq], FT());
#pragma unroll
                for (int j = 0; j < VEC / 2; ++j) {
                    float2 a = acc[n * (VEC / 2) + j];
                    a = __ffma2_rn(w00, f[0][j], a);
                    a = __ffma2_rn(w01, f[1][j], a);
                    a = __ffma2_rn(w10, f[2][j], a);
                    a = __ffma2_rn(w11, f[3][j], a);
                    acc[n * (VEC / 2) + j] = a;
                }
            }
        }
        __syncthreads();  // the list is rebuilt for the next chunk
    }
}

// Sum the teams' partial rows in team order and write out[row] (n = C values).
__device__ __forceinline__ void reduce_and_store(const float* spart, int nteams, int C, void* out,
                                                 int out_t, long long orow) {
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float v = spart[c];
        for (int t = 1; t < nteams; ++t) v += spart[(size_t)t * C + c];
        const long long o = orow * C + c;
        if (out_t == MSDA_F32)
            store_out(reinterpret_cast<float*>(out) + o, v);
        else if (out_t == MSDA_BF16)
            store_out(reinterpret_cast<__nv_bfloat16*>(out) + o, v);
        else
            store_out(reinterpret_cast<__half*>(out) + o, v);
    }
}

// One block per anchor.  The launch is sized so that, on the benchmark
// shapes, every anchor's block is resident at once: then all blocks walk the
// cameras in the same order together and each camera's maps are read from
// HBM about once.
template <typename FT, typename WT, int NV, bool CLEAR, bool UNITS>
__global__ void __launch_bounds__(256, NV == 2 ? 3 : (NV == 1 ? 4 : 1)) fwd_anchor_kernel(const FwdArgs p) {
    constexpr int CPL = Elem<FT>::VEC * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nmaps = p.Ncam * p.Nscale;
    const int tpw = 32 / p.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const FwdSmem lay(nmaps, p.P, p.Ncam, nteams, p.C, UNITS ? (int)blockDim.x * kUnitsPerThread : 0);
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem + lay.maps);
    float4* sbox = reinterpret_cast<float4*>(smem + lay.box);
    float* svn = reinterpret_cast<float*>(smem + lay.vn);
    float2* sloc = reinterpret_cast<float2*>(smem + lay.loc);
    float* spart = reinterpret_cast<float*>(smem + lay.part);

    const long long ba = blockIdx.x;
    if (p.vis) {
        // occlusion-aware fusion (Sec. 3.2, Eq. 2): camera k's weights scale by v_k / sum_j v_j
        const float* vrow = p.vis + ba * p.Ncam;
        if (threadIdx.x < 32) {
            float sum = 0.0f;
            for (int k = threadIdx.x; k < p.Ncam; k += 32) sum += __ldg(vrow + k);
            for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
            const float inv = sum != 0.0f ? 1.0f / sum : 0.0f;
            for (int k = threadIdx.x; k < p.Ncam; k += 32) svn[k] = __ldg(vrow + k) * inv;
        }
    }
    const int b = (int)(ba / p.A);
    for (int i = threadIdx.x; i < nmaps; i += blockDim.x)
        smap[i] = load_map(p.shape, p.start, i, p.sum_hw, p.status);
    const float2* gloc = reinterpret_cast<const float2*>(p.loc) + ba * (long long)(p.P * p.Ncam);
    for (int i = threadIdx.x; i < p.P * p.Ncam; i += blockDim.x) sloc[i] = __ldg(gloc + i);
    __syncthreads();
    for (int k = threadIdx.x; k < p.Ncam; k += blockDim.x) sbox[k] = camera_box(smap + k * p.Nscale, p.Nscale);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int team = (threadIdx.x >> 5) * tpw + lane / p.rt;
    const int c0 = (lane & (p.rt - 1)) * CPL;
    const int g = c0 / p.Cg;
    const FT* fb = reinterpret_cast<const FT*>(p.feat) + (long long)b * p.sum_hw * p.C + c0;
    const WT* wb = reinterpret_cast<const WT*>(p.w) + ba * ((long long)p.P * p.Ncam * p.Nscale * p.G) + g;

    float2 acc[CPL / 2];
#pragma unroll
    for (int j = 0; j < CPL / 2; ++j) acc[j] = make_float2(0.0f, 0.0f);
    if constexpr (CLEAR) {
        // training forward: this block's slice of grad_feat, one piece per item (the host guarantees items);
        // the slice bounds live in shared memory, not in registers held across the item loop
        __shared__ ZeroSlice s_zs;
        if (threadIdx.x == 0) {
            const unsigned long long per = (p.zero_n16 + gridDim.x - 1) / gridDim.x;
            s_zs.ptr = p.zero;
            s_zs.lo = min((unsigned long long)blockIdx.x * per, p.zero_n16);
            s_zs.hi = min(s_zs.lo + per, p.zero_n16);
            const unsigned long long nitems = (unsigned long long)p.Ncam * p.P;
            s_zs.chunk = (s_zs.hi - s_zs.lo + nitems - 1) / nitems;
        }
        __syncthreads();
        if constexpr (UNITS)
            accumulate_anchor_units<FT, WT, NV>(fb, wb, smap, sbox, sloc, p.C, p.Ncam, p.Nscale, p.P, p.G, team,
                                                nteams, acc, p.vis ? svn : nullptr,
                                                reinterpret_cast<UnitRec*>(smem + lay.list),
                                                reinterpret_cast<short*>(smem + lay.list + 24 * (size_t)blockDim.x *
                                                                                       kUnitsPerThread),
                                                reinterpret_cast<int*>(smem + lay.list + align16(26 * (size_t)blockDim.x *
                                                                                                 kUnitsPerThread)),
                                                &s_zs, p.wide != 0);
        else
            accumulate_anchor<FT, WT, NV>(fb, wb, smap, sbox, sloc, p.C, p.Ncam, p.Nscale, p.P, p.G, team, nteams,
                                          acc, p.vis ? svn : nullptr, &s_zs, lane & (p.rt - 1), p.rt);
    } else {
        if constexpr (UNITS)
            accumulate_anchor_units<FT, WT, NV>(fb, wb, smap, sbox, sloc, p.C, p.Ncam, p.Nscale, p.P, p.G, team,
                                                nteams, acc, p.vis ? svn : nullptr,
                                                reinterpret_cast<UnitRec*>(smem + lay.list),
                                                reinterpret_cast<short*>(smem + lay.list + 24 * (size_t)blockDim.x *
                                                                                       kUnitsPerThread),
                                                reinterpret_cast<int*>(smem + lay.list + align16(26 * (size_t)blockDim.x *
                                                                                                 kUnitsPerThread)),
                                                nullptr, p.wide != 0);
        else
            accumulate_anchor<FT, WT, NV>(fb, wb, smap, sbox, sloc, p.C, p.Ncam, p.Nscale, p.P, p.G, team, nteams,
                                          acc, p.vis ? svn : nullptr);
    }

    float* mine = spart + (size_t)team * p.C + c0;
#pragma unroll
    for (int j = 0; j < CPL / 2; j += 2)
        *reinterpret_cast<float4*>(mine + 2 * j) = make_float4(acc[j].x, acc[j].y, acc[j + 1].x, acc[j + 1].y);
    __syncthreads();
    reduce_and_store(spart, nteams, p.C, p.out, p.out_t, ba);
}

// ---------------------------------------------------------------------------
// Half2-accumulating forward (the paper's FP16 plugin arithmetic, Sec. 5.3):
// FP16 features and weights, two channels per instruction, and the weighted
// sum kept in half2 registers until the anchor's partial rows are written.
// The teams' partial rows are then added in FP32.  Same mapping, cull and
// loads as the FP32-accumulating kernel; only the arithmetic differs.
// ---------------------------------------------------------------------------
template <int NV>
__global__ void __launch_bounds__(256) fwd_anchor_h2_kernel(const FwdArgs p) {
    constexpr int VEC = 8;
    constexpr int CPL = VEC * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nmaps = p.Ncam * p.Nscale;
    const int tpw = 32 / p.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const FwdSmem lay(nmaps, p.P, p.Ncam, nteams, p.C);
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem + lay.maps);
    float4* sbox = reinterpret_cast<float4*>(smem + lay.box);
    float2* sloc = reinterpret_cast<float2*>(smem + lay.loc);
    float* spart = reinterpret_cast<float*>(smem + lay.part);
    const long long ba = blockIdx.x;
    const int b = (int)(ba / p.A);
    for (int i = threadIdx.x; i < nmaps; i += blockDim.x) smap[i] = load_map(p.shape, p.start, i, p.sum_hw, p.status);
    const float2* gloc = reinterpret_cast<const float2*>(p.loc) + ba * (long long)(p.P * p.Ncam);
    for (int i = threadIdx.x; i < p.P * p.Ncam; i += blockDim.x) sloc[i] = __ldg(gloc + i);
    __syncthreads();
    for (int k = threadIdx.x; k < p.Ncam; k += blockDim.x) sbox[k] = camera_box(smap + k * p.Nscale, p.Nscale);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int team = (threadIdx.x >> 5) * tpw + lane / p.rt;
    const int c0 = (lane & (p.rt - 1)) * CPL;
    const int g = c0 / p.Cg;
    const __half* fb = reinterpret_cast<const __half*>(p.feat) + (long long)b * p.sum_hw * p.C + c0;
    const __half* wb = reinterpret_cast<const __half*>(p.w) + ba * ((long long)p.P * p.Ncam * p.Nscale * p.G) + g;
    __half2 acc[CPL / 2];
#pragma unroll
    for (int j = 0; j < CPL / 2; ++j) acc[j] = __float2half2_rn(0.0f);
    const int nitems = p.Ncam * p.P;
    for (int item = team; item < nitems; item += nteams) {
        const int k = item / p.P;
        const int pp = item - k * p.P;
        const float2 uv = sloc[pp * p.Ncam + k];
        if (!in_box(uv, sbox[k])) continue;
        const __half* wrow = wb + ((long long)pp * p.Ncam + k) * p.Nscale * p.G;
        const MapInfo* mrow = smap + k * p.Nscale;
        for (int s = 0; s < p.Nscale; ++s) {
            const MapInfo m = mrow[s];
            Cell c;
            if (m.W == 0 || !locate(uv.x, uv.y, m.H, m.W, c)) continue;
            const float wv = __half2float(__ldg(wrow + (long long)s * p.G));
            const float ax = 1.0f - c.fx, ay = 1.0f - c.fy;
            const __half2 w00 = __float2half2_rn(wv * ax * ay), w01 = __float2half2_rn(wv * c.fx * ay);
            const __half2 w10 = __float2half2_rn(wv * ax * c.fy), w11 = __float2half2_rn(wv * c.fx * c.fy);
            const bool vx0 = c.x0 >= 0, vx1 = c.x0 + 1 < m.W, vy0 = c.y0 >= 0, vy1 = c.y0 + 1 < m.H;
            const __half* p00 = fb + (long long)(m.start + c.y0 * m.W + c.x0) * p.C;
            const __half* p10 = p00 + (long long)m.W * p.C;
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const uint4 q0 = (vy0 && vx0) ? ld16(p00 + n * VEC) : z;
                const uint4 q1 = (vy0 && vx1) ? ld16(p00 + p.C + n * VEC) : z;
                const uint4 q2 = (vy1 && vx0) ? ld16(p10 + n * VEC) : z;
                const uint4 q3 = (vy1 && vx1) ? ld16(p10 + p.C + n * VEC) : z;
                const __half2* h0 = reinterpret_cast<const __half2*>(&q0);
                const __half2* h1 = reinterpret_cast<const __half2*>(&q1);
                const __half2* h2 = reinterpret_cast<const __half2*>(&q2);
                const __half2* h3 = reinterpret_cast<const __half2*>(&q3);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    __half2 a = acc[n * 4 + j];
                    a = __hfma2(w00, h0[j], a);
                    a = __hfma2(w01, h1[j], a);
                    a = __hfma2(w10, h2[j], a);
                    a = __hfma2(w11, h3[j], a);
                    acc[n * 4 + j] = a;
                }
            }
        }
    }
    float* mine = spart + (size_t)team * p.C + c0;
#pragma unroll
    for (int j = 0; j < CPL / 2; ++j) {
        const float2 f = __half22float2(acc[j]);
        mine[2 * j] = f.x;
        mine[2 * j + 1] = f.y;
    }
    __syncthreads();
    reduce_and_store(spart, nteams, p.C, p.out, p.out_t, ba);
}

// ---------------------------------------------------------------------------
// Batched serving: one persistent launch over all scenes' anchors.
//
// Work units are anchors, numbered scene by scene (unit_begin).  Each
// resident block pulls the next unit from an atomic counter, so large and
// small scenes interleave and the tail stays short.  The scene of a unit is
// found by binary search over unit_begin.  When a block finishes the last
// anchor of a scene (per-scene counter), it stamps %globaltimer into
// done_ns[scene + 1]; block 0 stamps the start into done_ns[0].  No block
// waits on another.
// ---------------------------------------------------------------------------
struct BatchedArgs {
    const msda_scene* scenes;
    int num_scenes, total;
    int max_ncam, Nscale, C, P, G, Cg, rt, out_t;
    unsigned int* counters;  // [0] = next unit, [1 + i] = finished anchors of scene i
    uint64_t* done_ns;
    int* status;
};

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename FT, typename WT, int NV>
__global__ void __launch_bounds__(256) fwd_batched_kernel(const BatchedArgs p) {
    constexpr int CPL = Elem<FT>::VEC * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tpw = 32 / p.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const FwdSmem lay(p.max_ncam * p.Nscale, p.P, p.max_ncam, nteams, p.C, (int)blockDim.x * kUnitsPerThread);
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem + lay.maps);
    float4* sbox = reinterpret_cast<float4*>(smem + lay.box);
    float2* sloc = reinterpret_cast<float2*>(smem + lay.loc);
    float* spart = reinterpret_cast<float*>(smem + lay.part);
    __shared__ int s_unit, s_scene;

    if (blockIdx.x == 0 && threadIdx.x == 0 && p.done_ns) p.done_ns[0] = globaltimer();
    const int lane = threadIdx.x & 31;
    const int team = (threadIdx.x >> 5) * tpw + lane / p.rt;
    const int c0 = (lane & (p.rt - 1)) * CPL;
    const int g = c0 / p.Cg;
    int cur_scene = -1;

    for (;;) {
        if (threadIdx.x == 0) {
            const int u = (int)atomicAdd(p.counters, 1u);
            int sc = -1;
            if (u < p.total) {
                int lo = 0, hi = p.num_scenes - 1;  // last scene with unit_begin <= u
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.scenes[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
                }
                sc = lo;
            }
            s_unit = u;
            s_scene = sc;
        }
        __syncthreads();
        const int u = s_unit, sc = s_scene;
        if (u >= p.total) break;
        const msda_scene S = p.scenes[sc];
        const int a = u - S.unit_begin;
        const int ncam = S.Ncam;
        bool bad = (ncam > p.max_ncam || ncam < 0 || a >= S.A);
        if (bad) {
            if (threadIdx.x == 0) raise_status(p.status, MSDA_ERR_OUT_OF_RANGE);
        } else {
            if (sc != cur_scene) {
                for (int i = threadIdx.x; i < ncam * p.Nscale; i += blockDim.x)
                    smap[i] = load_map(S.spatial_shape, S.scale_start_index, i, S.sum_hw, p.status);
            }
            const float2* gloc = reinterpret_cast<const float2*>(S.sampling_location) + (long long)a * (p.P * ncam);
            for (int i = threadIdx.x; i < p.P * ncam; i += blockDim.x) sloc[i] = __ldg(gloc + i);
            __syncthreads();
            if (sc != cur_scene)
                for (int k = threadIdx.x; k < ncam; k += blockDim.x) sbox[k] = camera_box(smap + k * p.Nscale, p.Nscale);
            __syncthreads();
            const FT* fb = reinterpret_cast<const FT*>(S.feat) + c0;
            const WT* wb = reinterpret_cast<const WT*>(S.weights) + (long long)a * ((long long)p.P * ncam * p.Nscale * p.G) + g;
            float2 acc[CPL / 2];
#pragma unroll
            for (int j = 0; j < CPL / 2; ++j) acc[j] = make_float2(0.0f, 0.0f);
            const bool wide = NV == 2 && ((reinterpret_cast<uintptr_t>(S.feat) & 31) == 0) &&
                              ((size_t)p.C * sizeof(FT)) % 32 == 0;  // 256-bit loads for this scene
            accumulate_anchor_units<FT, WT, NV>(
                fb, wb, smap, sbox, sloc, p.C, ncam, p.Nscale, p.P, p.G, team, nteams, acc, nullptr,
                reinterpret_cast<UnitRec*>(smem + lay.list),
                reinterpret_cast<short*>(smem + lay.list + 24 * (size_t)blockDim.x * kUnitsPerThread),
                reinterpret_cast<int*>(smem + lay.list + align16(26 * (size_t)blockDim.x * kUnitsPerThread)), nullptr,
                wide);
            float* mine = spart + (size_t)team * p.C + c0;
#pragma unroll
            for (int j = 0; j < CPL / 2; j += 2)
                *reinterpret_cast<float4*>(mine + 2 * j) = make_float4(acc[j].x, acc[j].y, acc[j + 1].x, acc[j + 1].y);
            __syncthreads();
            reduce_and_store(spart, nteams, p.C, S.out, p.out_t, a);
            cur_scene = sc;
        }
        __syncthreads();  // partial rows, staged tables and s_unit are reused next round
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned int done = atomicAdd(p.counters + 1 + sc, 1u) + 1u;
            if (!bad && done == (unsigned int)S.A && p.done_ns) p.done_ns[1 + sc] = globaltimer();
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using FwdKernel = void (*)(const FwdArgs);
using BatchedKernel = void (*)(const BatchedArgs);

template <typename FT, typename WT, bool CLEAR, bool UNITS>
static FwdKernel fwd_pick_nv(int nv) {
    switch (nv) {
        case 1: return fwd_anchor_kernel<FT, WT, 1, CLEAR, UNITS>;
        case 2: return fwd_anchor_kernel<FT, WT, 2, CLEAR, UNITS>;
        case 4: return fwd_anchor_kernel<FT, WT, 4, CLEAR, UNITS>;
    }
    return nullptr;
}

template <typename FT, typename WT>
static BatchedKernel batched_pick_nv(int nv) {
    switch (nv) {
        case 1: return fwd_batched_kernel<FT, WT, 1>;
        case 2: return fwd_batched_kernel<FT, WT, 2>;
        case 4: return fwd_batched_kernel<FT, WT, 4>;
    }
    return nullptr;
}

// Supported (feature, weight) dtype pairs: weights in FP32 or in the feature dtype.
template <bool CLEAR, bool UNITS>
static FwdKernel fwd_kernel_for(msda_dtype ft, msda_dtype wt, int nv) {
    if (ft == MSDA_F32 && wt == MSDA_F32) return fwd_pick_nv<float, float, CLEAR, UNITS>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_BF16) return fwd_pick_nv<__nv_bfloat16, __nv_bfloat16, CLEAR, UNITS>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_F32) return fwd_pick_nv<__nv_bfloat16, float, CLEAR, UNITS>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F16) return fwd_pick_nv<__half, __half, CLEAR, UNITS>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F32) return fwd_pick_nv<__half, float, CLEAR, UNITS>(nv);
    return nullptr;
}

static BatchedKernel batched_kernel_for(msda_dtype ft, msda_dtype wt, int nv) {
    if (ft == MSDA_F32 && wt == MSDA_F32) return batched_pick_nv<float, float>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_BF16) return batched_pick_nv<__nv_bfloat16, __nv_bfloat16>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_F32) return batched_pick_nv<__nv_bfloat16, float>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F16) return batched_pick_nv<__half, __half>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F32) return batched_pick_nv<__half, float>(nv);
    return nullptr;
}

msda_status launch_forward(const Problem& p, void* out, msda_dtype out_t, int warps,
                           cudaStream_t stream, const float* vis, bool half_acc, float* clear, bool units) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    if (half_acc && (p.feat_t != MSDA_F16 || p.w_t != MSDA_F16 || vis))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward: half2 accumulation needs FP16 features and weights");
    const long long nblocks = (long long)p.B * p.A;
    const size_t clear_bytes = sizeof(float) * (size_t)p.B * p.sum_hw * p.C;
    if (clear && (clear_bytes == 0 || nblocks == 0 || (long long)p.Ncam * p.P == 0 || half_acc)) {
        // no items to carry the clearing (or the half2 kernel, which does not clear): a plain memset
        if (clear_bytes && cudaMemsetAsync(clear, 0, clear_bytes, stream) != cudaSuccess)
            return check_launch("msda_forward_train");
        clear = nullptr;
    }
    // the clearing kernel is chosen only when `clear` is still set, so its slice pointer is never NULL
    if ((long long)p.Ncam * p.P * p.Nscale >= (1ll << 26)) units = false;  // the unit index is a 32-bit int
    FwdKernel k = clear ? (units ? fwd_kernel_for<true, true>(p.feat_t, p.w_t, p.nv)
                                 : fwd_kernel_for<true, false>(p.feat_t, p.w_t, p.nv))
                        : (units ? fwd_kernel_for<false, true>(p.feat_t, p.w_t, p.nv)
                                 : fwd_kernel_for<false, false>(p.feat_t, p.w_t, p.nv));
    if (half_acc) k = p.nv == 1 ? fwd_anchor_h2_kernel<1> : p.nv == 2 ? fwd_anchor_h2_kernel<2> : fwd_anchor_h2_kernel<4>;
    if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward: unsupported feature/weight dtype pair");
    if (nblocks == 0) return MSDA_OK;
    if (nblocks > 0x7fffffffLL) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward: B*A too large");
    const int nteams = warps * (32 / p.rt);
    const FwdSmem lay(p.Ncam * p.Nscale, p.P, p.Ncam, nteams, p.C, units && !half_acc ? warps * 32 * kUnitsPerThread : 0);
    st = ensure_smem((const void*)k, lay.total, dev);
    if (st != MSDA_OK) return st;
    FwdArgs a;
    a.feat = p.feat; a.shape = p.shape; a.start = p.start; a.loc = p.loc; a.w = p.w; a.vis = vis;
    a.out = out; a.out_t = out_t;
    a.B = p.B; a.sum_hw = p.sum_hw; a.C = p.C; a.Ncam = p.Ncam; a.Nscale = p.Nscale;
    a.A = p.A; a.P = p.P; a.G = p.G; a.Cg = p.Cg; a.rt = p.rt; a.status = dev.status;
    a.zero = reinterpret_cast<uint4*>(clear);
    a.zero_n16 = clear ? clear_bytes / 16 : 0;
    // 256-bit loads need every lane's 32 bytes aligned: the base, the row pitch and the lane pitch
    const size_t esz = (size_t)dtype_size(p.feat_t);
    a.wide = (p.nv == 2 && ((uintptr_t)p.feat % 32) == 0 && ((size_t)p.C * esz) % 32 == 0 &&
              ((size_t)p.sum_hw * p.C * esz) % 32 == 0) ? 1 : 0;
    k<<<(unsigned)nblocks, warps * 32, lay.total, stream>>>(a);
    return check_launch("msda_forward");
}

size_t batched_workspace(int num_scenes) { return align_up(sizeof(unsigned int) * (size_t)(num_scenes + 1), 256); }

msda_status launch_forward_batched(const msda_scene* scenes, int num_scenes, int total_anchors,
                                   int max_ncam, int Nscale, int C, int P, int G, msda_dtype ft,
                                   msda_dtype wt, msda_dtype ot, void* ws, size_t ws_bytes,
                                   uint64_t* done_ns, int warps, int blocks_per_sm, int vec,
                                   cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    int nv, rt;
    if (!pick_split_pref(C, G, ft, vec, &nv, &rt))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: no lane split for C=%d G=%d", C, G);
    BatchedKernel k = batched_kernel_for(ft, wt, nv);
    if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: unsupported dtype pair");
    const size_t need = batched_workspace(num_scenes);
    if (!ws || ws_bytes < need)
        return fail(MSDA_ERR_WORKSPACE, "msda_forward_batched: workspace needs %zu bytes", need);
    const int nteams = warps * (32 / rt);
    const FwdSmem lay(max_ncam * Nscale, P, max_ncam, nteams, C, warps * 32 * kUnitsPerThread);
    st = ensure_smem((const void*)k, lay.total, dev);
    if (st != MSDA_OK) return st;
    if (cudaMemsetAsync(ws, 0, need, stream) != cudaSuccess) return check_launch("msda_forward_batched memset");
    if (total_anchors == 0) return MSDA_OK;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, warps * 32, lay.total) != cudaSuccess || occ < 1)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_forward_batched: kernel does not fit on an SM");
    const int per_sm = blocks_per_sm > 0 ? (blocks_per_sm < occ ? blocks_per_sm : occ) : occ;
    long long grid = (long long)per_sm * dev.sm_count;
    if (grid > total_anchors) grid = total_anchors;
    BatchedArgs a;
    a.scenes = scenes; a.num_scenes = num_scenes; a.total = total_anchors;
    a.max_ncam = max_ncam; a.Nscale = Nscale; a.C = C; a.P = P; a.G = G; a.Cg = C / G;
    a.rt = rt; a.out_t = ot; a.counters = reinterpret_cast<unsigned int*>(ws);
    a.done_ns = done_ns; a.status = dev.status;
    k<<<(unsigned)grid, warps * 32, lay.total, stream>>>(a);
    return check_launch("msda_forward_batched");
}

// ---------------------------------------------------------------------------
// Allocation-free batched forward.
//
// Some callers cannot allocate device memory at the point where they launch
// work: a plugin's enqueue inside an inference engine, a real-time serving
// loop with a fixed memory budget, or a plain C host program that links only
// this library and has no device allocator of its own.  For them the batched
// forward's scratch (one work counter plus one finished-anchor counter per
// scene) lives in this file-scope device array instead of a caller workspace.
// Every GPU that loads the library holds the array until the process exits.
// Host code cannot use the array's name as a device address, so its address
// is looked up once per device (the device being current) with
// cudaGetSymbolAddress and passed to the kernel.  The counters are cleared by
// every call; calls share them, so two calls that overlap on the GPU (on
// different streams without ordering) race and give wrong results.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxScenes = 1024;
// Sized from the batched forward's own workspace rule (one counter per scene plus the work counter, rounded
// up to 256 bytes), so every scene count up to the limit passes its workspace check.
constexpr size_t kNoAllocScratchBytes = ((sizeof(unsigned int) * (kNoAllocMaxScenes + 1) + 255) / 256) * 256;
static __device__ __align__(256) unsigned int g_batched_noalloc_scratch[kNoAllocScratchBytes / sizeof(unsigned int)];

int batched_noalloc_max_scenes() { return kNoAllocMaxScenes; }

msda_status launch_forward_batched_noalloc(const msda_scene* scenes, int num_scenes, int total_anchors,
                                           int max_ncam, int Nscale, int C, int P, int G, msda_dtype ft,
                                           msda_dtype wt, msda_dtype ot, uint64_t* done_ns, int warps,
                                           int blocks_per_sm, int vec, cudaStream_t stream) {
    if (num_scenes > kNoAllocMaxScenes)
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched_noalloc: %d scenes exceed the built-in limit of %d",
                    num_scenes, kNoAllocMaxScenes);
    static std::mutex mu;
    static void* addr[128];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MSDA_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(MSDA_ERR_UNSUPPORTED, "device index %d", dev);
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!addr[dev]) {
            e = cudaGetSymbolAddress(&addr[dev], g_batched_noalloc_scratch);
            if (e != cudaSuccess) {
                addr[dev] = nullptr;
                return fail(MSDA_ERR_CUDA, "msda_forward_batched_noalloc set-up: %s", cudaGetErrorString(e));
            }
        }
        scratch = addr[dev];
    }
    if (batched_workspace(num_scenes) > sizeof(g_batched_noalloc_scratch))
        return fail(MSDA_ERR_INVALID_ARG, "msda_forward_batched_noalloc: %d scenes exceed the built-in limit of %d",
                    num_scenes, kNoAllocMaxScenes);
    return launch_forward_batched(scenes, num_scenes, total_anchors, max_ncam, Nscale, C, P, G, ft, wt, ot,
                                  scratch, sizeof(g_batched_noalloc_scratch), done_ns, warps, blocks_per_sm, vec,
                                  stream);
}

}  // namespace msda
