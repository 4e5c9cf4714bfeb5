// MSDA backward, location and weight gradients, one block per anchor (sm_103a).
//
// The deterministic backward takes dloc and dw from this kernel (its feature
// gradient comes from the sort-and-reduce path of det.cu).  The block lists
// its anchor's in-view point-scales once (units.cuh) and deals them to teams
// of rt lanes, each lane holding its slice of the anchor's grad_out row in
// registers.  For a point-scale the team dots the four corner rows with
// grad_out (d_q, per lane over its channels) and forms, with the bilinear
// weights omega_q and the lane's group weight w_g:
//   dw[point-scale, g] = sum over the group's lanes of sum_q omega_q d_q
//   du_s = W_s * sum over the team of w_g (ay (d01 - d00) + fy (d11 - d10))
//   dv_s = H_s * sum over the team of w_g (ax (d10 - d00) + fx (d11 - d01))
// (the exact adjoint of the forward's bilinear sample, as in bwd.cu).  dw is
// stored at once; the two team sums wait in shared memory and dloc of a point
// is their sum, scaled by W_s and H_s, in scale order at the end.  A
// point-scale that is not listed gets dw = 0, a point with no listed scale
// dloc = 0.  Every sum has a fixed order, so the result is bitwise
// reproducible.  An anchor whose locations and sums do not fit in shared
// memory falls back to the per-point kernel of bwd.cu without its scatter.
#include "common.cuh"
#include "internal.h"
#include "units.cuh"

namespace msda {

struct LocWArgs {
    const void* feat;
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* go;
    float* gloc;
    float* gw;
    int B, sum_hw, C, Ncam, Nscale, A, P, G, Cg;
    int rt;
    int wide;  // 256-bit corner loads (NV = 2, 32-byte aligned rows)
    int* status;
};

// Shared memory: map table, camera boxes, locations, per point-scale (du, dv), point-scale list.
struct LocWSmem {
    size_t maps, box, loc, uv, list, total;
    __host__ __device__ LocWSmem(int nmaps, int P, int Ncam, int Nscale, int units) {
        maps = 0;
        box = align16(sizeof(MapInfo) * (size_t)nmaps);
        loc = box + sizeof(float4) * (size_t)Ncam;
        uv = loc + align16(sizeof(float2) * (size_t)P * Ncam);
        list = uv + align16(sizeof(float2) * (size_t)P * Ncam * Nscale);
        total = list + unit_list_bytes((size_t)units);
    }
};

// Sums over `width` lanes (a power of two up to 32), two values at once: the steps are unrolled, so the two
// chains of shuffles interleave.  The steps run from the widest down, the same order as a loop over
// off = width/2, ..., 1, so the sums are bitwise those of one value at a time.
__device__ __forceinline__ void team_sum2_lw(float& a, float& b, unsigned mask, int width) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        if (off < width) {
            const float ta = __shfl_xor_sync(mask, a, off), tb = __shfl_xor_sync(mask, b, off);
            a += ta;
            b += tb;
        }
    }
}

__device__ __forceinline__ float team_sum_lw(float v, unsigned mask, int width) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        if (off < width) v += __shfl_xor_sync(mask, v, off);
    return v;
}

template <typename FT, typename WT, int NV>
__global__ void __launch_bounds__(256, NV == 2 ? 3 : (NV == 1 ? 4 : 2)) bwd_locw_kernel(const LocWArgs p) {
    constexpr int VEC = Elem<FT>::VEC;
    constexpr int CPL = VEC * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nmaps = p.Ncam * p.Nscale;
    const int per_point = p.P * p.Ncam;
    const int npts = per_point * p.Nscale;
    const LocWSmem lay(nmaps, p.P, p.Ncam, p.Nscale, (int)blockDim.x * kUnitsPerThread);
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem + lay.maps);
    float4* sbox = reinterpret_cast<float4*>(smem + lay.box);
    float2* sloc = reinterpret_cast<float2*>(smem + lay.loc);
    float2* suv = reinterpret_cast<float2*>(smem + lay.uv);
    const UnitList ul(smem + lay.list, (int)blockDim.x * kUnitsPerThread);

    const long long ba = blockIdx.x;
    const int b = (int)(ba / p.A);
    for (int i = threadIdx.x; i < nmaps; i += blockDim.x) smap[i] = load_map(p.shape, p.start, i, p.sum_hw, p.status);
    const float2* gl = reinterpret_cast<const float2*>(p.loc) + ba * (long long)per_point;
    for (int i = threadIdx.x; i < per_point; i += blockDim.x) sloc[i] = __ldg(gl + i);
    for (int i = threadIdx.x; i < npts; i += blockDim.x) suv[i] = make_float2(0.0f, 0.0f);
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
    const int c0 = tl * CPL;
    const int g = c0 / p.Cg;
    const int lg = p.Cg / CPL;  // lanes per group
    const FT* fb = reinterpret_cast<const FT*>(p.feat) + (long long)b * p.sum_hw * p.C + c0;
    const WT* wb = reinterpret_cast<const WT*>(p.w) + ba * (long long)npts * p.G;
    float* gwb = p.gw + ba * (long long)npts * p.G;
    float2 go[CPL / 2];
#pragma unroll
    for (int j = 0; j < CPL / 4; ++j) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p.go + ba * p.C + c0) + j);
        go[2 * j] = make_float2(t.x, t.y);
        go[2 * j + 1] = make_float2(t.z, t.w);
    }

    const int chunk = blockDim.x * kUnitsPerThread;
    for (int u0 = 0; u0 < npts; u0 += chunk) {
        const int G = p.G, Ncam = p.Ncam, Nscale = p.Nscale;
        const int total = build_unit_list(u0, npts, p.P, p.Ncam, p.Nscale, smap, sbox, sloc, nullptr, ul,
                                          [&](int pp, int k, int sc) {
                                              float* d = gwb + ((long long)((pp * Ncam + k) * Nscale + sc)) * G;
                                              if ((G & 3) == 0) {  // 16-byte aligned rows of G values
                                                  for (int gg = 0; gg < G; gg += 4)
                                                      *reinterpret_cast<float4*>(d + gg) = make_float4(0.f, 0.f, 0.f, 0.f);
                                              } else {
                                                  for (int gg = 0; gg < G; ++gg) d[gg] = 0.0f;
                                              }
                                          });
        for (int q = team; q < total; q += nteams) {
            const UnitRec r = ul.rec[ul.list[q]];
            const int ps = r.wf >> 4;  // (pp * Ncam + k) * Nscale + s
            const float wv = ldw(wb + (long long)ps * p.G + g);
            const FT* p00 = fb + (long long)r.row00 * p.C;
            const FT* p10 = p00 + (long long)r.W * p.C;
            uint4 q4[4][NV];
            if (NV == 2 && p.wide && (r.wf & 15) == 15) {
                ld32(p00, q4[0][0], q4[0][NV - 1]);
                ld32(p00 + p.C, q4[1][0], q4[1][NV - 1]);
                ld32(p10, q4[2][0], q4[2][NV - 1]);
                ld32(p10 + p.C, q4[3][0], q4[3][NV - 1]);
            } else {
                const bool vx0 = r.wf & 1, vx1 = r.wf & 2, vy0 = r.wf & 4, vy1 = r.wf & 8;
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    q4[0][n] = (vy0 && vx0) ? ld16(p00 + n * VEC) : z;
                    q4[1][n] = (vy0 && vx1) ? ld16(p00 + p.C + n * VEC) : z;
                    q4[2][n] = (vy1 && vx0) ? ld16(p10 + n * VEC) : z;
                    q4[3][n] = (vy1 && vx1) ? ld16(p10 + p.C + n * VEC) : z;
                }
            }
            float2 d2[4];
#pragma unroll
            for (int cq = 0; cq < 4; ++cq) d2[cq] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
#pragma unroll
                for (int cq = 0; cq < 4; ++cq) {
                    float2 f[VEC / 2];
                    widen2(q4[cq][n], f, FT());
#pragma unroll
                    for (int j = 0; j < VEC / 2; ++j) d2[cq] = __ffma2_rn(go[n * (VEC / 2) + j], f[j], d2[cq]);
                }
            }
            const float d00 = d2[0].x + d2[0].y, d01 = d2[1].x + d2[1].y;
            const float d10 = d2[2].x + d2[2].y, d11 = d2[3].x + d2[3].y;
            const float ax = 1.0f - r.fx, ay = 1.0f - r.fy;
            const float dwp = ax * ay * d00 + r.fx * ay * d01 + ax * r.fy * d10 + r.fx * r.fy * d11;
            const float dw = team_sum_lw(dwp, tmask, lg);
            if ((tl & (lg - 1)) == 0) gwb[(long long)ps * p.G + g] = dw;
            float du = wv * (ay * (d01 - d00) + r.fy * (d11 - d10));
            float dv = wv * (ax * (d10 - d00) + r.fx * (d11 - d01));
            team_sum2_lw(du, dv, tmask, p.rt);
            if (tl == 0) suv[ps] = make_float2(du, dv);  // scaled by W_s, H_s at the end
        }
        __syncthreads();  // the list is rebuilt for the next chunk; suv is complete after the last one
    }
    // dloc of each point: its scales' terms in scale order
    float2* glb = reinterpret_cast<float2*>(p.gloc) + ba * (long long)per_point;
    for (int pt = threadIdx.x; pt < per_point; pt += blockDim.x) {
        const MapInfo* mrow = smap + (pt % p.Ncam) * p.Nscale;
        float du = 0.0f, dv = 0.0f;
        for (int s = 0; s < p.Nscale; ++s) {
            const float2 t = suv[pt * p.Nscale + s];
            du = fmaf((float)mrow[s].W, t.x, du);
            dv = fmaf((float)mrow[s].H, t.y, dv);
        }
        glb[pt] = make_float2(du, dv);
    }
}

using LocWKernel = void (*)(const LocWArgs);

template <typename FT, typename WT>
static LocWKernel locw_pick_nv(int nv) {
    switch (nv) {
        case 1: return bwd_locw_kernel<FT, WT, 1>;
        case 2: return bwd_locw_kernel<FT, WT, 2>;
        case 4: return bwd_locw_kernel<FT, WT, 4>;
    }
    return nullptr;
}

static LocWKernel locw_kernel_for(msda_dtype ft, msda_dtype wt, int nv) {
    if (ft == MSDA_F32 && wt == MSDA_F32) return locw_pick_nv<float, float>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_BF16) return locw_pick_nv<__nv_bfloat16, __nv_bfloat16>(nv);
    if (ft == MSDA_BF16 && wt == MSDA_F32) return locw_pick_nv<__nv_bfloat16, float>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F16) return locw_pick_nv<__half, __half>(nv);
    if (ft == MSDA_F16 && wt == MSDA_F32) return locw_pick_nv<__half, float>(nv);
    return nullptr;
}

msda_status launch_backward_locw(const Problem& p, const float* grad_out, float* grad_loc, float* grad_w, int warps,
                                 cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    LocWKernel k = locw_kernel_for(p.feat_t, p.w_t, p.nv);
    if (!k) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: unsupported feature/weight dtype pair");
    const long long nblocks = (long long)p.B * p.A;
    if (nblocks == 0) return MSDA_OK;
    if (nblocks > 0x7fffffffLL) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: B*A too large");
    if ((long long)p.P * p.Ncam * p.Nscale >= (1ll << 26))
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: too many point-scales per anchor");
    const LocWSmem lay(p.Ncam * p.Nscale, p.P, p.Ncam, p.Nscale, warps * 32 * kUnitsPerThread);
    if (lay.total > (size_t)dev.max_smem_optin)  // an anchor too large to stage: the per-point kernel
        return launch_backward_loc_w(p, grad_out, nullptr, grad_loc, grad_w, warps, 0, stream);
    st = ensure_smem((const void*)k, lay.total, dev);
    if (st != MSDA_OK) return st;
    LocWArgs a;
    a.feat = p.feat; a.shape = p.shape; a.start = p.start; a.loc = p.loc; a.w = p.w; a.go = grad_out;
    a.gloc = grad_loc; a.gw = grad_w;
    a.B = p.B; a.sum_hw = p.sum_hw; a.C = p.C; a.Ncam = p.Ncam; a.Nscale = p.Nscale;
    a.A = p.A; a.P = p.P; a.G = p.G; a.Cg = p.Cg; a.rt = p.rt; a.status = dev.status;
    const size_t esz = (size_t)dtype_size(p.feat_t);
    a.wide = (p.nv == 2 && ((uintptr_t)p.feat % 32) == 0 && ((size_t)p.C * esz) % 32 == 0 &&
              ((size_t)p.sum_hw * p.C * esz) % 32 == 0) ? 1 : 0;
    k<<<(unsigned)nblocks, warps * 32, lay.total, stream>>>(a);
    return check_launch("msda_backward dloc/dw");
}

}  // namespace msda
