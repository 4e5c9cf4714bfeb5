// MSDA backward, deterministic feature gradient (sm_103a).
//
// The feature gradient is a scatter: every in-bound corner of every sampled
// point adds w_g * omega * go[c] to one feature row.  Scattering with
// atomics makes the FP32 summation order depend on timing.  This mode
// instead gathers: it builds, for every in-bound corner of every
// point-scale, the key (feature row) and the value (the corner's slot id),
// compacted in slot order, sorts the pairs by key with a stable LSD radix
// sort, so that equal rows keep the slot order,
// turns the sorted slots into flat (omega, point-scale, anchor row) arrays,
// and then lets one team per feature row sum its contributions in that
// order and write the row once (rows nobody touches get zeros, so no memset
// is needed).  The result is bitwise reproducible for any launch.
//
// Point index t = (((b*A + a)*P + p)*Ncam + k); a corner's slot id packs
// (t, s, q) as (t << (sbits + 2)) | (s << 2) | q, with sbits the bits of
// Nscale - 1, so slot order is (t, s, q) order and the reduce decodes a slot
// with shifts and two divisions by constants (multiply-high).  The reduce
// kernel recomputes the corner weight omega from the location with the same
// arithmetic as every other kernel, so keys and weights agree.
#include "common.cuh"
#include "internal.h"

namespace msda {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;  // keys per sort block
constexpr int kKeyPts = 4;                         // point-scales per thread in the key kernels
constexpr int kKeyBlock = 256 * kKeyPts;           // point-scales per key block

struct DetLayout {
    size_t n;       // slots: 4 per point-scale
    size_t nrows;   // B * sum_hw
    int nb;         // sort tiles
    int passes;     // 8-bit digit passes
    size_t k0, v0, k1, v1, hist, tot, rowptr, cnt, nvalid, total;
    int nkb;        // key blocks
};

static DetLayout det_layout(long long npts, long long nrows) {
    DetLayout L;
    L.n = (size_t)npts * 4;
    L.nrows = (size_t)nrows;
    L.nb = (int)((L.n + kTile - 1) / kTile);
    int bits = 0;
    while (bits < 32 && ((unsigned long long)nrows >> bits) != 0) ++bits;  // keys go up to nrows
    L.passes = (bits + 7) / 8;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.k0 = take(4 * L.n);
    L.v0 = take(4 * L.n);
    L.k1 = take(4 * L.n);
    L.v1 = take(4 * L.n);
    L.hist = take(4 * (size_t)256 * (L.nb > 0 ? L.nb : 1));
    L.tot = take(4 * 256);
    L.rowptr = take(4 * (L.nrows + 1));
    L.nkb = (int)((npts + kKeyBlock - 1) / kKeyBlock);
    L.cnt = take(4 * (size_t)(L.nkb > 0 ? L.nkb : 1));
    L.nvalid = take(4);
    L.total = off;
    return L;
}

size_t backward_det_workspace(const Problem& p) {
    const long long npts = (long long)p.B * p.A * p.P * p.Ncam * p.Nscale;
    return det_layout(npts, (long long)p.B * p.sum_hw).total;
}

// ---------------------------------------------------------------------------
// 1. Keys and slot ids
// ---------------------------------------------------------------------------
struct KeyArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    uint32_t* keys;
    uint32_t* vals;
    long long npts;
    int sum_hw, A, P, Ncam, Nscale, sbits;
    uint32_t* counts;  // per key block: in-bound corners (count pass), then their exclusive prefix (write pass)
    int* status;
};

// Division by a fixed d >= 1 for numerators below 2^31 (the round-up method
// of Granlund and Montgomery): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l; the sum
// stays below 2^32 because umulhi(n, m) <= n.
struct FastDiv {
    uint32_t d, m, l;
};

static FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((1ull << f.l) < d) ++f.l;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1ull);
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.l; }

static int scale_bits(int Nscale) {
    int b = 0;
    while ((1 << b) < Nscale) ++b;
    return b;
}

// Inclusive scan of one value per thread over a block of 32*W threads.
template <int W>
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < W ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < W) warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t r = v + (warp > 0 ? warp_sums[warp - 1] : 0u);
    if (total) *total = warp_sums[W - 1];
    __syncthreads();
    return r;
}

// 32 FP32 bytes (p 32-byte aligned) in one 256-bit read-only load.
__device__ __forceinline__ void ld32(const void* p, float4& lo, float4& hi) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
                 : "l"(p));
}

// Keys of the in-bound corners of one point-scale; bit q of the result marks corner q in bounds.
__device__ __forceinline__ unsigned corner_keys(const KeyArgs& a, long long pt, uint32_t key[4]) {
    const int s = (int)(pt % a.Nscale);
    const long long t = pt / a.Nscale;            // ((b*A + a)*P + p)*Ncam + k
    const int k = (int)(t % a.Ncam);
    const long long b = t / ((long long)a.Ncam * a.P * a.A);
    const MapInfo m = load_map(a.shape, a.start, k * a.Nscale + s, a.sum_hw, a.status);
    const float2 uv = __ldg(reinterpret_cast<const float2*>(a.loc) + t);
    Cell c;
    const bool in = (m.W != 0) && locate(uv.x, uv.y, m.H, m.W, c);
    unsigned mask = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = c.y0 + (q >> 1), j = c.x0 + (q & 1);
        const bool ok = in && i >= 0 && i < m.H && j >= 0 && j < m.W;
        key[q] = ok ? (uint32_t)(b * a.sum_hw + m.start + i * m.W + j) : 0u;
        mask |= ok ? (1u << q) : 0u;
    }
    return mask;
}

// Block b handles point-scales [b*kKeyBlock, (b+1)*kKeyBlock), kKeyPts consecutive ones per thread.  The count
// pass stores the block's number of in-bound corners; the write pass stores only those corners' (key, slot)
// pairs, at the block's prefix plus the thread's prefix inside the block, so the pairs stay in slot order
// (which the stable sort keeps for equal keys) and the sort sees no out-of-bounds corners at all.
template <bool WRITE>
__global__ void __launch_bounds__(256) det_keys_kernel(const KeyArgs a) {
    __shared__ uint32_t ws[32];
    const long long base = (long long)blockIdx.x * kKeyBlock + (long long)threadIdx.x * kKeyPts;
    uint32_t key[kKeyPts][4];
    unsigned mask[kKeyPts];
    uint32_t cnt = 0u;
#pragma unroll
    for (int i = 0; i < kKeyPts; ++i) {
        mask[i] = (base + i < a.npts) ? corner_keys(a, base + i, key[i]) : 0u;
        cnt += (uint32_t)__popc(mask[i]);
    }
    uint32_t total;
    const uint32_t incl = block_inclusive_scan<8>(cnt, ws, &total);
    if (!WRITE) {
        if (threadIdx.x == 0) a.counts[blockIdx.x] = total;
        return;
    }
    uint32_t off = a.counts[blockIdx.x] + incl - cnt;
#pragma unroll
    for (int i = 0; i < kKeyPts; ++i) {
        const long long pt = base + i;
        const uint32_t slot = ((((uint32_t)(pt / a.Nscale)) << a.sbits) | (uint32_t)(pt % a.Nscale)) << 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (mask[i] & (1u << q)) {
                a.keys[off] = key[i][q];
                a.vals[off] = slot + (uint32_t)q;
                ++off;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2. Stable LSD radix sort, 8-bit digits: histogram, per-digit scan, scatter
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                  const uint32_t* __restrict__ n_dev, int shift,
                                                                  uint32_t* __restrict__ hist, int nb) {
    const size_t n = *n_dev;  // keys to sort (the grid covers the most there can be)
    const size_t base = (size_t)blockIdx.x * kTile;
    if (base >= n) {  // a tile past the keys: empty counts (uniform over the block)
        hist[(size_t)threadIdx.x * nb + blockIdx.x] = 0u;
        return;
    }
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        const size_t i = base + (size_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(__ldg(keys + i) >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Block d turns hist[d][0..nb) into exclusive prefixes and writes totals[d].
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* __restrict__ hist, int nb,
                                                          uint32_t* __restrict__ totals) {
    __shared__ uint32_t ws[32];
    uint32_t* h = hist + (size_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? h[i] : 0u;
        uint32_t tot;
        const uint32_t incl = block_inclusive_scan<32>(v, ws, &tot);
        if (i < nb) h[i] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_dev, int shift, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ totals, int nb) {
    const size_t n = *n_dev;
    if ((size_t)blockIdx.x * kTile >= n) return;  // a tile past the keys (uniform over the block)
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t ws[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    {
        const uint32_t tot = totals[t];
        const uint32_t incl = block_inclusive_scan<NW>(tot, ws, nullptr);
        base[t] = incl - tot + hist[(size_t)t * nb + blockIdx.x];
#pragma unroll
        for (int w = 0; w < NW; ++w) wcnt[w][t] = 0u;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const size_t tile = (size_t)blockIdx.x * kTile;
    for (int r = 0; r < kSortItems; ++r) {
        const size_t i = tile + (size_t)r * kSortThreads + t;
        const bool ok = i < n;
        const uint32_t key = ok ? kin[i] : 0u;
        const uint32_t val = ok ? vin[i] : 0u;
        const int d = ok ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            sum += wcnt[w][t];
            wcnt[w][t] = 0u;
        }
        base[t] += sum;
        __syncthreads();
    }
}

// rowptr[r] = number of sorted keys < r, for r in [0, nrows].
__global__ void __launch_bounds__(256) row_ptr_kernel(const uint32_t* __restrict__ ks,
                                                      const uint32_t* __restrict__ n_dev, uint32_t nrows,
                                                      uint32_t* __restrict__ rowptr) {
    const size_t n = *n_dev;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i <= n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long lo = (i == 0) ? 0ull : (unsigned long long)ks[i - 1] + 1ull;
        unsigned long long hi = (i == n) ? (unsigned long long)nrows : (unsigned long long)ks[i];
        if (hi > nrows) hi = nrows;
        for (unsigned long long r = lo; r <= hi; ++r) rowptr[r] = (uint32_t)i;
    }
}

// ---------------------------------------------------------------------------
// 3. Fixed-order segment reduce: one team of rt lanes per feature row
// ---------------------------------------------------------------------------
struct RedArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* go;
    const uint32_t* vals;
    const uint32_t* rowptr;
    const float* e_om;       // per sorted contribution: bilinear weight omega of its corner
    const uint32_t* e_pt;    //   point-scale index (t * Nscale + s)
    const uint32_t* e_ba;    //   anchor row b * A + a of grad_out
    int wide;                // grad_out rows and lane chunks 32-byte aligned: 256-bit loads
    float* gfeat;
    long long nrows;
    int sum_hw, C, Ncam, Nscale, A, P, G, Cg, rt, sbits;
    FastDiv ncam, pncam;  // divisions by Ncam and P*Ncam
    int* status;
};

// Per sorted contribution e (in key order, valid keys only): decode the slot, recompute the corner weight
// omega from the location, and store (omega, point-scale, anchor row) in three flat arrays, so that the row
// reduce reads them contiguously instead of chasing slot -> location -> cell for every contribution.
__global__ void __launch_bounds__(256) det_prep_kernel(RedArgs a, size_t n, float* om_out, uint32_t* pt_out,
                                                       uint32_t* ba_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    MapInfo* smap = reinterpret_cast<MapInfo*>(smem);
    const int nmaps = a.Ncam * a.Nscale;
    for (int i = threadIdx.x; i < nmaps; i += blockDim.x)
        smap[i] = load_map(a.shape, a.start, i, a.sum_hw, nullptr);
    __syncthreads();
    const size_t nvalid = a.rowptr[a.nrows];  // every sorted key is an in-bound corner
    const uint32_t smask = (1u << a.sbits) - 1u;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nvalid && e < n;
         e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t v = __ldg(a.vals + e);
        const int q = (int)(v & 3u);
        const int s = (int)((v >> 2) & smask);
        const uint32_t t = v >> (a.sbits + 2);
        const int k = (int)(t - fdiv(t, a.ncam) * (uint32_t)a.Ncam);
        const MapInfo m = smap[k * a.Nscale + s];
        const float2 uv = __ldg(reinterpret_cast<const float2*>(a.loc) + t);
        Cell c;
        locate(uv.x, uv.y, m.H, m.W, c);  // in range: the key was valid
        const float ax = 1.0f - c.fx, ay = 1.0f - c.fy;
        om_out[e] = (q == 0) ? ax * ay : (q == 1) ? c.fx * ay : (q == 2) ? ax * c.fy : c.fx * c.fy;
        pt_out[e] = t * (uint32_t)a.Nscale + (uint32_t)s;
        ba_out[e] = fdiv(t, a.pncam);
    }
}

// One team of rt lanes per feature row sums its contributions in sorted (slot) order; U contributions are
// loaded together, then added in order.
template <typename WT, int CPL>
__global__ void __launch_bounds__(256) det_reduce_kernel(const RedArgs a) {
    constexpr int U = CPL >= 32 ? 1 : 32 / CPL;
    const int tpw = 32 / a.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const int lane = threadIdx.x & 31;
    const int team = (threadIdx.x >> 5) * tpw + lane / a.rt;
    const int c0 = (lane & (a.rt - 1)) * CPL;
    const int g = c0 / a.Cg;
    const long long row = (long long)blockIdx.x * nteams + team;
    if (row >= a.nrows) return;
    const WT* wp = reinterpret_cast<const WT*>(a.w);
    float acc[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) acc[j] = 0.0f;
    const uint32_t e0 = a.rowptr[row], e1 = a.rowptr[row + 1];
    for (uint32_t e = e0; e < e1; e += U) {
        float coef[U];
        float4 gv[U][CPL / 4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = (e + u < e1) ? e + u : e;  // the tail repeats a valid entry, not added below
            coef[u] = ldw(wp + (long long)__ldg(a.e_pt + eu) * a.G + g) * __ldg(a.e_om + eu);
            const float4* gsrc = reinterpret_cast<const float4*>(a.go + (long long)__ldg(a.e_ba + eu) * a.C + c0);
#pragma unroll
            for (int j = 0; j + 1 < CPL / 4; j += 2) {
                if (a.wide) {
                    ld32(gsrc + j, gv[u][j], gv[u][j + 1]);  // one 256-bit load for two chunks
                } else {
                    gv[u][j] = __ldg(gsrc + j);
                    gv[u][j + 1] = __ldg(gsrc + j + 1);
                }
            }
            if ((CPL / 4) & 1) gv[u][CPL / 4 - 1] = __ldg(gsrc + CPL / 4 - 1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (e + u < e1) {
#pragma unroll
                for (int j = 0; j < CPL / 4; ++j) {
                    acc[4 * j + 0] = fmaf(coef[u], gv[u][j].x, acc[4 * j + 0]);
                    acc[4 * j + 1] = fmaf(coef[u], gv[u][j].y, acc[4 * j + 1]);
                    acc[4 * j + 2] = fmaf(coef[u], gv[u][j].z, acc[4 * j + 2]);
                    acc[4 * j + 3] = fmaf(coef[u], gv[u][j].w, acc[4 * j + 3]);
                }
            }
        }
    }
    float4* dst = reinterpret_cast<float4*>(a.gfeat + row * a.C + c0);
#pragma unroll
    for (int j = 0; j < CPL / 4; ++j) dst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
}

using RedKernel = void (*)(const RedArgs);

template <typename WT>
static RedKernel red_pick(int cpl) {
    switch (cpl) {
        case 4: return det_reduce_kernel<WT, 4>;
        case 8: return det_reduce_kernel<WT, 8>;
        case 16: return det_reduce_kernel<WT, 16>;
        case 32: return det_reduce_kernel<WT, 32>;
    }
    return nullptr;
}

msda_status launch_backward_det(const Problem& p, const float* grad_out, float* grad_feat,
                                float* grad_loc, float* grad_w, void* ws, size_t ws_bytes,
                                int warps, cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    const long long npts = (long long)p.B * p.A * p.P * p.Ncam * p.Nscale;
    const long long nrows = (long long)p.B * p.sum_hw;
    const int sbits = scale_bits(p.Nscale);
    const long long npoints = (long long)p.B * p.A * p.P * p.Ncam;
    if (npts * 4 >= (1ll << 32) || (npoints << (sbits + 2)) >= (1ll << 31) || nrows >= (1ll << 32) - 1)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: deterministic mode limited to 2^31 corner slots and 2^32 rows");
    const DetLayout L = det_layout(npts, nrows);
    if (!ws || ws_bytes < L.total)
        return fail(MSDA_ERR_WORKSPACE, "msda_backward: deterministic mode needs %zu workspace bytes", L.total);
    // The row reduce has its own lane split, independent of the gather kernel's: 8 channels per lane when C
    // and the group width allow it (measured fastest: short rows of ~10 contributions favour many lanes),
    // else the split of the gather kernel.
    int red_rt = p.rt;
    for (int cand : {8, 4, 16, 32}) {
        const int r = p.C / cand;
        if (p.C % cand == 0 && p.Cg % cand == 0 && r >= 1 && r <= 32 && (r & (r - 1)) == 0) {
            red_rt = r;
            break;
        }
    }
    const int cpl = p.C / red_rt;
    RedKernel red = (p.w_t == MSDA_F32) ? red_pick<float>(cpl)
                  : (p.w_t == MSDA_BF16) ? red_pick<__nv_bfloat16>(cpl) : red_pick<__half>(cpl);
    if (!red) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: no reduce kernel for %d channels per lane", cpl);

    // dloc and dw (no feature scatter)
    st = launch_backward_locw(p, grad_out, grad_loc, grad_w, warps, stream);
    if (st != MSDA_OK) return st;
    if (nrows == 0) return MSDA_OK;

    unsigned char* base = reinterpret_cast<unsigned char*>(ws);
    uint32_t* kbuf[2] = {reinterpret_cast<uint32_t*>(base + L.k0), reinterpret_cast<uint32_t*>(base + L.k1)};
    uint32_t* vbuf[2] = {reinterpret_cast<uint32_t*>(base + L.v0), reinterpret_cast<uint32_t*>(base + L.v1)};
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + L.hist);
    uint32_t* tot = reinterpret_cast<uint32_t*>(base + L.tot);
    uint32_t* rowptr = reinterpret_cast<uint32_t*>(base + L.rowptr);
    int cur = 0;
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.cnt);
    uint32_t* nvalid = reinterpret_cast<uint32_t*>(base + L.nvalid);
    if (cudaMemsetAsync(nvalid, 0, sizeof(uint32_t), stream) != cudaSuccess) return check_launch("msda_backward");
    if (npts > 0) {
        KeyArgs ka;
        ka.shape = p.shape; ka.start = p.start; ka.loc = p.loc; ka.keys = kbuf[0]; ka.vals = vbuf[0];
        ka.npts = npts; ka.sum_hw = p.sum_hw; ka.A = p.A; ka.P = p.P; ka.Ncam = p.Ncam;
        ka.Nscale = p.Nscale; ka.sbits = sbits; ka.counts = counts; ka.status = dev.status;
        // in-bound corners per key block, their prefix (and total), then the compacted (key, slot) pairs
        det_keys_kernel<false><<<L.nkb, 256, 0, stream>>>(ka);
        radix_scan_kernel<<<1, 1024, 0, stream>>>(counts, L.nkb, nvalid);
        det_keys_kernel<true><<<L.nkb, 256, 0, stream>>>(ka);
        if ((st = check_launch("msda_backward keys")) != MSDA_OK) return st;
        for (int pass = 0; pass < L.passes; ++pass) {
            const int shift = 8 * pass;
            radix_hist_kernel<<<L.nb, kSortThreads, 0, stream>>>(kbuf[cur], nvalid, shift, hist, L.nb);
            radix_scan_kernel<<<256, 1024, 0, stream>>>(hist, L.nb, tot);
            radix_scatter_kernel<<<L.nb, kSortThreads, 0, stream>>>(kbuf[cur], vbuf[cur], kbuf[cur ^ 1],
                                                                    vbuf[cur ^ 1], nvalid, shift, hist, tot, L.nb);
            if ((st = check_launch("msda_backward sort")) != MSDA_OK) return st;
            cur ^= 1;
        }
    }
    {
        long long rb = ((long long)L.n + 1 + 255) / 256;
        if (rb > (long long)dev.sm_count * 32) rb = (long long)dev.sm_count * 32;
        row_ptr_kernel<<<(unsigned)rb, 256, 0, stream>>>(kbuf[cur], nvalid, (uint32_t)nrows, rowptr);
        if ((st = check_launch("msda_backward row offsets")) != MSDA_OK) return st;
    }
    RedArgs ra;
    ra.shape = p.shape; ra.start = p.start; ra.loc = p.loc; ra.w = p.w; ra.go = grad_out;
    ra.vals = vbuf[cur]; ra.rowptr = rowptr; ra.gfeat = grad_feat; ra.nrows = nrows;
    // the sorted keys and the other sort buffers are free once the row offsets exist
    ra.e_om = reinterpret_cast<const float*>(kbuf[cur ^ 1]);
    ra.e_pt = vbuf[cur ^ 1];
    ra.e_ba = kbuf[cur];
    ra.wide = (((uintptr_t)grad_out % 32) == 0 && ((size_t)p.C * 4) % 32 == 0) ? 1 : 0;
    ra.sum_hw = p.sum_hw; ra.C = p.C; ra.Ncam = p.Ncam; ra.Nscale = p.Nscale; ra.A = p.A; ra.P = p.P;
    ra.G = p.G; ra.Cg = p.Cg; ra.rt = red_rt; ra.sbits = sbits; ra.status = dev.status;
    ra.ncam = make_fastdiv((uint32_t)(p.Ncam > 0 ? p.Ncam : 1));
    ra.pncam = make_fastdiv((uint32_t)((long long)p.P * p.Ncam > 0 ? (long long)p.P * p.Ncam : 1));
    const size_t smem = sizeof(MapInfo) * (size_t)p.Ncam * p.Nscale;
    if (L.n > 0) {
        if ((st = ensure_smem((const void*)det_prep_kernel, smem, dev)) != MSDA_OK) return st;
        long long pb = ((long long)L.n + 255) / 256;
        if (pb > (long long)dev.sm_count * 32) pb = (long long)dev.sm_count * 32;
        det_prep_kernel<<<(unsigned)pb, 256, smem, stream>>>(ra, L.n, reinterpret_cast<float*>(kbuf[cur ^ 1]),
                                                             vbuf[cur ^ 1], kbuf[cur]);
        if ((st = check_launch("msda_backward prep")) != MSDA_OK) return st;
    }
    const int nteams = 8 * (32 / red_rt);
    const long long rblocks = (nrows + nteams - 1) / nteams;
    red<<<(unsigned)rblocks, 256, 0, stream>>>(ra);
    return check_launch("msda_backward reduce");
}

}  // namespace msda
