// MSDA backward, deterministic feature gradient (sm_103a).
//
// The feature gradient is a scatter: every in-bound corner of every sampled
// point adds w_g * omega * go[c] to one feature row.  Scattering with FP32
// atomics makes the summation order depend on timing.  This mode instead
// gathers: it groups the in-bound corners by feature row (a counting sort:
// per-row counts, their prefix sum as row offsets, then every corner's slot
// id written into its row's segment), sorts each row's segment by slot id,
// turns the sorted slots into flat (omega, point-scale, anchor row) arrays,
// and then lets one team per feature row sum its contributions in slot order
// and write the row once (rows nobody touches get zeros, so no memset of the
// gradient is needed).  Integer atomics place the slot ids, in an order that
// varies run to run, but the per-row sort fixes it, so the FP32 sums, and the
// result, are bitwise reproducible for any launch.
//
// Point index t = (((b*A + a)*P + p)*Ncam + k); a corner's slot id packs
// (t, s, q) as (t << (sbits + 2)) | (s << 2) | q, with sbits the bits of
// Nscale - 1, so slot order is (t, s, q) order and the reduce decodes a slot
// with shifts and two divisions by constants (multiply-high).  The reduce
// kernel recomputes the corner weight omega from the location with the same
// arithmetic as every other kernel, so keys and weights agree.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "wsort.cuh"

namespace msda {

constexpr int kKeyPts = 4;                 // point-scales per thread in the corner kernels
constexpr int kKeyBlock = 256 * kKeyPts;   // point-scales per corner block
constexpr int kRowTile = 4096;             // rows per block of the row-offset scan (1024 threads x 4)
constexpr int kSegWarps = 8;               // warps per block of the long-segment sort
constexpr int kSegSmem = 1024;             // longest segment sorted in shared memory (per warp)
constexpr int kLaneSeg = 16;               // longest segment a single thread sorts in registers

struct DetLayout {
    size_t n;       // slots: 4 per point-scale (the most in-bound corners there can be)
    size_t nrows;   // B * sum_hw
    int ntiles;     // row-offset scan tiles
    size_t vals, e_om, e_pt, e_ba, cnt, rowptr, tsum, total;
};

static DetLayout det_layout(long long npts, long long nrows, size_t base = 0) {
    DetLayout L;
    L.n = (size_t)npts * 4;
    L.nrows = (size_t)nrows;
    L.ntiles = (int)((nrows + kRowTile - 1) / kRowTile);
    size_t off = base;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.vals = take(4 * L.n);   // slot ids grouped by row (sorted within each row)
    L.e_om = take(4 * L.n);   // flat arrays per contribution; e_om is also the large-segment sort's scratch
    L.e_pt = take(4 * L.n);
    L.e_ba = take(4 * L.n);
    L.cnt = take(4 * (L.nrows + 1));  // per-row counts (then the list of long rows) and the list's length
    L.rowptr = take(4 * (L.nrows + 1));
    L.tsum = take(4 * (size_t)(L.ntiles > 0 ? L.ntiles : 1));
    L.total = off;
    return L;
}

// The corner-slot arrays start after the cell-binned path's plan area when that path can apply (its flag
// gates these kernels); both paths' arrays then share the rest of the workspace.
static size_t det_body_base(const Problem& p) { return cb_shape_ok(p) ? cb_plan_bytes(p) : 0; }

size_t backward_det_workspace(const Problem& p) {
    const long long npts = (long long)p.B * p.A * p.P * p.Ncam * p.Nscale;
    const size_t base = det_body_base(p);
    const size_t slots = det_layout(npts, (long long)p.B * p.sum_hw, base).total;
    const size_t cells = cb_shape_ok(p) ? cb_workspace(p, base) : 0;
    return slots > cells ? slots : cells;
}

// True when the cell-binned path ran and set its flag: the corner-slot kernels have nothing to do (they read the
// flag themselves only when they were recorded in a graph capture; otherwise they are launched only if needed).
__device__ __forceinline__ bool gated(const int* gate) { return gate && *reinterpret_cast<const volatile int*>(gate); }

__global__ void __launch_bounds__(256) det_zero_kernel(uint32_t* __restrict__ p, long long n, const int* gate) {
    if (gated(gate)) return;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) p[i] = 0u;
}

// ---------------------------------------------------------------------------
// 1. Corners grouped by row
// ---------------------------------------------------------------------------
struct KeyArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    long long npts;
    int sum_hw, A, P, Ncam, Nscale, sbits;
    uint32_t* cnt;           // per row: in-bound corners (count pass); counted down by the fill pass
    const uint32_t* rowptr;  // row offsets (fill pass)
    uint32_t* vals;          // slot ids grouped by row (fill pass)
    int* status;
    const int* gate;         // the cell-binned path's flag, or NULL
    long long nblk;          // point-scale blocks of kKeyBlock
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
// pass adds each in-bound corner to its row's count; the fill pass takes a place in the row's segment for it
// (counting the row down) and stores the corner's slot id there.  Both passes see the same corners, so a row
// never runs out of places; the check only keeps a store inside the row if they ever differed.
template <bool FILL>
__global__ void __launch_bounds__(256) det_rows_kernel(const KeyArgs a) {
    if (gated(a.gate)) return;
    for (long long blk = blockIdx.x; blk < a.nblk; blk += gridDim.x) {
    const long long base = blk * kKeyBlock + (long long)threadIdx.x * kKeyPts;
#pragma unroll
    for (int i = 0; i < kKeyPts; ++i) {
        const long long pt = base + i;
        if (pt >= a.npts) break;
        uint32_t key[4];
        const unsigned mask = corner_keys(a, pt, key);
        const uint32_t slot = ((((uint32_t)(pt / a.Nscale)) << a.sbits) | (uint32_t)(pt % a.Nscale)) << 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!(mask & (1u << q))) continue;
            if (!FILL) {
                atomicAdd(a.cnt + key[q], 1u);
            } else {
                const uint32_t r0 = a.rowptr[key[q]], len = a.rowptr[key[q] + 1] - r0;
                const uint32_t left = atomicSub(a.cnt + key[q], 1u);  // places left in the row, this one included
                if (left - 1u < len)
                    a.vals[r0 + left - 1u] = slot + (uint32_t)q;
                else
                    raise_status(a.status, MSDA_ERR_OUT_OF_RANGE);
            }
        }
    }
    }
}

// Row offsets, step 1: per tile of kRowTile rows, the exclusive prefix of the counts inside the tile, and the
// tile's total.
__global__ void __launch_bounds__(1024) row_scan_tile_kernel(const uint32_t* __restrict__ cnt, long long nrows,
                                                             uint32_t* __restrict__ rowptr,
                                                             uint32_t* __restrict__ tsum, const int* gate) {
    if (gated(gate)) return;
    __shared__ uint32_t ws[32];
    const long long r0 = (long long)blockIdx.x * kRowTile + (long long)threadIdx.x * 4;
    uint32_t v[4], s = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = (r0 + j < nrows) ? cnt[r0 + j] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t run = block_inclusive_scan<32>(s, ws, &tot) - s;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (r0 + j < nrows) rowptr[r0 + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// Step 2 (one block): the tile totals become their exclusive prefix; *total gets the number of corners.
__global__ void __launch_bounds__(1024) row_scan_totals_kernel(uint32_t* __restrict__ tsum, int ntiles,
                                                               uint32_t* __restrict__ total, const int* gate) {
    if (gated(gate)) return;
    __shared__ uint32_t ws[32];
    uint32_t carry = 0u;
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? tsum[i] : 0u;
        uint32_t tot;
        const uint32_t incl = block_inclusive_scan<32>(v, ws, &tot);
        if (i < ntiles) tsum[i] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// Step 3: each row offset gets its tile's prefix.
__global__ void __launch_bounds__(256) row_scan_add_kernel(uint32_t* __restrict__ rowptr,
                                                           const uint32_t* __restrict__ tsum, long long nrows,
                                                           const int* gate) {
    if (gated(gate)) return;
    for (long long r = (long long)blockIdx.x * 256 + threadIdx.x; r < nrows; r += (long long)gridDim.x * 256)
        rowptr[r] += tsum[r / kRowTile];
}

// Segment sort, pass 1 of 2 (every row's slot ids ascending): one thread per row sorts a segment of up to
// kLaneSeg slots in registers (odd-even transposition); the longer rows are appended to a list (in any
// order: each row is sorted on its own) for pass 2.
__global__ void __launch_bounds__(256) det_segsort_short_kernel(const uint32_t* __restrict__ rowptr,
                                                                long long nrows, uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ longrows,
                                                                uint32_t* __restrict__ nlong, const int* gate) {
    if (gated(gate)) return;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long end = (nrows + 31) & ~31ll;  // whole warps iterate together
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < end; r += stride) {
        uint32_t e0 = 0u, n = 0u;
        if (r < nrows) {
            e0 = rowptr[r];
            n = rowptr[r + 1] - e0;
        }
        if (n > 1u && n <= (uint32_t)kLaneSeg) {
            uint32_t v[kLaneSeg];
#pragma unroll
            for (int j = 0; j < kLaneSeg; ++j) v[j] = ((uint32_t)j < n) ? vals[e0 + j] : 0xffffffffu;
#pragma unroll
            for (int rd = 0; rd < kLaneSeg; ++rd) {
#pragma unroll
                for (int j = rd & 1; j + 1 < kLaneSeg; j += 2) {
                    const uint32_t lo = min(v[j], v[j + 1]), hi = max(v[j], v[j + 1]);
                    v[j] = lo;
                    v[j + 1] = hi;
                }
            }
#pragma unroll
            for (int j = 0; j < kLaneSeg; ++j)
                if ((uint32_t)j < n) vals[e0 + j] = v[j];
        }
        const bool lng = n > (uint32_t)kLaneSeg;
        const unsigned bal = __ballot_sync(0xffffffffu, lng);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            uint32_t at = 0u;
            if (lane == leader) at = atomicAdd(nlong, (uint32_t)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, leader);
            if (lng) longrows[at + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)r;
        }
    }
}

// Load up to 32 * E slots of a row into registers, sort them, store them back.
template <int E>
__device__ __forceinline__ void sort_row_regs(uint32_t* v, uint32_t m, int lane) {
    uint32_t x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)(lane * E + e);
        x[e] = (i < m) ? v[i] : 0xffffffffu;
    }
    warp_sort_regs<E>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)(lane * E + e);
        if (i < m) v[i] = x[e];
    }
}

// Segment sort, pass 2: one warp per listed row: up to 256 slots in registers (bitonic, shuffles across lanes),
// up to kSegSmem with a bitonic sort in shared memory, longer ones by rank (every slot counts the smaller ones;
// slot ids are distinct) through the scratch array.
__global__ void __launch_bounds__(kSegWarps * 32) det_segsort_long_kernel(const uint32_t* __restrict__ rowptr,
                                                                          const uint32_t* __restrict__ longrows,
                                                                          const uint32_t* __restrict__ nlong,
                                                                          uint32_t* __restrict__ vals,
                                                                          uint32_t* __restrict__ scratch,
                                                                          const int* gate) {
    if (gated(gate)) return;
    __shared__ uint32_t sbuf[kSegWarps][kSegSmem];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* buf = sbuf[warp];
    const uint32_t nl = *nlong;
    for (uint32_t li = blockIdx.x * kSegWarps + warp; li < nl; li += gridDim.x * kSegWarps) {
        const uint32_t r = longrows[li];
        const uint32_t b0 = rowptr[r], m = rowptr[r + 1] - b0;
        uint32_t* v = vals + b0;
        if (m <= 32u) {
            uint32_t x = ((uint32_t)lane < m) ? v[lane] : 0xffffffffu;
            x = warp_sort32(x, lane);
            if ((uint32_t)lane < m) v[lane] = x;
        } else if (m <= 64u) {
            sort_row_regs<2>(v, m, lane);
        } else if (m <= 128u) {
            sort_row_regs<4>(v, m, lane);
        } else if (m <= 256u) {
            sort_row_regs<8>(v, m, lane);
        } else if (m <= (uint32_t)kSegSmem) {
            uint32_t p2 = 64u;
            while (p2 < m) p2 <<= 1;
            for (uint32_t i = lane; i < p2; i += 32) buf[i] = (i < m) ? v[i] : 0xffffffffu;
            __syncwarp();
            for (uint32_t k = 2; k <= p2; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t i = lane; i < p2; i += 32) {
                        const uint32_t ij = i ^ j;
                        if (ij > i) {
                            const uint32_t x = buf[i], y = buf[ij];
                            if ((x > y) == ((i & k) == 0)) {
                                buf[i] = y;
                                buf[ij] = x;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            for (uint32_t i = lane; i < m; i += 32) v[i] = buf[i];
            __syncwarp();  // buf is reused by the next row
        } else {
            uint32_t* w = scratch + b0;
            for (uint32_t i = lane; i < m; i += 32) {
                const uint32_t x = v[i];
                uint32_t rank = 0u;
                for (uint32_t j = 0; j < m; ++j) rank += (v[j] < x) ? 1u : 0u;
                w[rank] = x;
            }
            __syncwarp();
            for (uint32_t i = lane; i < m; i += 32) v[i] = w[i];
            __syncwarp();
        }
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
    const int* gate;      // the cell-binned path's flag, or NULL
    long long nrb;        // row blocks of the reduce
};

// Per sorted contribution e (in key order, valid keys only): decode the slot, recompute the corner weight
// omega from the location, and store (omega, point-scale, anchor row) in three flat arrays, so that the row
// reduce reads them contiguously instead of chasing slot -> location -> cell for every contribution.
__global__ void __launch_bounds__(256) det_prep_kernel(RedArgs a, size_t n, float* om_out, uint32_t* pt_out,
                                                       uint32_t* ba_out) {
    if (gated(a.gate)) return;
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
    if (gated(a.gate)) return;
    const int tpw = 32 / a.rt;
    const int nteams = (blockDim.x >> 5) * tpw;
    const int lane = threadIdx.x & 31;
    const int team = (threadIdx.x >> 5) * tpw + lane / a.rt;
    const int c0 = (lane & (a.rt - 1)) * CPL;
    const int g = c0 / a.Cg;
    for (long long rb = blockIdx.x; rb < a.nrb; rb += gridDim.x) {
    const long long row = rb * nteams + team;
    if (row >= a.nrows) continue;
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
}

// Launch parameters of the corner-slot form, computed on the host.  enqueue_corner_slot issues its kernels in
// order on `stream`: from the host (the cell-binned path does not apply), or from det_fallback_kernel on the
// device as tail launches (they run one after the other, after the launching grid, before the stream's next
// work), only when the cell-binned plan has cleared its flag; so a backward that the cell-binned path
// completes costs one single-thread launch here instead of ten empty grids.
struct SlotLaunch {
    KeyArgs ka;
    RedArgs ra;
    uint32_t *vals, *e_om, *e_pt, *e_ba, *cnt, *rowptr, *tsum;
    long long nrows, nkb, kgrid, zb, ab, sb, pb, rgrid, ntiles, n;
    unsigned segblocks;
    size_t prep_smem;
    int red_w;        // weights of the reduce: 0 FP32, 1 BF16, 2 FP16
    int red_cpl;      // channels per lane of the reduce (4, 8, 16, 32)
    const int* flag;  // the cell-binned plan's flag (device launcher only)
    const int* gate;  // the flag for the kernels to read themselves (launches recorded in a graph capture), or NULL
};

template <typename WT>
__host__ __device__ void enqueue_reduce(const SlotLaunch& s, cudaStream_t stream) {
    const unsigned g = (unsigned)s.rgrid;
    switch (s.red_cpl) {
        case 4: det_reduce_kernel<WT, 4><<<g, 256, 0, stream>>>(s.ra); break;
        case 8: det_reduce_kernel<WT, 8><<<g, 256, 0, stream>>>(s.ra); break;
        case 16: det_reduce_kernel<WT, 16><<<g, 256, 0, stream>>>(s.ra); break;
        default: det_reduce_kernel<WT, 32><<<g, 256, 0, stream>>>(s.ra); break;
    }
}

__host__ __device__ void enqueue_corner_slot(const SlotLaunch& s, cudaStream_t stream) {
    // per-row counts of the in-bound corners, row offsets (three-step scan), then the slot ids in place
    det_zero_kernel<<<(unsigned)s.zb, 256, 0, stream>>>(s.cnt, s.nrows + 1, s.gate);
    if (s.nkb > 0) det_rows_kernel<false><<<(unsigned)s.kgrid, 256, 0, stream>>>(s.ka);
    row_scan_tile_kernel<<<(unsigned)s.ntiles, 1024, 0, stream>>>(s.cnt, s.nrows, s.rowptr, s.tsum, s.gate);
    row_scan_totals_kernel<<<1, 1024, 0, stream>>>(s.tsum, (int)s.ntiles, s.rowptr + s.nrows, s.gate);
    row_scan_add_kernel<<<(unsigned)s.ab, 256, 0, stream>>>(s.rowptr, s.tsum, s.nrows, s.gate);
    if (s.nkb > 0) {
        det_rows_kernel<true><<<(unsigned)s.kgrid, 256, 0, stream>>>(s.ka);
        // the per-row counts are all zero again after the fill: their array takes the list of long rows
        det_segsort_short_kernel<<<(unsigned)s.sb, 256, 0, stream>>>(s.rowptr, s.nrows, s.vals, s.cnt, s.cnt + s.nrows,
                                                                      s.gate);
        det_segsort_long_kernel<<<s.segblocks, kSegWarps * 32, 0, stream>>>(s.rowptr, s.cnt, s.cnt + s.nrows, s.vals,
                                                                              s.e_om, s.gate);
    }
    if (s.n > 0)
        det_prep_kernel<<<(unsigned)s.pb, 256, s.prep_smem, stream>>>(s.ra, (size_t)s.n, reinterpret_cast<float*>(s.e_om),
                                                                       s.e_pt, s.e_ba);
    if (s.red_w == 0) enqueue_reduce<float>(s, stream);
    else if (s.red_w == 1) enqueue_reduce<__nv_bfloat16>(s, stream);
    else enqueue_reduce<__half>(s, stream);
}

__global__ void det_fallback_kernel(const SlotLaunch s) {
    if (*reinterpret_cast<const volatile int*>(s.flag)) return;  // the cell-binned path computed the gradient
    enqueue_corner_slot(s, cudaStreamTailLaunch);
    // a launch the device runtime refused leaves the gradient unwritten: say so in the status word
    if (cudaGetLastError() != cudaSuccess) raise_status(s.ka.status, MSDA_ERR_CUDA);
}

// A second stream per device for the cell-binned kernels, which read nothing the dloc/dw kernel writes: the
// two chains run side by side (the binning kernel alone fills under two blocks per SM).  Events fork the side
// stream from the caller's stream and join it back before anything that reads the flag or the gradient, so the
// call stays ordered on the caller's stream, and a graph capture of that stream takes the side stream's kernels
// in as a parallel branch.  The mutex is held from the fork to the join, so calls from several host threads do
// not interleave their events.
struct SideStream {
    cudaStream_t s;
    cudaEvent_t fork, join;
};
static std::mutex g_side_mu;
static SideStream g_side[128];
static signed char g_side_state[128];  // 0: not made yet, 1: made, -1: creation failed (no side stream)

// The device's side stream, made on the first call outside a graph capture; nullptr while none exists.  The
// caller holds g_side_mu.
static SideStream* side_stream(int device, bool may_create) {
    if (device < 0 || device >= 128) return nullptr;
    if (g_side_state[device] == 0 && may_create) {
        SideStream ss;
        if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) == cudaSuccess) {
            if (cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess) {
                if (cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) == cudaSuccess) {
                    g_side[device] = ss;
                    g_side_state[device] = 1;
                    return &g_side[device];
                }
                cudaEventDestroy(ss.fork);
            }
            cudaStreamDestroy(ss.s);
        }
        (void)cudaGetLastError();  // the call runs on the caller's stream alone; no error is left behind
        g_side_state[device] = -1;
    }
    return g_side_state[device] == 1 ? &g_side[device] : nullptr;
}

msda_status launch_backward_det(const Problem& p, const float* grad_out, float* grad_feat,
                                float* grad_loc, float* grad_w, void* ws, size_t ws_bytes,
                                int warps, bool allow_cells, cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    const long long npts = (long long)p.B * p.A * p.P * p.Ncam * p.Nscale;
    const long long nrows = (long long)p.B * p.sum_hw;
    const int sbits = scale_bits(p.Nscale);
    const long long npoints = (long long)p.B * p.A * p.P * p.Ncam;
    if (npts * 4 >= (1ll << 32) || (npoints << (sbits + 2)) >= (1ll << 31) || nrows >= (1ll << 32) - 1)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: deterministic mode limited to 2^31 corner slots and 2^32 rows");
    const size_t body = det_body_base(p);
    const DetLayout L = det_layout(npts, nrows, body);
    const size_t need = backward_det_workspace(p);
    if (!ws || ws_bytes < need)
        return fail(MSDA_ERR_WORKSPACE, "msda_backward: deterministic mode needs %zu workspace bytes", need);
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
    if (cpl != 4 && cpl != 8 && cpl != 16 && cpl != 32)
        return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: no reduce kernel for %d channels per lane", cpl);

    // The feature gradient: the cell-binned path when it applies (decided on the device for the maps), else the
    // corner-slot path, which the launcher below issues from the device only when the cell-binned plan has
    // cleared its flag.  The cell-binned kernels go to the side stream, beside dloc and dw (no feature scatter)
    // on the caller's stream.
    const bool cells = nrows > 0 && allow_cells && cb_shape_ok(p) && cb_device_ok(p, dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cells && cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return check_launch("msda_backward capture query");
    std::unique_lock<std::mutex> side_lock(g_side_mu, std::defer_lock);
    SideStream* side = nullptr;
    if (cells) {
        side_lock.lock();
        side = side_stream(dev.device, cap == cudaStreamCaptureStatusNone);
        if (side && (cudaEventRecord(side->fork, stream) != cudaSuccess ||
                     cudaStreamWaitEvent(side->s, side->fork, 0) != cudaSuccess))
            return check_launch("msda_backward side-stream fork");
    }
    const int* gate = nullptr;
    msda_status st_cells = MSDA_OK;
    if (cells) {
        st_cells = launch_backward_cb(p, grad_out, grad_feat, ws, body, side ? side->s : stream);
        gate = reinterpret_cast<const int*>(ws);
    }
    st = launch_backward_locw(p, grad_out, grad_loc, grad_w, warps, stream);
    if (side) {
        // joined whatever the launches above returned, so no capture is left with an unjoined branch
        if (cudaEventRecord(side->join, side->s) != cudaSuccess || cudaStreamWaitEvent(stream, side->join, 0) != cudaSuccess)
            return check_launch("msda_backward side-stream join");
        side_lock.unlock();
    }
    if (st != MSDA_OK) return st;
    if (st_cells != MSDA_OK) return st_cells;
    if (nrows == 0) return MSDA_OK;

    unsigned char* base = reinterpret_cast<unsigned char*>(ws);
    SlotLaunch sl;
    sl.vals = reinterpret_cast<uint32_t*>(base + L.vals);
    sl.e_om = reinterpret_cast<uint32_t*>(base + L.e_om);
    sl.e_pt = reinterpret_cast<uint32_t*>(base + L.e_pt);
    sl.e_ba = reinterpret_cast<uint32_t*>(base + L.e_ba);
    sl.cnt = reinterpret_cast<uint32_t*>(base + L.cnt);
    sl.rowptr = reinterpret_cast<uint32_t*>(base + L.rowptr);
    sl.tsum = reinterpret_cast<uint32_t*>(base + L.tsum);
    sl.nrows = nrows;
    KeyArgs& ka = sl.ka;
    ka.shape = p.shape; ka.start = p.start; ka.loc = p.loc; ka.npts = npts; ka.sum_hw = p.sum_hw; ka.A = p.A;
    ka.P = p.P; ka.Ncam = p.Ncam; ka.Nscale = p.Nscale; ka.sbits = sbits; ka.cnt = sl.cnt; ka.rowptr = sl.rowptr;
    ka.vals = sl.vals; ka.status = dev.status; ka.gate = nullptr;
    const long long cap8 = (long long)dev.sm_count * 8;  // grid-stride kernels: one wave of 8 blocks per SM
    sl.nkb = (npts + kKeyBlock - 1) / kKeyBlock;
    ka.nblk = sl.nkb;
    sl.kgrid = sl.nkb < cap8 ? sl.nkb : cap8;
    sl.zb = (nrows + 1 + 255) / 256;
    if (sl.zb > cap8) sl.zb = cap8;
    sl.ab = (nrows + 255) / 256;
    if (sl.ab > cap8) sl.ab = cap8;
    sl.sb = sl.ab;
    sl.segblocks = (long long)dev.sm_count * 8;
    sl.ntiles = L.ntiles;
    RedArgs& ra = sl.ra;
    ra.shape = p.shape; ra.start = p.start; ra.loc = p.loc; ra.w = p.w; ra.go = grad_out;
    ra.vals = sl.vals; ra.rowptr = sl.rowptr; ra.gfeat = grad_feat; ra.nrows = nrows;
    ra.e_om = reinterpret_cast<const float*>(sl.e_om);
    ra.e_pt = sl.e_pt;
    ra.e_ba = sl.e_ba;
    ra.wide = (((uintptr_t)grad_out % 32) == 0 && ((size_t)p.C * 4) % 32 == 0) ? 1 : 0;
    ra.sum_hw = p.sum_hw; ra.C = p.C; ra.Ncam = p.Ncam; ra.Nscale = p.Nscale; ra.A = p.A; ra.P = p.P;
    ra.G = p.G; ra.Cg = p.Cg; ra.rt = red_rt; ra.sbits = sbits; ra.status = dev.status; ra.gate = nullptr;
    ra.ncam = make_fastdiv((uint32_t)(p.Ncam > 0 ? p.Ncam : 1));
    ra.pncam = make_fastdiv((uint32_t)((long long)p.P * p.Ncam > 0 ? (long long)p.P * p.Ncam : 1));
    sl.n = (long long)L.n;
    sl.prep_smem = sizeof(MapInfo) * (size_t)p.Ncam * p.Nscale;
    if (sl.n > 0 && (st = ensure_smem((const void*)det_prep_kernel, sl.prep_smem, dev)) != MSDA_OK) return st;
    sl.pb = (sl.n + 255) / 256;
    if (sl.pb > cap8) sl.pb = cap8;
    const int nteams = 8 * (32 / red_rt);
    ra.nrb = (nrows + nteams - 1) / nteams;
    sl.rgrid = ra.nrb < cap8 ? ra.nrb : cap8;
    sl.red_w = p.w_t == MSDA_F32 ? 0 : p.w_t == MSDA_BF16 ? 1 : 2;
    sl.red_cpl = cpl;
    sl.flag = gate;
    sl.gate = nullptr;
    if (gate && cap == cudaStreamCaptureStatusNone) {
        // the cell-binned path is in the stream: one thread checks its flag and issues the corner-slot kernels
        // as tail launches only when the flag is clear
        det_fallback_kernel<<<1, 1, 0, stream>>>(sl);
    } else {
        // no cell-binned path, or a graph capture (its replays do not run the tail launches): the kernels are
        // enqueued here, each returning at once when the flag is set
        sl.gate = gate;
        sl.ka.gate = gate;
        sl.ra.gate = gate;
        enqueue_corner_slot(sl, stream);
    }
    return check_launch("msda_backward corner-slot form");
}

}  // namespace msda
