// MSDA backward, deterministic feature gradient by bilinear cell (sm_103a).
//
// Every in-view point-scale lies in one bilinear cell (y0, x0) of its map and adds to the feature rows at the
// cell's four corners.  Seen from the other side, feature row (i, j) of a map receives exactly the points of
// four cells: (i-1, j-1) through their corner 3 (y0+1, x0+1), (i-1, j) through corner 2 (y0+1, x0),
// (i, j-1) through corner 1 (y0, x0+1) and (i, j) through corner 0.  This path therefore bins each map's
// point-scales by cell, in point order (an ordered placement, so neither a sort nor floating-point atomics
// are needed), and then forms every feature row as one fixed-order sum over the bins of its four cells:
//
//   grad_feat[row, group g] = sum over the cells (i-1,j-1), (i-1,j), (i,j-1), (i,j), over the cell's points in
//                             point order, of w[point-scale, g] * omega_q(fx, fy) * grad_out[b, a, group g]
//
// with omega_q the corner's bilinear weight and the same products as every other kernel (w * (x factor *
// y factor)), so only the order of the sums differs from the atomic form.  A block works on one channel group
// at a time with grad_out[b, :, group g] staged in shared memory (A * C/G FP32 values): the per-contribution
// read of grad_out, which bounds the corner-slot path of det.cu, comes from shared memory instead of L2.
//
// Cells of an H x W map are (cy, cx), cy in [-1, H-1], cx in [-1, W-1] (a point at x in (-1, 0) has
// x0 = -1), numbered (cy + 1) * (W + 1) + (cx + 1).  With c the number of cell (i, j), the cells of row (i, j)
// are c - W - 2, c - W - 1 (consecutive) and c - 1, c, so a row reads two contiguous ranges of bins.
//
// The bins of a map only describe that map, so the maps must not overlap.  cb_plan_kernel checks this on the
// device, together with the sizes the path needs; when a check fails it clears the plan's flag and the
// corner-slot path of det.cu (whose kernels read the same flag) computes the gradient instead.
#include "common.cuh"
#include "internal.h"
#include "tma.cuh"
#include "wsort.cuh"

namespace msda {

constexpr int kCbThreads = 1024;     // threads of the bin and reduce blocks
constexpr int kCbWarps = kCbThreads / 32;
constexpr int kCbMaxMaps = 4096;     // maps the single-block plan kernel can sort
constexpr int kCbHeavyPerRow = 32;   // expected contributions per row from which a warp sweeps a column
constexpr unsigned short kNoCell = 0xffffu;
constexpr int kCbMaxBin = 256;       // points one cell may hold (more: the corner-slot path takes over)
constexpr int kCbMaxRows = 1024;     // image rows of a map the reduce's band planner holds
constexpr int kCbDirect = 1 << 30;   // band-end flag: the band is read in place, not staged

struct CbMap {
    int H, W, start;  // W == 0: the map is invalid and skipped
    int cbase;        // first entry of the map in one batch element's cell-pointer array
    int nseg;         // row segments per column (columns * segments = sweep tasks)
    int heavy;        // 1: a warp sweeps a column segment; 0: a lane group does
    int pad[2];
};

struct CbHeader {
    int ok;           // 1: this path runs and the corner-slot form is not issued
    int ngaps;        // row ranges of a batch element that no valid map covers
    int pad[62];
};

struct CbLayout {
    size_t maps, gaps, queues, plan_end;  // plan area (read by the corner-slot kernels: header.ok)
    size_t cellptr, aoff, coef, loct;     // cell pointers, anchor offsets, per-group corner coefficients,
    size_t total;                         // locations camera-major [B, Ncam, A*P] (float2)
    long long nccap;                      // cell-pointer entries per batch element
    long long nrec;                       // record slots: B * Nmaps * A * P
};

static CbLayout cb_layout(const Problem& p, size_t body_base = 0) {
    CbLayout L;
    const long long nmaps = (long long)p.Ncam * p.Nscale;
    L.maps = 256;
    L.gaps = align_up(L.maps + sizeof(CbMap) * (size_t)nmaps, 256);
    L.queues = align_up(L.gaps + sizeof(int2) * (size_t)(nmaps + 1), 256);
    L.plan_end = align_up(L.queues + sizeof(int) * (size_t)p.B * p.G, 256);
    // Disjoint valid maps fit in sum_hw rows, and (H+1)(W+1) + 1 <= 2 H W + 3 for H, W >= 1, so the cell
    // pointers of one batch element need at most 2 sum_hw + 3 Nmaps entries.
    L.nccap = (2ll * p.sum_hw + 3 * nmaps + 3) & ~3ll;  // a multiple of 4: 16-byte aligned batch slices
    L.nrec = (long long)p.B * nmaps * p.A * p.P;
    L.cellptr = body_base > L.plan_end ? body_base : L.plan_end;
    // 16 spare bytes after the cell pointers and the anchor offsets: band copies round their ends up to 16 bytes
    L.aoff = align_up(L.cellptr + sizeof(uint32_t) * (size_t)p.B * L.nccap + 16, 256);
    L.coef = align_up(L.aoff + sizeof(uint32_t) * (size_t)L.nrec + 16, 256);
    L.loct = align_up(L.coef + sizeof(float4) * (size_t)p.G * L.nrec, 256);
    L.total = align_up(L.loct + sizeof(float2) * (size_t)p.B * p.Ncam * p.A * p.P, 256);
    return L;
}

size_t cb_plan_bytes(const Problem& p) { return cb_layout(p).plan_end; }

// Shared memory of the binning block: a counter per cell (and the end), the camera's A * P cell numbers and
// the placed point indices (16 bits each), and the list of cells too full for one thread's sort.  Two blocks
// fit on an SM.
static size_t cb_bin_smem_cap(const DeviceInfo& dev) {
    return ((size_t)dev.max_smem_optin / 2 - 1024) & ~size_t(15);
}
__host__ __device__ static size_t cb_bin_fixed(long long ap) {
    return 2 * align16(2 * (size_t)ap) + align16(sizeof(uint32_t) * (size_t)(ap / 17 + 2));
}

bool cb_shape_ok(const Problem& p) {
    const long long nmaps = (long long)p.Ncam * p.Nscale;
    const long long ap = (long long)p.A * p.P;
    if (p.B < 1 || p.sum_hw < 1 || nmaps < 1 || nmaps > kCbMaxMaps || ap < 1 || ap > 65535) return false;
    if (p.Cg % 4 != 0 || p.C % 4 != 0) return false;
    const int lg = p.Cg / 4;
    if (lg > 32 || (lg & (lg - 1))) return false;
    if ((long long)p.A * p.Cg >= (1ll << 24)) return false;
    const CbLayout L = cb_layout(p);
    return L.nrec < (1ll << 31) && (long long)p.B * L.nccap < (1ll << 31);
}

// Shared memory of a reduce block: grad_out of one group, two band buffers of `nb` records and `nb` cell
// pointers each (16 + 4 + 4 bytes a slot, 8 slots of rounding each), the band planner's row starts and band
// ends.  `nb` takes what the grad_out copy leaves.
struct CbRedSmem {
    size_t buf;                // first band buffer; the second follows at buf + bsize
    size_t aoff, cptr, bsize;  // inside a buffer: coefficients at 0, anchor offsets, cell pointers
    size_t rp, bend, total;    // the planner's row starts and band ends
    __host__ __device__ CbRedSmem(int A, int Cg, int nb) {
        buf = align16(sizeof(float) * (size_t)A * Cg);
        aoff = 16 * (size_t)nb;
        cptr = aoff + align16(4 * (size_t)(nb + 8));
        bsize = cptr + align16(4 * (size_t)(nb + 8));
        rp = buf + 2 * bsize;
        bend = rp + align16(4 * (size_t)(kCbMaxRows + 2));
        total = bend + align16(4 * (size_t)kCbMaxRows);
    }
};

static int cb_band_slots(const Problem& p, const DeviceInfo& dev) {
    const CbRedSmem z(p.A, p.Cg, 0);
    const long long room = (long long)dev.max_smem_optin - 1024 - (long long)z.total - 2 * 3 * 48;
    if (room <= 0) return 0;
    return (int)((room / (2 * 24)) & ~3ll);
}

bool cb_device_ok(const Problem& p, const DeviceInfo& dev) {
    if (p.G > dev.sm_count) return false;  // at least one reduce block per group
    if (cb_band_slots(p, dev) < 256) return false;  // grad_out of one group leaves room for the band buffers
    return cb_bin_fixed((long long)p.A * p.P) + 64 <= cb_bin_smem_cap(dev);
}

size_t cb_workspace(const Problem& p, size_t body_base) { return cb_layout(p, body_base).total; }

struct CbArgs {
    const int32_t* shape;
    const int32_t* start;
    const float* loc;
    const void* w;
    const float* go;
    float* gfeat;
    unsigned char* ws;
    CbLayout L;
    int B, sum_hw, C, Ncam, Nscale, nmaps, A, P, G, Cg;
    int nlg;       // lane groups of a reduce block (light sweep tasks run at once)
    int bin_smem;  // dynamic shared memory of a binning block
    int nb;        // band buffer slots of a reduce block
    int* status;
};

// ---------------------------------------------------------------------------
// Plan (one block): validate the maps, check that the valid ones are disjoint, number their cells and work
// items, list the uncovered row ranges, clear the work queues.
// ---------------------------------------------------------------------------
// Exclusive prefix sum over n <= 4 * blockDim.x values (4 consecutive per thread) of v(i); *total = sum.
template <typename F>
__device__ __forceinline__ void plan_scan(int n, F v, int* out, int* wsum, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i0 = threadIdx.x * 4;
    int loc[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        loc[j] = (i0 + j < n) ? v(i0 + j) : 0;
        s += loc[j];
    }
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int y = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) wsum[lane] = y;
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) out[i0 + j] = run;
        run += loc[j];
    }
    if (total && threadIdx.x == 0) *total = wsum[nw - 1];
    __syncthreads();
}

__global__ void __launch_bounds__(kCbThreads) cb_plan_kernel(const CbArgs a) {
    __shared__ unsigned long long key[kCbMaxMaps];
    int* tmp = reinterpret_cast<int*>(key);  // scan output, once the sorted keys are no longer read
    __shared__ int wsum[32];
    __shared__ int s_bad, s_nvalid, s_cells;
    CbHeader* hdr = reinterpret_cast<CbHeader*>(a.ws);
    CbMap* maps = reinterpret_cast<CbMap*>(a.ws + a.L.maps);
    int2* gaps = reinterpret_cast<int2*>(a.ws + a.L.gaps);
    int* queues = reinterpret_cast<int*>(a.ws + a.L.queues);
    const int nm = a.nmaps;
    const long long ap = (long long)a.A * a.P;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int np2 = 1;
    while (np2 < nm) np2 <<= 1;
    for (int m = threadIdx.x; m < np2; m += blockDim.x) {
        unsigned long long kv = ~0ull;
        if (m < nm) {
            const MapInfo mi = load_map(a.shape, a.start, m, a.sum_hw, a.status);
            CbMap cm;
            cm.H = mi.H; cm.W = mi.W; cm.start = mi.start; cm.cbase = 0; cm.nseg = 1; cm.heavy = 0;
            cm.pad[0] = cm.pad[1] = 0;
            if (mi.W != 0) {
                const long long ncell = (long long)(mi.H + 1) * (mi.W + 1);
                const long long hw = (long long)mi.H * mi.W;
                // a warp per column where rows expect many contributions, else a lane group; columns are cut
                // into row segments until the block's lane groups (warps) have a task each
                cm.heavy = (4 * ap >= (long long)kCbHeavyPerRow * hw) ? 1 : 0;
                const int slots = cm.heavy ? kCbWarps : a.nlg;
                int nseg = slots / mi.W;
                cm.nseg = nseg < 1 ? 1 : (nseg > mi.H ? mi.H : nseg);
                if (ncell >= (long long)kNoCell ||
                    align16(4 * (size_t)(ncell + 1)) + cb_bin_fixed(ap) > (size_t)a.bin_smem ||
                    mi.H > kCbMaxRows || 2 * (mi.W + 1) + 9 > a.nb)
                    atomicOr(&s_bad, 1);  // 16-bit cells, counters fit the binning block, one row fits a band
                kv = ((unsigned long long)(unsigned)mi.start << 32) | (unsigned)m;
            }
            maps[m] = cm;
        }
        key[m] = kv;
    }
    __syncthreads();
    // valid maps in order of their first row (bitonic sort; invalid maps sort last), unless they already are
    int unsorted = 0;
    for (int m = threadIdx.x; m + 1 < np2; m += blockDim.x) unsorted |= key[m] > key[m + 1];
    unsorted = __syncthreads_or(unsorted);
    for (int k = 2; unsorted && k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int ij = i ^ j;
                if (ij > i) {
                    const unsigned long long x = key[i], y = key[ij];
                    if ((x > y) == ((i & k) == 0)) {
                        key[i] = y;
                        key[ij] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) s_nvalid = 0;
    __syncthreads();
    {
        int n = 0;
        for (int m = threadIdx.x; m < nm; m += blockDim.x) n += key[m] != ~0ull;  // valid keys come first
        if (n) atomicAdd(&s_nvalid, n);
    }
    __syncthreads();
    const int nv = s_nvalid;
    // disjointness of consecutive valid maps, and the uncovered ranges between them
    for (int i = threadIdx.x; i <= nv; i += blockDim.x) {
        int lo = 0, hi = a.sum_hw;
        if (i > 0) {
            const CbMap mp = maps[(int)(key[i - 1] & 0xffffffffu)];
            lo = mp.start + mp.H * mp.W;
        }
        if (i < nv) hi = (int)(key[i] >> 32);
        if (hi < lo) atomicOr(&s_bad, 1);  // overlap
        gaps[i] = make_int2(lo, hi > lo ? hi : lo);
    }
    // cell pointers numbered in map order (plan_scan's first barrier ends the reads of key)
    plan_scan(nm, [&](int m) { const CbMap c = maps[m]; return c.W ? (c.H + 1) * (c.W + 1) + 1 : 0; }, tmp, wsum,
              &s_cells);
    for (int m = threadIdx.x; m < nm; m += blockDim.x) maps[m].cbase = tmp[m];
    for (int q = threadIdx.x; q < a.B * a.G; q += blockDim.x) queues[q] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        hdr->ok = (s_bad == 0 && (long long)s_cells <= a.L.nccap) ? 1 : 0;
        hdr->ngaps = nv + 1;
    }
}

// ---------------------------------------------------------------------------
// Binning: one block per (batch element, map).  The camera's A * P points get their cells (0xffff when out of
// view) and are counted per cell with shared-memory atomics; the counts' prefix sums are the map's cell
// pointers; the points are placed into their cells (shared-memory atomics again) and every cell's points are
// sorted by point index (one thread per cell of up to 16 points, a warp per fuller cell), which makes the
// order inside a cell the point order whatever the atomics did.  A cell of more than kCbMaxBin points clears
// the plan's flag, which hands the whole feature gradient to the corner-slot path.  Then, in record order, each
// in-view point gets its anchor's offset a * C/G in grad_out's staged copy and, per group g, the weights of its
// four corners w_g * (x factor * y factor), in the products every other kernel forms.  Blocks past the maps
// clear the uncovered rows.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void cb_sort_small(unsigned short* seg, int n) {
    uint32_t v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = j < n ? seg[j] : 0xffffffffu;
    thread_sort<N>(v);
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j < n) seg[j] = (unsigned short)v[j];
}

template <int E>
__device__ __forceinline__ void cb_sort_warp(unsigned short* seg, int n, int lane) {
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane * E + e;
        v[e] = i < n ? seg[i] : 0xffffffffu;
    }
    warp_sort_regs<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane * E + e;
        if (i < n) seg[i] = (unsigned short)v[e];
    }
}

// Eight consecutive weights (16-byte aligned) widened to FP32, in 16-byte loads.
__device__ __forceinline__ void cb_load8(const float* p, float* v) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p)), y = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
}
__device__ __forceinline__ void cb_load8(const __nv_bfloat16* p, float* v) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
    widen(x, v, __nv_bfloat16());
}
__device__ __forceinline__ void cb_load8(const __half* p, float* v) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
    widen(x, v, __half());
}

template <typename WT>
__global__ void __launch_bounds__(kCbThreads, 2) cb_bin_kernel(const CbArgs a) {
    CbHeader* hdr = reinterpret_cast<CbHeader*>(a.ws);
    if (!hdr->ok) return;
    const CbMap* maps = reinterpret_cast<const CbMap*>(a.ws + a.L.maps);
    const long long nbm = (long long)a.B * a.nmaps;
    if ((long long)blockIdx.x >= nbm) {
        // rows of no valid map: zero gradient; the extra blocks take the uncovered ranges in turn
        const int2* gaps = reinterpret_cast<const int2*>(a.ws + a.L.gaps);
        const int zb = (int)(blockIdx.x - nbm), nzb = (int)(gridDim.x - nbm);
        const int c4 = a.C / 4;
        const int ngaps = hdr->ngaps;
        for (int gi = zb; gi < ngaps; gi += nzb) {
            const int2 gp = gaps[gi];
            const long long n = (long long)(gp.y - gp.x) * c4;
            for (int b = 0; b < a.B && n > 0; ++b) {
                float4* dst = reinterpret_cast<float4*>(a.gfeat + ((long long)b * a.sum_hw + gp.x) * a.C);
                for (long long i = threadIdx.x; i < n; i += blockDim.x) dst[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        return;
    }
    const int b = (int)(blockIdx.x / a.nmaps), m = (int)(blockIdx.x % a.nmaps);
    const CbMap mp = maps[m];
    if (mp.W == 0) return;
    const int k = m / a.Nscale, s = m - k * a.Nscale;
    const int H = mp.H, W = mp.W, W1 = W + 1;
    const int ncell = (H + 1) * W1;
    const int ap = a.A * a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Maps of few cells place their points stably with per-warp cell cursors (each warp owns a chunk of the
    // points); maps of many cells with one counter per cell and a sort of every cell afterwards.
    const size_t arrays = cb_bin_fixed(ap);
    const bool stable = align16((size_t)kCbWarps * 4 * (ncell + 1)) + arrays <= (size_t)a.bin_smem;
    const int cstride = ncell + 1;  // stable: counter of (cell c, warp w) at w * cstride + c
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);
    const size_t cbytes = align16(4 * (size_t)(stable ? kCbWarps * cstride : ncell + 1));
    unsigned short* cell = reinterpret_cast<unsigned short*>(smem + cbytes);
    unsigned short* idx = cell + align16(2 * (size_t)ap) / 2;
    uint32_t* lng = reinterpret_cast<uint32_t*>(idx + align16(2 * (size_t)ap) / 2);
    __shared__ int wsum[32];
    __shared__ int s_nlong, s_abort;
    const int chunk = (ap + kCbWarps - 1) / kCbWarps;  // stable: points of warp w are [w * chunk, ...)
    const int ncnt = stable ? kCbWarps * cstride : ncell + 1;

    for (int c = threadIdx.x; c < ncnt; c += blockDim.x) cnt[c] = 0u;
    if (threadIdx.x == 0) { s_nlong = 0; s_abort = 0; }
    __syncthreads();
    const float2* lk = reinterpret_cast<const float2*>(a.ws + a.L.loct) + ((long long)b * a.Ncam + k) * ap;
    for (int i0 = threadIdx.x; i0 < ap; i0 += 4 * blockDim.x) {
        float2 uv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            uv[u] = i < ap ? __ldg(lk + i) : make_float2(-9.f, -9.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < ap) {
                Cell cl;
                unsigned short c = kNoCell;
                if (locate(uv[u].x, uv[u].y, H, W, cl)) {
                    c = (unsigned short)((cl.y0 + 1) * W1 + cl.x0 + 1);
                    atomicAdd(cnt + (stable ? (i / chunk) * cstride + c : c), 1u);
                }
                cell[i] = c;
            }
        }
    }
    __syncthreads();
    // exclusive scan of the counters in (cell, warp) order (the end entry is 0, so it receives the total);
    // the start of cell c, its first warp's entry, is its cell pointer
    const uint32_t recbase = (uint32_t)(((long long)b * a.nmaps + m) * ap);
    {
        uint32_t* gptr = reinterpret_cast<uint32_t*>(a.ws + a.L.cellptr) + (long long)b * a.L.nccap + mp.cbase;
        const int nw = stable ? kCbWarps : 1;
        const int nent = stable ? kCbWarps * cstride - (kCbWarps - 1) : ncell + 1;  // (ncell, 0) ends the order
        const int per = (nent + blockDim.x - 1) / blockDim.x;
        const int c0 = threadIdx.x * per;
        // scan position q is (cell q / nw, warp q % nw), at counter (q % nw) * cstride + q / nw
        uint32_t sum = 0u;
        for (int j = 0; j < per && c0 + j < nent; ++j) {
            const int q = c0 + j;
            sum += cnt[(q % nw) * cstride + q / nw];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) wsum[warp] = (int)x;
        __syncthreads();
        if (warp == 0) {
            uint32_t y = (uint32_t)wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += t;
            }
            wsum[lane] = (int)y;
        }
        __syncthreads();
        uint32_t run = x - sum + (warp > 0 ? (uint32_t)wsum[warp - 1] : 0u);
        for (int j = 0; j < per && c0 + j < nent; ++j) {
            const int q = c0 + j;
            uint32_t* e = cnt + (q % nw) * cstride + q / nw;
            const uint32_t v = *e;
            *e = run;
            if (q % nw == 0) gptr[q / nw] = recbase + run;
            run += v;
        }
    }
    __syncthreads();
    if (stable) {
        // warp w walks its chunk in point order; ranks inside a batch of 32 from ballots over the cell bits
        int cbits = 1;
        while ((1 << cbits) < ncell) ++cbits;
        const unsigned lt = (1u << lane) - 1u;
        const int lo = warp * chunk, hi = min(lo + chunk, ap);
        uint32_t* cur = cnt + warp * cstride;
        for (int i0 = lo; i0 < hi; i0 += 32) {
            const int i = i0 + lane;
            const unsigned c = i < hi ? (unsigned)cell[i] : (unsigned)kNoCell;
            const bool valid = c != kNoCell;
            unsigned peers = __ballot_sync(0xffffffffu, valid);
            for (int bit = 0; bit < cbits; ++bit) {
                const unsigned mb = __ballot_sync(0xffffffffu, (c >> bit) & 1u);
                peers &= ((c >> bit) & 1u) ? mb : ~mb;
            }
            const int leader = valid ? __ffs(peers) - 1 : 0;
            uint32_t base = 0u;
            if (valid && lane == leader) {
                base = cur[c];
                cur[c] = base + (uint32_t)__popc(peers);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            if (valid) idx[base + __popc(peers & lt)] = (unsigned short)i;
        }
    } else {
        // place the points; afterwards cnt[c] is the end of cell c
        for (int i = threadIdx.x; i < ap; i += blockDim.x) {
            const unsigned short c = cell[i];
            if (c != kNoCell) idx[atomicAdd(cnt + c, 1u)] = (unsigned short)i;
        }
    }
    __syncthreads();
    // end of cell c (the start of cell c + 1): the last warp's cursor when stable, else the counter
    const uint32_t* cend = stable ? cnt + (kCbWarps - 1) * cstride : cnt;
    const int total = (int)cend[ncell - 1];
    if (!stable) {
        // point order inside every cell
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int e0 = c > 0 ? (int)cend[c - 1] : 0, n = (int)cend[c] - e0;
            if (n <= 1) continue;
            if (n <= 4) cb_sort_small<4>(idx + e0, n);
            else if (n <= 16) cb_sort_small<16>(idx + e0, n);
            else if (n <= kCbMaxBin) lng[atomicAdd(&s_nlong, 1)] = (uint32_t)c;
            else s_abort = 1;
        }
    }
    __syncthreads();
    if (s_abort) {
        if (threadIdx.x == 0) atomicExch(&hdr->ok, 0);
        return;
    }
    for (int li = warp; li < s_nlong; li += kCbWarps) {
        const int c = (int)lng[li];
        const int e0 = c > 0 ? (int)cend[c - 1] : 0, n = (int)cend[c] - e0;
        if (n <= 32) cb_sort_warp<1>(idx + e0, n, lane);
        else if (n <= 64) cb_sort_warp<2>(idx + e0, n, lane);
        else if (n <= 128) cb_sort_warp<4>(idx + e0, n, lane);
        else cb_sort_warp<8>(idx + e0, n, lane);
    }
    __syncthreads();
    // records in record order: anchor offsets and the corner coefficients of each group, two at a time
    const long long rb = (long long)recbase;
    uint32_t* aoffp = reinterpret_cast<uint32_t*>(a.ws + a.L.aoff);
    float4* coef = reinterpret_cast<float4*>(a.ws + a.L.coef);
    const WT* wp = reinterpret_cast<const WT*>(a.w);
    const long long tbase = ((long long)b * a.A * a.P) * a.Ncam + k;  // point (a, p) is tbase + (a*P + p)*Ncam
    for (int p0 = threadIdx.x; p0 < total; p0 += 2 * blockDim.x) {
        int ii[2];
        float2 uv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int pos = p0 + u * blockDim.x;
            ii[u] = pos < total ? (int)idx[pos] : -1;
            uv[u] = ii[u] >= 0 ? __ldg(lk + ii[u]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int pos = p0 + u * blockDim.x;
            if (ii[u] < 0) continue;
            const int i = ii[u];
            Cell cl;
            locate(uv[u].x, uv[u].y, H, W, cl);  // in view: it was binned
            const float ax = 1.0f - cl.fx, ay = 1.0f - cl.fy;
            const float f00 = ax * ay, f01 = cl.fx * ay, f10 = ax * cl.fy, f11 = cl.fx * cl.fy;
            aoffp[rb + pos] = (uint32_t)((i / a.P) * a.Cg);
            const WT* wrow = wp + ((tbase + (long long)i * a.Ncam) * a.Nscale + s) * a.G;
            for (int g0 = 0; g0 < a.G; g0 += 8) {
                float v[8];
                if (a.G - g0 >= 8 && ((size_t)a.G * sizeof(WT)) % 16 == 0) {
                    cb_load8(wrow + g0, v);  // 16-byte aligned: G * sizeof(WT) is a multiple of 16
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = g0 + j < a.G ? ldw(wrow + g0 + j) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (g0 + j < a.G)
                        coef[(long long)(g0 + j) * a.L.nrec + rb + pos] =
                            make_float4(v[j] * f00, v[j] * f01, v[j] * f10, v[j] * f11);
            }
        }
    }
}

// Locations camera-major: loct[b, k, i] = loc[b, i, k] with i = a * P + p (32 x 32 tiles through shared memory).
__global__ void __launch_bounds__(256) cb_loc_kernel(const CbArgs a) {
    const CbHeader* hdr = reinterpret_cast<const CbHeader*>(a.ws);
    if (!hdr->ok) return;
    __shared__ float2 tile[32][33];
    const int ap = a.A * a.P;
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32, b = blockIdx.z;
    const float2* src = reinterpret_cast<const float2*>(a.loc) + (long long)b * ap * a.Ncam;
    float2* dst = reinterpret_cast<float2*>(a.ws + a.L.loct) + (long long)b * a.Ncam * ap;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, kk = k0 + tx;
        if (i < ap && kk < a.Ncam) tile[r][tx] = __ldg(src + (long long)i * a.Ncam + kk);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int kk = k0 + r, i = i0 + tx;
        if (i < ap && kk < a.Ncam) dst[(long long)kk * ap + i] = tile[tx][r];
    }
}

// ---------------------------------------------------------------------------
// Row reduce as column sweeps.  Block j works on channel group g = j % G: it stages grad_out[b, :, group g] in
// shared memory for b = 0, 1, ... in turn and takes whole maps of (b, g) from that pair's queue.  A map's
// columns, cut into row segments, are swept top to bottom: at cell row cy a column j reads the records of its
// two cells (cy, j-1) and (cy, j), which are adjacent in record order, and adds each record once to the row it
// finishes, (cy, j), with weight x * (1 - fy), and once to the row below, (cy+1, j), with weight x * fy (x = fx
// for the left cell, 1 - fx for the right one).  The row below therefore receives its cell-row cy records
// before its own, which is the order (i-1, j-1), (i-1, j), (i, j-1), (i, j) for every row (i, j); a segment
// starting at row i0 first sweeps cell row i0 - 1 for the row below only.  Light maps: a lane group (LG lanes,
// 4 channels each) sweeps a column; heavy maps: a warp does, its lane groups taking every (32/LG)-th record of
// a cell pair and adding their partial rows with a fixed butterfly when a row is finished.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cb_fma4(float4& acc, float k, const float4& v) {
    acc.x = fmaf(k, v.x, acc.x);
    acc.y = fmaf(k, v.y, acc.y);
    acc.z = fmaf(k, v.z, acc.z);
    acc.w = fmaf(k, v.w, acc.w);
}

// cur += k * v and nxt += k' * v with packed FP32 FMAs (each half is an FP32 fma, rounded as fmaf).
__device__ __forceinline__ void cb_fma2x2(float4& cur, float4& nxt, float kc, float kn, const float4& v) {
    const float2 va = make_float2(v.x, v.y), vb = make_float2(v.z, v.w);
    const float2 kcc = make_float2(kc, kc), knn = make_float2(kn, kn);
    float2 c0 = make_float2(cur.x, cur.y), c1 = make_float2(cur.z, cur.w);
    float2 n0 = make_float2(nxt.x, nxt.y), n1 = make_float2(nxt.z, nxt.w);
    c0 = __ffma2_rn(kcc, va, c0);
    c1 = __ffma2_rn(kcc, vb, c1);
    n0 = __ffma2_rn(knn, va, n0);
    n1 = __ffma2_rn(knn, vb, n1);
    cur = make_float4(c0.x, c0.y, c1.x, c1.y);
    nxt = make_float4(n0.x, n0.y, n1.x, n1.y);
}

// One cell row of a column from a staged band: records [e, e2) every `step` (record e is coefficient slot
// e - ce and anchor-offset slot e - ae of the band); records before e1 are the left cell's (corners 1 and 3
// reach this column: coefficient .y to the finished row, .w to the row below), the others the right cell's
// (corners 0 and 2: .x and .z).  ONLY_NEXT: the finished row is not this task's.
template <bool ONLY_NEXT>
__device__ __forceinline__ void cb_step(const uint32_t* __restrict__ Ao, const float4* __restrict__ Cf,
                                        const float4* __restrict__ sgo, int l, uint32_t e, uint32_t e1, uint32_t e2,
                                        uint32_t ae, uint32_t ce, int step, float4& cur, float4& nxt) {
    for (; e + step < e2; e += 2 * step) {
        const uint32_t o0 = Ao[e - ae], o1 = Ao[e + step - ae];
        const float4 k0 = Cf[e - ce], k1 = Cf[e + step - ce];
        const bool l0 = e < e1, l1 = e + step < e1;
        const float4 v0 = sgo[(o0 >> 2) + l];
        const float4 v1 = sgo[(o1 >> 2) + l];
        if (ONLY_NEXT) {
            cb_fma4(nxt, l0 ? k0.w : k0.z, v0);
            cb_fma4(nxt, l1 ? k1.w : k1.z, v1);
        } else {
            cb_fma2x2(cur, nxt, l0 ? k0.y : k0.x, l0 ? k0.w : k0.z, v0);
            cb_fma2x2(cur, nxt, l1 ? k1.y : k1.x, l1 ? k1.w : k1.z, v1);
        }
    }
    if (e < e2) {
        const uint32_t o0 = Ao[e - ae];
        const float4 k0 = Cf[e - ce];
        const bool l0 = e < e1;
        const float4 v0 = sgo[(o0 >> 2) + l];
        if (ONLY_NEXT)
            cb_fma4(nxt, l0 ? k0.w : k0.z, v0);
        else
            cb_fma2x2(cur, nxt, l0 ? k0.y : k0.x, l0 ? k0.w : k0.z, v0);
    }
}

// Band copies of one map: band k covers image rows [i0, i1), so cell rows i0 - 1 .. i1 - 1: their records
// [rp[i0], rp[i1 + 1]) (coefficients of group g and anchor offsets) and their cell pointers, the pointer and
// offset ranges rounded out to 16 bytes.  Issued by one thread; completes on `bar`.  A band whose end carries
// kCbDirect holds rows of which even one exceeds a buffer (cells of hundreds of points in a coarse map): the
// sweep reads its records and cell pointers from the workspace itself, and its barrier phase completes with a
// plain arrival, so the buffers' phases stay in step.
struct CbBand {
    uint32_t e0, ea0, ca0;  // first record, first staged anchor-offset slot, first staged cell pointer
};

__device__ __forceinline__ CbBand cb_issue_band(const CbArgs& a, unsigned char* buf, const CbRedSmem& L,
                                                const uint32_t* rp, int i0, int i1, long long pm, int W1,
                                                const float4* coef_g, uint64_t* bar) {
    CbBand bd;
    if (i1 & kCbDirect) {  // read in place from the workspace: nothing to copy, the phase completes at once
        mbar_arrive(bar);
        bd.e0 = bd.ea0 = bd.ca0 = 0u;
        return bd;
    }
    const uint32_t e0 = rp[i0], e1 = rp[i1 + 1];
    const uint32_t ea0 = e0 & ~3u, ea1 = (e1 + 3u) & ~3u;
    const long long c0 = pm + (long long)i0 * W1, c1 = pm + (long long)(i1 + 1) * W1 + 1;
    const long long ca0 = c0 & ~3ll, ca1 = (c1 + 3) & ~3ll;
    const uint32_t bytes = (e1 - e0) * 16u + (ea1 - ea0) * 4u + (uint32_t)(ca1 - ca0) * 4u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the threads' reads of this buffer come first
    mbar_arrive_expect_tx(bar, bytes);
    const uint32_t* aoff = reinterpret_cast<const uint32_t*>(a.ws + a.L.aoff);
    const uint32_t* cptr = reinterpret_cast<const uint32_t*>(a.ws + a.L.cellptr);
    if (e1 > e0) bulk_load(buf, coef_g + e0, (e1 - e0) * 16u, bar);
    if (ea1 > ea0) bulk_load(buf + L.aoff, aoff + ea0, (ea1 - ea0) * 4u, bar);
    bulk_load(buf + L.cptr, cptr + ca0, (uint32_t)(ca1 - ca0) * 4u, bar);
    bd.e0 = e0;
    bd.ea0 = ea0;
    bd.ca0 = (uint32_t)ca0;
    return bd;
}

// The column sweeps of a band read in place: the same steps as the staged sweep in cb_reduce_kernel, with the
// records, anchor offsets and cell pointers taken from the workspace (record e, anchor offset e, cell pointer c
// at their own indices).  Kept out of line so the staged sweep, which nearly every band takes, is compiled
// as if it were alone.
template <int LG>
__device__ __noinline__ void cb_sweep_in_place(const CbArgs& a, const float4* __restrict__ coef_g,
                                               const float4* __restrict__ sgo, float* gfm, long long pm, int i0,
                                               int i1, int W, int seg, int ntask, bool heavy, int l, int lgi, int t0,
                                               int tstep, bool failed) {
    constexpr int NLGW = 32 / LG;
    const int W1 = W + 1;
    const int off = heavy ? lgi : 0, step = heavy ? NLGW : 1;
    const uint32_t* Ao = reinterpret_cast<const uint32_t*>(a.ws + a.L.aoff);
    const uint32_t* Cp = reinterpret_cast<const uint32_t*>(a.ws + a.L.cellptr);
    for (int task = t0; task < ntask && !failed; task += tstep) {
        const int sg = task / W, j = task - sg * W;
        const int r0 = i0 + sg * seg, r1 = min(r0 + seg, i1);
        if (r0 >= r1) continue;
        float4 cur = make_float4(0.f, 0.f, 0.f, 0.f), nxt = cur;
        long long ci = pm + (long long)r0 * W1 + j;  // left cell of cell row r0 - 1
#pragma unroll 2
        for (int cy = r0 - 1; cy < r1; ++cy) {
            const uint32_t q0 = Cp[ci], q1 = Cp[ci + 1], q2 = Cp[ci + 2];
            if (cy < r0) {
                cb_step<true>(Ao, coef_g, sgo, l, q0 + off, q1, q2, 0u, 0u, step, cur, nxt);
            } else {
                cb_step<false>(Ao, coef_g, sgo, l, q0 + off, q1, q2, 0u, 0u, step, cur, nxt);
                if (heavy) {
#pragma unroll
                    for (int o = LG; o < 32; o <<= 1) {
                        cur.x += __shfl_xor_sync(0xffffffffu, cur.x, o);
                        cur.y += __shfl_xor_sync(0xffffffffu, cur.y, o);
                        cur.z += __shfl_xor_sync(0xffffffffu, cur.z, o);
                        cur.w += __shfl_xor_sync(0xffffffffu, cur.w, o);
                    }
                }
                if (!heavy || lgi == 0) *reinterpret_cast<float4*>(gfm + ((long long)cy * W + j) * a.C) = cur;
            }
            cur = nxt;
            nxt = make_float4(0.f, 0.f, 0.f, 0.f);
            ci += W1;
        }
    }
}

template <int LG>
__global__ void __launch_bounds__(kCbThreads, 1) cb_reduce_kernel(const CbArgs a) {
    constexpr int NLGW = 32 / LG;  // lane groups per warp
    const CbHeader* hdr = reinterpret_cast<const CbHeader*>(a.ws);
    if (!hdr->ok) return;
    const int ngb = gridDim.x / a.G;
    if ((int)blockIdx.x >= ngb * a.G) return;
    const int g = blockIdx.x % a.G;
    const CbMap* maps = reinterpret_cast<const CbMap*>(a.ws + a.L.maps);
    int* queues = reinterpret_cast<int*>(a.ws + a.L.queues);
    const uint32_t* cellptr = reinterpret_cast<const uint32_t*>(a.ws + a.L.cellptr);
    const float4* coef_g = reinterpret_cast<const float4*>(a.ws + a.L.coef) + (long long)g * a.L.nrec;
    const CbRedSmem L(a.A, a.Cg, a.nb);
    extern __shared__ __align__(16) unsigned char smem[];
    float4* sgo = reinterpret_cast<float4*>(smem);
    unsigned char* const buf0 = smem + L.buf;  // band buffer bf is buf0 + bf * L.bsize
    uint32_t* rp = reinterpret_cast<uint32_t*>(smem + L.rp);
    int* bend = reinterpret_cast<int*>(smem + L.bend);
    __shared__ uint64_t mbar[2];
    __shared__ CbBand s_band[2];
    __shared__ int s_item[2], s_nb, s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lgi = lane / LG, l = lane % LG;
    const int lgid = warp * NLGW + lgi;
    const int nlg = kCbWarps * NLGW;
    const int cg4 = a.Cg / 4;
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        s_fail = 0;
    }
    uint32_t ph0 = 0u, ph1 = 0u;  // parity of each buffer's barrier

    for (int b = 0; b < a.B; ++b) {
        // stage grad_out[b, :, group g]
        const float4* gsrc = reinterpret_cast<const float4*>(a.go + (long long)b * a.A * a.C + g * a.Cg);
        for (int i = threadIdx.x; i < a.A * cg4; i += blockDim.x) {
            const int aa = i / cg4, q = i - aa * cg4;
            sgo[i] = __ldg(gsrc + (long long)aa * (a.C / 4) + q);
        }
        int* queue = queues + b * a.G + g;
        if (threadIdx.x == 0) s_item[0] = atomicAdd(queue, 1);
        __syncthreads();
        float* gfb = a.gfeat + (long long)b * a.sum_hw * a.C + g * a.Cg + l * 4;
        for (int cur_slot = 0;; cur_slot ^= 1) {
            const int m = s_item[cur_slot];
            if (m >= a.nmaps) break;
            if (threadIdx.x == 0) s_item[cur_slot ^ 1] = atomicAdd(queue, 1);  // the next map, fetched meanwhile
            const CbMap mp = maps[m];
            if (mp.W != 0) {
                const int H = mp.H, W = mp.W, W1 = W + 1;
                const long long pm = (long long)b * a.L.nccap + mp.cbase;  // the map's cell pointers
                // record starts of the cell rows (cell row index r = cy + 1), then the bands
                for (int r = threadIdx.x; r <= H + 1; r += blockDim.x) rp[r] = __ldg(cellptr + pm + (long long)r * W1);
                __syncthreads();
                if (warp == 0) {
                    int i0 = 0, nb = 0;
                    while (i0 < H) {
                        int i1 = i0;
                        for (int base = 1;; base += 32) {  // the band grows while it fits (a prefix of candidates)
                            const int c = i0 + base + lane;
                            const bool fits = c <= H && (int)(rp[c + 1] - rp[i0]) <= a.nb - 8 &&
                                              (long long)(c - i0 + 1) * W1 + 9 <= a.nb;
                            const unsigned bal = __ballot_sync(0xffffffffu, fits);
                            if (bal) i1 = i0 + base + 31 - __clz(bal);
                            if (bal != 0xffffffffu) break;
                        }
                        int flag = 0;
                        if (i1 == i0) {
                            // row i0 alone (cell rows i0 - 1 and i0) exceeds a buffer: it and the rows after it that
                            // do too form one band read in place
                            i1 = i0 + 1;
                            while (i1 < H && (int)(rp[i1 + 2] - rp[i1]) > a.nb - 8) ++i1;
                            flag = kCbDirect;
                        }
                        if (lane == 0) bend[nb] = i1 | flag;
                        ++nb;
                        i0 = i1;
                    }
                    if (lane == 0) s_nb = nb;
                }
                __syncthreads();
                const int nb = s_nb;
                if (threadIdx.x == 0) {
                    for (int k = 0; k < 2 && k < nb; ++k)
                        s_band[k] = cb_issue_band(a, buf0 + k * L.bsize, L, rp, k ? bend[k - 1] & ~kCbDirect : 0,
                                                  bend[k], pm, W1, coef_g, &mbar[k]);
                }
                float* gfm = gfb + (long long)mp.start * a.C;
                const bool heavy = mp.heavy != 0;
                for (int k = 0; k < nb; ++k) {
                    const int bf = k & 1;
                    const uint32_t par = bf ? ph1 : ph0;
                    if (threadIdx.x == 0 && !mbar_wait_first(&mbar[bf], par)) {
                        s_fail = 1;
                        raise_status(a.status, MSDA_ERR_TIMEOUT);
                        mbar_wait_drain(&mbar[bf], par);  // the copies in flight land before the buffer is reused
                    }
                    __syncthreads();
                    if (bf) ph1 ^= 1u; else ph0 ^= 1u;
                    const int i0 = k ? bend[k - 1] & ~kCbDirect : 0, i1 = bend[k] & ~kCbDirect;
                    const bool direct = (bend[k] & kCbDirect) != 0;
                    const CbBand bd = s_band[bf];
                    const unsigned char* bb = buf0 + bf * L.bsize;
                    const int R = i1 - i0;
                    const int slots = heavy ? kCbWarps : nlg;
                    int S = slots / W;
                    S = S < 1 ? 1 : (S > R ? R : S);
                    const int seg = (R + S - 1) / S;
                    const int ntask = W * S;
                    const int t0 = heavy ? warp : lgid, tstep = heavy ? kCbWarps : nlg;
                    const int off = heavy ? lgi : 0, step = heavy ? NLGW : 1;
                    const bool failed = s_fail != 0;
                    if (direct) {
                        cb_sweep_in_place<LG>(a, coef_g, sgo, gfm, pm, i0, i1, W, seg, ntask, heavy, l, lgi,
                                              t0, tstep, failed);
                    } else {
                        const float4* Cf = reinterpret_cast<const float4*>(bb);
                        const uint32_t* Ao = reinterpret_cast<const uint32_t*>(bb + L.aoff);
                        const uint32_t* Cp = reinterpret_cast<const uint32_t*>(bb + L.cptr);
                        for (int task = t0; task < ntask && !failed; task += tstep) {
                            const int sg = task / W, j = task - sg * W;
                            const int r0 = i0 + sg * seg, r1 = min(r0 + seg, i1);
                            if (r0 >= r1) continue;
                            float4 cur = make_float4(0.f, 0.f, 0.f, 0.f), nxt = cur;
                            // left cell of cell row r0 - 1 (cell row index r0), as a slot of the staged pointers
                            int ci = (int)(pm - (long long)bd.ca0) + r0 * W1 + j;
#pragma unroll 2
                            for (int cy = r0 - 1; cy < r1; ++cy) {
                                const uint32_t q0 = Cp[ci], q1 = Cp[ci + 1], q2 = Cp[ci + 2];
                                if (cy < r0) {
                                    cb_step<true>(Ao, Cf, sgo, l, q0 + off, q1, q2, bd.ea0, bd.e0, step, cur, nxt);
                                } else {
                                    cb_step<false>(Ao, Cf, sgo, l, q0 + off, q1, q2, bd.ea0, bd.e0, step, cur, nxt);
                                    if (heavy) {
#pragma unroll
                                        for (int o = LG; o < 32; o <<= 1) {
                                            cur.x += __shfl_xor_sync(0xffffffffu, cur.x, o);
                                            cur.y += __shfl_xor_sync(0xffffffffu, cur.y, o);
                                            cur.z += __shfl_xor_sync(0xffffffffu, cur.z, o);
                                            cur.w += __shfl_xor_sync(0xffffffffu, cur.w, o);
                                        }
                                    }
                                    if (!heavy || lgi == 0)
                                        *reinterpret_cast<float4*>(gfm + ((long long)cy * W + j) * a.C) = cur;
                                }
                                cur = nxt;
                                nxt = make_float4(0.f, 0.f, 0.f, 0.f);
                                ci += W1;
                            }
                        }
                    }
                    __syncthreads();  // the buffer is free again
                    if (threadIdx.x == 0 && k + 2 < nb)
                        s_band[bf] = cb_issue_band(a, buf0 + bf * L.bsize, L, rp, bend[k + 1] & ~kCbDirect,
                                                   bend[k + 2], pm, W1, coef_g, &mbar[bf]);
                }
            }
            __syncthreads();  // every thread has read s_item[cur_slot] and finished the map
        }
        __syncthreads();  // every warp is done with this batch element's grad_out
    }
}

using CbBinKernel = void (*)(const CbArgs);
using CbRedKernel = void (*)(const CbArgs);

static CbRedKernel cb_red_pick(int lg) {
    switch (lg) {
        case 1: return cb_reduce_kernel<1>;
        case 2: return cb_reduce_kernel<2>;
        case 4: return cb_reduce_kernel<4>;
        case 8: return cb_reduce_kernel<8>;
        case 16: return cb_reduce_kernel<16>;
        case 32: return cb_reduce_kernel<32>;
    }
    return nullptr;
}

// Enqueue the plan, binning and reduce kernels.  The plan's flag (the first int of `ws`) tells the corner-slot
// kernels launched after these whether they have to run.
msda_status launch_backward_cb(const Problem& p, const float* grad_out, float* grad_feat, void* ws,
                               size_t body_base, cudaStream_t stream) {
    DeviceInfo dev;
    msda_status st = device_info(&dev);
    if (st != MSDA_OK) return st;
    CbArgs a;
    a.shape = p.shape; a.start = p.start; a.loc = p.loc; a.w = p.w; a.go = grad_out; a.gfeat = grad_feat;
    a.ws = reinterpret_cast<unsigned char*>(ws);
    a.L = cb_layout(p, body_base);
    a.B = p.B; a.sum_hw = p.sum_hw; a.C = p.C; a.Ncam = p.Ncam; a.Nscale = p.Nscale; a.nmaps = p.Ncam * p.Nscale;
    a.A = p.A; a.P = p.P; a.G = p.G; a.Cg = p.Cg;
    a.nlg = kCbWarps * (32 / (p.Cg / 4));
    a.bin_smem = (int)cb_bin_smem_cap(dev);
    a.nb = cb_band_slots(p, dev);
    a.status = dev.status;
    CbBinKernel bin = p.w_t == MSDA_F32 ? cb_bin_kernel<float>
                    : p.w_t == MSDA_BF16 ? cb_bin_kernel<__nv_bfloat16> : cb_bin_kernel<__half>;
    CbRedKernel red = cb_red_pick(p.Cg / 4);
    if (!red) return fail(MSDA_ERR_UNSUPPORTED, "msda_backward: no cell-binned reduce for C/G = %d", p.Cg);
    const size_t bin_smem = (size_t)a.bin_smem;
    const size_t red_smem = CbRedSmem(p.A, p.Cg, a.nb).total;
    if ((st = ensure_smem((const void*)bin, bin_smem, dev)) != MSDA_OK) return st;
    if ((st = ensure_smem((const void*)red, red_smem, dev)) != MSDA_OK) return st;
    cb_plan_kernel<<<1, kCbThreads, 0, stream>>>(a);
    {
        const dim3 lg((unsigned)((p.A * p.P + 31) / 32), (unsigned)((p.Ncam + 31) / 32), (unsigned)p.B);
        cb_loc_kernel<<<lg, 256, 0, stream>>>(a);
    }
    const long long nbm = (long long)p.B * a.nmaps;
    bin<<<(unsigned)(nbm + 16), kCbThreads, bin_smem, stream>>>(a);
    const int ngb = dev.sm_count / p.G;
    red<<<(unsigned)(ngb * p.G), kCbThreads, red_smem, stream>>>(a);
    return check_launch("msda_backward cell-binned");
}

// The first-wait poll limit of this file's band waits (msda_debug_set_wait_limit).
msda_status cb_set_wait_limit(long long polls) {
    if (polls < 0) polls = kSpinLimit;
    const cudaError_t e = cudaMemcpyToSymbol(g_first_wait_limit, &polls, sizeof(polls));
    return e == cudaSuccess ? MSDA_OK : fail(MSDA_ERR_CUDA, "msda_debug_set_wait_limit: %s", cudaGetErrorString(e));
}

}  // namespace msda
