// Binning and ordering of Sec. 3.2: points are sorted by depth and, per
// screen tile, composited front to back; only points within the cutoff of
// a pixel are considered, so each point is listed only in the tiles its
// cutoff disc touches.
//
// Pipeline (all counts live on the device; grids are sized by capacity and
// idle blocks exit, so the chain has no host synchronisation):
//   1. compact_visible  : scan of the visibility flags -> (depth bits, pv)
//   2. radix_sort_pairs : stable LSD radix sort by fp32 depth bits
//   3. emit_pairs       : scan of tile counts in depth order, writing one
//                         (global tile id, pv) pair per covered tile
//   4. radix_sort_pairs : stable LSD radix sort by tile id only; stability
//                         keeps depth order, so the result is ordered by
//                         (tile, depth, pv) -- the order Eqs. 6-7 need
//   5. tile_ranges      : [start, end) of every tile in the sorted list
//
// Scans are reduce-then-scan (three kernels, no inter-block waiting).  The
// radix pass ranks keys stably inside a block with warp match/ballot and a
// shared-memory reorder so that the scatter writes contiguous runs.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS; // 4096
constexpr int SCAN_WARPS = SCAN_THREADS / 32;

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS; // 4096
constexpr int SORT_WARPS = SORT_THREADS / 32;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t dev_count(const uint32_t *n_dev, int64_t cap)
{
    if (!n_dev) return cap;
    const int64_t n = (int64_t)*n_dev;
    return n < cap ? n : cap;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---------------------------------------------------------------- scans
// Load: uint32_t operator()(int64_t i) for i < n.
template <class Load>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_kernel(Load ld, const uint32_t *n_dev, int64_t cap, uint32_t *block_sums)
{
    const int64_t n = dev_count(n_dev, cap);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t acc = 0;
    if (base < n) {
#pragma unroll 4
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const int64_t i = base + k * SCAN_THREADS + threadIdx.x;
            if (i < n) acc += ld(i);
        }
    }
    acc = __reduce_add_sync(0xffffffffu, acc);
    __shared__ uint32_t s_w[SCAN_WARPS];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_WARPS; ++w) t += s_w[w];
        block_sums[blockIdx.x] = t;
    }
}

// One block: exclusive scan of block_sums[0..nb) in place; the total goes to
// *total (64-bit) when non-NULL; sets ST_COUNT_OVERFLOW if it exceeds 2^32-1.
__global__ void __launch_bounds__(1024)
scan_top_kernel(uint32_t *block_sums, int64_t nb, unsigned long long *total, uint32_t *status)
{
    __shared__ unsigned long long s_w[32];
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = lo + per < nb ? lo + per : nb;
    unsigned long long acc = 0;
    for (int64_t j = lo; j < hi; ++j) acc += block_sums[j];
    // block exclusive scan of acc (64-bit)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long v = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long x = lane < nw ? s_w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < nw) s_w[lane] = x; // inclusive per warp
    }
    __syncthreads();
    unsigned long long run = (w > 0 ? s_w[w - 1] : 0ull) + v - acc;
    for (int64_t j = lo; j < hi; ++j) {
        const uint32_t x = block_sums[j];
        block_sums[j] = (uint32_t)run;
        run += x;
    }
    if (threadIdx.x == blockDim.x - 1) {
        const unsigned long long tot = s_w[(blockDim.x >> 5) - 1];
        if (total) *total = tot;
        if (status && tot > 0xffffffffull) atomicOr(status, ST_COUNT_OVERFLOW);
    }
}

// Act: void operator()(int64_t i, uint32_t exclusive_prefix, uint32_t value).
template <class Load, class Act>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_down_kernel(Load ld, Act act, const uint32_t *n_dev, int64_t cap,
                 const uint32_t *block_offsets)
{
    const int64_t n = dev_count(n_dev, cap);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    if (base >= n) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wbase = base + (int64_t)w * 32 * SCAN_ITEMS;
    uint32_t val[SCAN_ITEMS], pre[SCAN_ITEMS];
    uint32_t carry = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const uint32_t v = i < n ? ld(i) : 0u;
        const uint32_t inc = warp_incl_scan(v);
        val[r] = v;
        pre[r] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __shared__ uint32_t s_w[SCAN_WARPS];
    if (lane == 0) s_w[w] = carry;
    __syncthreads();
    uint32_t woff = block_offsets[blockIdx.x];
    for (int j = 0; j < w; ++j) woff += s_w[j];
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < n) act(i, woff + pre[r], val[r]);
    }
}

template <class Load, class Act>
void run_scan(Load ld, Act act, const uint32_t *n_dev, int64_t cap, void *temp,
              unsigned long long *total, uint32_t *status, cudaStream_t s)
{
    if (cap <= 0) return;
    const int64_t nb = (cap + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t *sums = (uint32_t *)temp;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(ld, n_dev, cap, sums);
    scan_top_kernel<<<1, 1024, 0, s>>>(sums, nb, total, status);
    scan_down_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(ld, act, n_dev, cap, sums);
    count_launches(3);
}

// ----------------------------------------------------------- functors
struct LoadVisible {
    const uint32_t *ntiles;
    __device__ uint32_t operator()(int64_t i) const { return ntiles[i] > 0 ? 1u : 0u; }
};
struct ActCompact {
    const uint32_t *ntiles, *zbits;
    uint32_t *keys, *vals;
    __device__ void operator()(int64_t i, uint32_t pos, uint32_t v) const
    {
        if (v) {
            keys[pos] = zbits[i];
            vals[pos] = (uint32_t)i;
        }
    }
};
struct LoadU32 {
    const uint32_t *p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct ActStore {
    uint32_t *p;
    __device__ void operator()(int64_t i, uint32_t pos, uint32_t) const { p[i] = pos; }
};
struct LoadTileCount {
    const uint32_t *sorted_pv, *ntiles;
    __device__ uint32_t operator()(int64_t j) const { return ntiles[sorted_pv[j]]; }
};
struct ActEmit {
    const uint32_t *sorted_pv;
    const uint2 *rect;
    const DevView *views;
    int32_t n_views;
    uint32_t *keys, *vals;
    int64_t cap;
    uint32_t *status;
    __device__ void operator()(int64_t j, uint32_t pos, uint32_t nt) const
    {
        const uint32_t pv = sorted_pv[j];
        // view of this point-view: last view with pv_base <= pv
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (views[mid].pv_base <= (int64_t)pv) lo = mid; else hi = mid - 1;
        }
        const DevView &V = views[lo];
        const uint2 rc = rect[pv];
        const int tx0 = rc.x & 0xffff, ty0 = rc.x >> 16, tx1 = rc.y & 0xffff, ty1 = rc.y >> 16;
        if ((int64_t)pos + nt > cap) {
            atomicOr(status, ST_PAIR_OVERFLOW);
            return;
        }
        uint32_t q = pos;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                keys[q] = V.tile_base + (uint32_t)(ty * V.tiles_x + tx);
                vals[q] = pv;
                ++q;
            }
    }
};

// ----------------------------------------------------------- radix sort
__global__ void __launch_bounds__(SORT_THREADS)
radix_hist_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_dev, int64_t cap,
                  int shift, uint32_t *__restrict__ hist, int64_t nb)
{
    __shared__ uint32_t s_h[SORT_WARPS][RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < SORT_WARPS * RADIX; j += SORT_THREADS) (&s_h[0][0])[j] = 0;
    __syncthreads();
    const int64_t n = dev_count(n_dev, cap);
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE + (int64_t)w * 32 * SORT_ITEMS;
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const uint32_t d = i < n ? (keys[i] >> shift) & (RADIX - 1) : RADIX;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < RADIX && (peers & lanemask_lt()) == 0) s_h[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) {
        uint32_t t = 0;
        for (int j = 0; j < SORT_WARPS; ++j) t += s_h[j][d];
        hist[(int64_t)d * nb + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(SORT_THREADS)
radix_scatter_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                     uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                     const uint32_t *n_dev, int64_t cap, int shift,
                     const uint32_t *__restrict__ hist, int64_t nb)
{
    __shared__ uint32_t s_k[SORT_TILE];
    __shared__ uint32_t s_v[SORT_TILE];
    __shared__ uint32_t s_wh[SORT_WARPS][RADIX];
    __shared__ uint32_t s_dbase[RADIX];
    __shared__ uint32_t s_gbase[RADIX];
    __shared__ uint32_t s_scan[SORT_WARPS];
    const int64_t n = dev_count(n_dev, cap);
    const int64_t blk = (int64_t)blockIdx.x * SORT_TILE;
    if (blk >= n) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < SORT_WARPS * RADIX; j += SORT_THREADS) (&s_wh[0][0])[j] = 0;
    __syncthreads();
    const int64_t base = blk + (int64_t)w * 32 * SORT_ITEMS;
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? keys_in[i] : 0u;
        val[r] = ok ? vals_in[i] : 0u;
        const uint32_t d = ok ? (key[r] >> shift) & (RADIX - 1) : RADIX;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = d < RADIX ? s_wh[w][d] : 0u;
        __syncwarp();
        if (d < RADIX && (peers & lt) == 0) s_wh[w][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, digit total, global base
    uint32_t dtot = 0;
    {
        const int d = threadIdx.x; // SORT_THREADS == RADIX
        for (int j = 0; j < SORT_WARPS; ++j) {
            const uint32_t t = s_wh[j][d];
            s_wh[j][d] = dtot;
            dtot += t;
        }
        s_gbase[d] = hist[(int64_t)d * nb + blockIdx.x];
    }
    // block exclusive scan of dtot over the 256 digits
    {
        const uint32_t inc = warp_incl_scan(dtot);
        if (lane == 31) s_scan[w] = inc;
        __syncthreads();
        uint32_t off = 0;
        for (int j = 0; j < w; ++j) off += s_scan[j];
        s_dbase[threadIdx.x] = off + inc - dtot;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & (RADIX - 1);
            const uint32_t loc = s_dbase[d] + s_wh[w][d] + rank[r];
            s_k[loc] = key[r];
            s_v[loc] = val[r];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - blk < SORT_TILE ? n - blk : SORT_TILE);
    for (int j = threadIdx.x; j < cnt; j += SORT_THREADS) {
        const uint32_t k = s_k[j];
        const uint32_t d = (k >> shift) & (RADIX - 1);
        const uint32_t g = s_gbase[d] + (uint32_t)j - s_dbase[d];
        keys_out[g] = k;
        vals_out[g] = s_v[j];
    }
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                   int64_t cap, uint2 *__restrict__ ranges, uint32_t n_tiles)
{
    const int64_t n = dev_count(n_dev, cap);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t t = keys[j];
    if (t >= n_tiles) return;
    if (j == 0 || keys[j - 1] != t) ranges[t].x = (uint32_t)j;
    if (j == n - 1 || keys[j + 1] != t) ranges[t].y = (uint32_t)(j + 1);
}

} // namespace

size_t scan_temp_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(nb > 0 ? nb : 1) * sizeof(uint32_t);
}

void launch_compact_visible(const uint32_t *ntiles, const uint32_t *zbits, int64_t n_pv,
                            uint32_t *keys_out, uint32_t *vals_out, uint32_t *n_vis, void *temp,
                            cudaStream_t s)
{
    // the visible count comes from the preprocess counters; here only the
    // positions are needed
    (void)n_vis;
    run_scan(LoadVisible{ntiles}, ActCompact{ntiles, zbits, keys_out, vals_out}, nullptr, n_pv,
             temp, nullptr, nullptr, s);
}

size_t radix_temp_bytes(int64_t cap)
{
    const int64_t nb = (cap + SORT_TILE - 1) / SORT_TILE;
    const int64_t hist = (nb > 0 ? nb : 1) * RADIX;
    return (size_t)hist * sizeof(uint32_t) + scan_temp_bytes(hist);
}

void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *&keys_alt, uint32_t *&vals_alt,
                      const uint32_t *n_dev, int64_t cap, int key_bits, void *temp,
                      cudaStream_t s)
{
    if (cap <= 0) return;
    const int64_t nb = (cap + SORT_TILE - 1) / SORT_TILE;
    uint32_t *hist = (uint32_t *)temp;
    void *scan_tmp = hist + nb * RADIX;
    for (int shift = 0; shift < key_bits; shift += RADIX_BITS) {
        radix_hist_kernel<<<(unsigned)nb, SORT_THREADS, 0, s>>>(keys, n_dev, cap, shift, hist, nb);
        run_scan(LoadU32{hist}, ActStore{hist}, nullptr, nb * RADIX, scan_tmp, nullptr, nullptr, s);
        radix_scatter_kernel<<<(unsigned)nb, SORT_THREADS, 0, s>>>(keys, vals, keys_alt, vals_alt,
                                                                   n_dev, cap, shift, hist, nb);
        count_launches(2);
        uint32_t *tk = keys, *tv = vals;
        keys = keys_alt;
        vals = vals_alt;
        keys_alt = tk;
        vals_alt = tv;
    }
}

void launch_emit_pairs(const Batch &b, const DevOpts &o, const uint32_t *sorted_pv,
                       const uint32_t *n_vis, int64_t cap_vis, const uint32_t *ntiles,
                       const uint2 *rect, uint32_t *keys, uint32_t *vals, int64_t cap_pairs,
                       uint32_t *status, void *temp, cudaStream_t s)
{
    (void)o;
    run_scan(LoadTileCount{sorted_pv, ntiles},
             ActEmit{sorted_pv, rect, b.views, b.n_views, keys, vals, cap_pairs, status}, n_vis,
             cap_vis, temp, nullptr, status, s);
}

void launch_tile_ranges(const uint32_t *keys, const uint32_t *n_pairs, int64_t cap_pairs,
                        uint2 *ranges, uint32_t n_tiles, cudaStream_t s)
{
    if (cap_pairs <= 0) return;
    const int th = 256;
    const int64_t nb = (cap_pairs + th - 1) / th;
    tile_ranges_kernel<<<(unsigned)nb, th, 0, s>>>(keys, n_pairs, cap_pairs, ranges, n_tiles);
    count_launches(1);
}

} // namespace pbr
