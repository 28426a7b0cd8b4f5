// Binning and ordering of Sec. 3.2: points are sorted by depth and, per
// screen tile, composited front to back; only points within the cutoff of
// a pixel are considered, so each point is listed only in the tiles its
// cutoff disc touches.
//
// Pipeline (all counts live on the device; grids are sized by capacity and
// idle blocks exit, so the chain has no host synchronisation):
//   1. compact_visible  : scan of the visibility flags -> (depth bits, pv);
//                         skipped when most point-views are visible: the
//                         sort then takes every point-view, the invisible
//                         ones keyed behind every depth
//   2. radix_sort_pairs : stable LSD radix sort by fp32 depth bits
//   3. emit_pairs       : scan of tile counts in depth order, writing one
//                         (global tile id, pv) pair per covered tile
//   4. radix_sort_pairs : stable LSD radix sort by tile id only; stability
//                         keeps depth order, so the result is ordered by
//                         (tile, depth, pv) -- the order Eqs. 6-7 need
//   5. tile_ranges      : [start, end) of every tile in the sorted list
//
// Scans are reduce-then-scan (three kernels, no inter-block waiting).  The
// radix pass ranks keys stably inside a block with per-warp peer masks
// (shared-memory OR) and shared atomics, and reorders them in shared memory
// so that the scatter writes contiguous runs.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS; // 4096
constexpr int SCAN_WARPS = SCAN_THREADS / 32;

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
// ----------------------------------------------------------- radix sort
// One LSD pass over a digit of `width` <= RB bits of (key - key_lo) at
// `shift`.  Keys are loaded before any warp-synchronous work so that all of a
// thread's loads are in flight together.
constexpr int RB = 9;
constexpr int RBINS = 1 << RB;

// Digit of min(key - key_lo, key_max): keys above the range (the marker of
// an invisible point-view) all take the largest value.
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint32_t key_lo, uint32_t key_max,
                                             int shift, uint32_t mask)
{
    const uint32_t k = key - key_lo;
    return ((k < key_max ? k : key_max) >> shift) & mask;
}

// Peers of each lane: lanes holding the same digit (digits < 2^10, the
// out-of-range marker RBINS included), built from ballots.  full: no lane
// holds the marker (warp-uniform), so its bit needs no ballot.
__device__ __forceinline__ uint32_t peers_by_ballot(uint32_t d, bool full)
{
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < RB; ++bit) {
        const uint32_t m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
        peers &= ((d >> bit) & 1u) ? m : ~m;
    }
    if (!full) {
        const uint32_t m = __ballot_sync(0xffffffffu, (d >> RB) & 1u);
        peers &= ((d >> RB) & 1u) ? m : ~m;
    }
    return peers;
}

// Digit histograms of HIST_TILES consecutive scatter tiles (SORT_TILE keys
// each) per block: shared-memory atomics into one counter per (tile,
// digit), written out as hist[digit][tile].
constexpr int HIST_TILES = 4;

__global__ void __launch_bounds__(SORT_THREADS)
radix_hist_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_dev, int64_t cap,
                  uint32_t key_lo, uint32_t key_max, int shift, int width,
                  uint32_t *__restrict__ hist, int64_t nb)
{
    __shared__ uint32_t s_h[HIST_TILES][RBINS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < HIST_TILES * RBINS; j += SORT_THREADS) (&s_h[0][0])[j] = 0;
    const int64_t n = dev_count(n_dev, cap);
    const uint32_t mask = (1u << width) - 1u;
    const int64_t t0 = (int64_t)blockIdx.x * HIST_TILES;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < HIST_TILES; ++k) {
        const int64_t base = (t0 + k) * SORT_TILE + (int64_t)w * 32 * SORT_ITEMS;
        uint32_t d[SORT_ITEMS];
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; ++r) {
            const int64_t i = base + r * 32 + lane;
            d[r] = i < n ? digit_of(keys[i], key_lo, key_max, shift, mask) : (uint32_t)RBINS;
        }
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; ++r)
            if (d[r] < RBINS) atomicAdd(&s_h[k][d[r]], 1u);
    }
    __syncthreads();
    const int bins = 1 << width;
    for (int k = 0; k < HIST_TILES && t0 + k < nb; ++k)
        for (int dd = threadIdx.x; dd < bins; dd += SORT_THREADS)
            hist[(int64_t)dd * nb + t0 + k] = s_h[k][dd];
}

constexpr size_t SCATTER_SMEM = sizeof(uint32_t) * (3 * SORT_TILE + SORT_WARPS * RBINS + 3 * RBINS +
                                                    SORT_WARPS);

__global__ void __launch_bounds__(SORT_THREADS)
radix_scatter_kernel(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                     uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                     const uint32_t *n_dev, int64_t cap, uint32_t key_lo, uint32_t key_max,
                     int shift, int width, const uint32_t *__restrict__ hist, int64_t nb,
                     bool index_vals)
{
    extern __shared__ uint32_t s_mem[];
    uint32_t *s_k = s_mem;                               // [SORT_TILE] keys, ranked order
    uint32_t *s_v = s_k + SORT_TILE;                     // [SORT_TILE] values, ranked order
    uint32_t *s_vin = s_v + SORT_TILE;                   // [SORT_TILE] values, input order
    uint32_t(*s_wh)[RBINS] = (uint32_t(*)[RBINS])(s_vin + SORT_TILE); // [warps][RBINS]
    uint32_t *s_tot = s_vin + SORT_TILE + SORT_WARPS * RBINS;
    uint32_t *s_dbase = s_tot + RBINS;
    uint32_t *s_gbase = s_dbase + RBINS;
    uint32_t *s_scan = s_gbase + RBINS;
    const int64_t n = dev_count(n_dev, cap);
    const int64_t blk = (int64_t)blockIdx.x * SORT_TILE;
    if (blk >= n) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t mask = (1u << width) - 1u;
    const int bins = 1 << width;
    // the block's global digit bases, loaded now so that their latency
    // hides behind the ranking (digits threadIdx.x + k SORT_THREADS)
    constexpr int PER_T = RBINS / SORT_THREADS;
    uint32_t gb[PER_T];
#pragma unroll
    for (int k = 0; k < PER_T; ++k) {
        const int dd = threadIdx.x + k * SORT_THREADS;
        gb[k] = dd < bins ? hist[(int64_t)dd * nb + blockIdx.x] : 0u;
    }
    for (int j = threadIdx.x; j < SORT_WARPS * RBINS; j += SORT_THREADS) (&s_wh[0][0])[j] = 0;
    // the warps' peer masks (one word per digit) live in s_k, free until the
    // placement below
    uint32_t *s_pm = s_k + w * RBINS;
    for (int j = threadIdx.x; j < SORT_TILE; j += SORT_THREADS) s_k[j] = 0;
    const int64_t base = blk + (int64_t)w * 32 * SORT_ITEMS;
    uint32_t key[SORT_ITEMS], rank[SORT_ITEMS];
    const int lbase = w * 32 * SORT_ITEMS + lane; // local index of round 0
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? keys_in[i] : 0u;
        s_vin[lbase + r * 32] = ok ? (index_vals ? (uint32_t)i : vals_in[i]) : 0u;
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    const bool full = blk + SORT_TILE <= n; // every key of the block is in range
    {
        // stable rank inside the warp: the lanes holding the same digit (each
        // lane ORs its bit into its digit's word of the warp's peer masks and
        // reads the word back; with out-of-range keys, from ballots), the
        // group leader's shared-memory atomic on the warp's digit counter
        // (one warp's shared atomics execute in program order, so rounds stay
        // ordered) and its reset of the peer word, then the broadcast of each
        // group's base
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; ++r) {
            const bool ok = base + r * 32 + lane < n;
            const uint32_t d = ok ? digit_of(key[r], key_lo, key_max, shift, mask) : (uint32_t)RBINS;
            uint32_t peers;
            if (full || __all_sync(0xffffffffu, ok)) {
                atomicOr(&s_pm[d], 1u << lane);
                __syncwarp();
                peers = s_pm[d];
                __syncwarp();
            } else {
                peers = peers_by_ballot(d, false);
            }
            uint32_t old = 0;
            if (d < RBINS && (peers & lt) == 0) {
                old = atomicAdd(&s_wh[w][d], (uint32_t)__popc(peers));
                s_pm[d] = 0;
            }
            __syncwarp(); // peer words clear before the next round's ORs
            rank[r] = (uint32_t)(__ffs(peers) - 1) | ((uint32_t)__popc(peers & lt) << 5) | (old << 10);
        }
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; ++r) {
            const uint32_t packed = rank[r];
            const uint32_t base_r = __shfl_sync(0xffffffffu, packed >> 10, packed & 31);
            rank[r] = base_r + ((packed >> 5) & 31);
        }
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, digit total, global base
#pragma unroll
    for (int k = 0; k < PER_T; ++k) {
        const int dd = threadIdx.x + k * SORT_THREADS;
        uint32_t t = 0;
        if (dd < bins) {
#pragma unroll
            for (int j = 0; j < SORT_WARPS; ++j) {
                const uint32_t x = s_wh[j][dd];
                s_wh[j][dd] = t;
                t += x;
            }
            s_gbase[dd] = gb[k];
        }
        s_tot[dd] = t;
    }
    __syncthreads();
    // block exclusive scan of the digit totals (RBINS / SORT_THREADS per thread)
    {
        constexpr int PER = RBINS / SORT_THREADS;
        uint32_t loc[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            loc[q] = s_tot[threadIdx.x * PER + q];
            sum += loc[q];
        }
        const uint32_t inc = warp_incl_scan(sum);
        if (lane == 31) s_scan[w] = inc;
        __syncthreads();
        uint32_t off = inc - sum;
        for (int j = 0; j < w; ++j) off += s_scan[j];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            s_dbase[threadIdx.x * PER + q] = off;
            off += loc[q];
        }
    }
    __syncthreads();
    // output position of ranked slot j of digit d: s_gbase[d] + j - s_dbase[d]
#pragma unroll
    for (int k = 0; k < PER_T; ++k) {
        const int dd = threadIdx.x + k * SORT_THREADS;
        s_gbase[dd] -= s_dbase[dd];
    }
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        if (base + r * 32 + lane < n) {
            const uint32_t d = digit_of(key[r], key_lo, key_max, shift, mask);
            const uint32_t l = s_dbase[d] + s_wh[w][d] + rank[r];
            s_k[l] = key[r];
            s_v[l] = s_vin[lbase + r * 32];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - blk < SORT_TILE ? n - blk : SORT_TILE);
    for (int j = threadIdx.x; j < cnt; j += SORT_THREADS) {
        const uint32_t k = s_k[j];
        const uint32_t d = digit_of(k, key_lo, key_max, shift, mask);
        const uint32_t g = s_gbase[d] + (uint32_t)j;
        keys_out[g] = k;
        vals_out[g] = s_v[j];
    }
}

// ------------------------------------------------------------ emission
// Tile counts in depth order (the scan that places each point-view's run of
// pairs reads them).
// The random gather reads the one-byte copy (a fourth of the bytes, which
// stay in L2) and the full count only for the rare counts above 254.
__global__ void gather_counts_kernel(const uint32_t *__restrict__ sorted_pv,
                                     const uint32_t *__restrict__ ntiles,
                                     const uint8_t *__restrict__ nt8, const uint32_t *n_dev,
                                     int64_t cap, uint32_t *__restrict__ nt_sorted)
{
    const int64_t n = dev_count(n_dev, cap);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t pv = sorted_pv[j];
    const uint32_t c = nt8[pv];
    nt_sorted[j] = c < 255u ? c : ntiles[pv];
}

// Position of the (t+1)-th set bit of m (t < popc(m)), by halving.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t t)
{
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << w) - 1u));
        if (t >= c) {
            t -= c;
            pos += w;
            m >>= w;
        }
    }
    return pos;
}

// Each warp owns 32 consecutive depth-sorted point-views; their pair runs
// are contiguous in the output, so the warp writes them together: output q
// belongs to the last lane whose run starts at or before q.  The run of a
// box wider than 32 tiles (no listed-tile mask) is written afterwards by the
// whole warp, 32 tiles of the box at a time.  Key of a pair: global tile <<
// sb | the 8 x 8 block mask of the pair (sb = block_bits; 0: no mask).
template <int TW, int TH>
__global__ void __launch_bounds__(256)
emit_pairs_kernel(const DevView *__restrict__ views, int32_t n_views,
                  const uint32_t *__restrict__ sorted_pv, const uint32_t *__restrict__ nt_sorted,
                  const uint32_t *__restrict__ offs, const uint4 *__restrict__ rect,
                  const uint32_t *n_dev, int64_t cap_vis, uint32_t *__restrict__ keys,
                  uint32_t *__restrict__ vals, int64_t cap_pairs, uint32_t *status)
{
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr int sb = block_bits(TW, TH);
    constexpr int tws = TW == 8 ? 3 : 4, ths = TH == 8 ? 3 : (TH == 16 ? 4 : 5);
    static_assert((1 << tws) == TW && (1 << ths) == TH, "tile sizes are powers of two");
    const int64_t n = dev_count(n_dev, cap_vis);
    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31;
    if (j0 >= n) return; // whole warp past the end
    const int lane = threadIdx.x & 31;
    const int64_t j = j0 + lane;
    const bool ok = j < n;
    // the lane's point-view (invalid lanes own no output)
    uint32_t pre = 0xffffffffu, nt = 0, pv = 0, tb = 0, wxt = 1, mask = 0, box = 0, wh = 0;
    uint32_t wy = 1;
    float px = 0.f, py = 0.f, rc2 = 0.f;
    bool big = false;
    if (ok) {
        pre = offs[j];
        nt = nt_sorted[j];
        pv = sorted_pv[j];
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (views[mid].pv_base <= (int64_t)pv) lo = mid; else hi = mid - 1;
        }
        const DevView &V = views[lo];
        const uint4 r4 = rect[pv];
        px = __uint_as_float(r4.x);
        py = __uint_as_float(r4.y);
        const float rc = __uint_as_float(r4.z);
        rc2 = __fmul_rn(rc, rc);
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        pixel_box(px, py, rc, V.W, V.H, x0, x1, y0, y1); // meets the image: the pv is listed
        const uint32_t tx0 = (uint32_t)x0 >> tws, ty0 = (uint32_t)y0 >> ths;
        const uint32_t wx = ((uint32_t)x1 >> tws) - tx0 + 1;
        wy = ((uint32_t)y1 >> ths) - ty0 + 1;
        big = wx * wy > 32;
        mask = big ? 0u : r4.w;
        tb = V.tile_base + ty0 * (uint32_t)V.tiles_x + tx0;
        wxt = wx | ((uint32_t)V.tiles_x << 16);
        box = (tx0 << tws) | ((ty0 << ths) << 16);
        wh = (uint32_t)V.W | ((uint32_t)V.H << 16);
    }
    const uint32_t start = __shfl_sync(FULL, pre, 0);
    const uint32_t last_lane = (uint32_t)(n - 1 - j0 < 31 ? n - 1 - j0 : 31);
    const uint32_t end = __shfl_sync(FULL, pre + nt, last_lane);
    if (lane == 0 && (int64_t)end > cap_pairs) atomicOr(status, ST_PAIR_OVERFLOW);
    // Owner of output q: the last lane whose run starts at or before q.  Every
    // valid lane's run is non-empty (a listed point-view covers a tile), so
    // the runs starting inside a window of 32 outputs are one bit each of a
    // mask, and the owner is the lane owning the window's first output
    // minus one, plus the starts at or before q.
    const uint32_t le = lanemask_lt() | (1u << lane);
    int before = -1; // owner of output q0 - 1 (none before the first window)
    for (uint32_t q0 = start; q0 < end; q0 += 32) {
        const uint32_t q = q0 + lane;
        const uint32_t rel = pre - q0; // valid lanes: pre >= q0 once their run is due
        const uint32_t starts = __reduce_or_sync(FULL, rel < 32u ? 1u << rel : 0u);
        const int ow = before + __popc(starts & le);
        before += __popc(starts);
        const uint32_t opre = __shfl_sync(FULL, pre, ow);
        const uint32_t otb = __shfl_sync(FULL, tb, ow);
        const uint32_t owxt = __shfl_sync(FULL, wxt, ow);
        const uint32_t opv = __shfl_sync(FULL, pv, ow);
        const uint32_t omask = __shfl_sync(FULL, mask, ow);
        uint32_t obox = 0, owh = 0;
        float opx = 0.f, opy = 0.f, orc2 = 0.f;
        if (sb) {
            obox = __shfl_sync(FULL, box, ow);
            owh = __shfl_sync(FULL, wh, ow);
            opx = __shfl_sync(FULL, px, ow);
            opy = __shfl_sync(FULL, py, ow);
            orc2 = __shfl_sync(FULL, rc2, ow);
        }
        // omask == 0: a wide box, written below
        if (q < end && (int64_t)q < cap_pairs && omask) {
            const uint32_t t = nth_set_bit(omask, q - opre); // position of the listed tile
            const uint32_t owx = owxt & 0xffff;
            // row = floor(t / owx), exactly: (t + 0.5) / owx is at least
            // 0.5 / owx away from an integer and the two roundings move it
            // by less than 2^-23 of itself (t < 32)
            const uint32_t row =
                (uint32_t)__fmul_rn((float)t + 0.5f, __frcp_rn((float)owx));
            const uint32_t col = t - row * owx;
            uint32_t key = otb + row * (owxt >> 16) + col;
            if (sb) {
                const int ox = (int)(obox & 0xffff) + ((int)col << tws);
                const int oy = (int)(obox >> 16) + ((int)row << ths);
                key = (key << sb) | tile_block_mask<TW, TH>(opx, opy, orc2, ox, oy,
                                                            (int)(owh & 0xffff), (int)(owh >> 16));
            }
            keys[q] = key;
            vals[q] = opv;
        }
    }
    // wide boxes: the warp tests 32 tiles of the box at a time and writes the
    // listed ones in row-major order (the same test the count came from)
    uint32_t wide = __ballot_sync(FULL, ok && big);
    while (wide) {
        const int bl = __ffs(wide) - 1;
        wide &= wide - 1;
        const uint32_t bpre = __shfl_sync(FULL, pre, bl), bnt = __shfl_sync(FULL, nt, bl);
        const uint32_t btb = __shfl_sync(FULL, tb, bl), bwxt = __shfl_sync(FULL, wxt, bl);
        const uint32_t bwy = __shfl_sync(FULL, wy, bl), bpv = __shfl_sync(FULL, pv, bl);
        const uint32_t bbox = __shfl_sync(FULL, box, bl), bwh = __shfl_sync(FULL, wh, bl);
        const float bpx = __shfl_sync(FULL, px, bl), bpy = __shfl_sync(FULL, py, bl);
        const float brc2 = __shfl_sync(FULL, rc2, bl);
        const uint32_t bwx = bwxt & 0xffff, total = bwx * bwy;
        const int W = (int)(bwh & 0xffff), H = (int)(bwh >> 16);
        uint32_t written = 0;
        for (uint32_t k0 = 0; k0 < total; k0 += 32) {
            const uint32_t k = k0 + lane;
            bool listed = false;
            uint32_t key = 0;
            if (k < total) {
                const uint32_t row = k / bwx, col = k - row * bwx;
                const int xa = (int)(bbox & 0xffff) + ((int)col << tws);
                const int ya = (int)(bbox >> 16) + ((int)row << ths);
                listed = rect_reached(bpx, bpy, brc2, xa, min(xa + TW, W) - 1, ya,
                                      min(ya + TH, H) - 1);
                key = btb + row * (bwxt >> 16) + col;
                if (listed && sb)
                    key = (key << sb) | tile_block_mask<TW, TH>(bpx, bpy, brc2, xa, ya, W, H);
            }
            const uint32_t m = __ballot_sync(FULL, listed);
            const uint32_t rank = written + (uint32_t)__popc(m & lanemask_lt());
            const uint32_t q = bpre + rank;
            if (listed && rank < bnt && (int64_t)q < cap_pairs) {
                keys[q] = key;
                vals[q] = bpv;
            }
            written += (uint32_t)__popc(m);
        }
        if (lane == 0 && written != bnt) atomicOr(status, ST_BAD_RANGE);
    }
}

// [start, end) of every tile (key >> shift) in the sorted key list; four
// keys per thread.
__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                   int64_t cap, uint2 *__restrict__ ranges, uint32_t n_tiles,
                                   int shift)
{
    const int64_t n = dev_count(n_dev, cap);
    const int64_t j4 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (j4 >= n) return;
    uint32_t k[6]; // k[0] = tile before the group, k[5] = tile after it
    if (j4 + 3 < n) {
        const uint4 q = *reinterpret_cast<const uint4 *>(keys + j4);
        k[1] = q.x >> shift;
        k[2] = q.y >> shift;
        k[3] = q.z >> shift;
        k[4] = q.w >> shift;
    } else {
        for (int i = 0; i < 4; ++i) k[1 + i] = j4 + i < n ? keys[j4 + i] >> shift : 0xffffffffu;
    }
    k[0] = j4 > 0 ? keys[j4 - 1] >> shift : 0xffffffffu;
    k[5] = j4 + 4 < n ? keys[j4 + 4] >> shift : 0xffffffffu;
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        const int64_t j = j4 + i - 1;
        if (j >= n || k[i] >= n_tiles) continue;
        if (j == 0 || k[i - 1] != k[i]) ranges[k[i]].x = (uint32_t)j;
        if (j == n - 1 || k[i + 1] != k[i]) ranges[k[i]].y = (uint32_t)(j + 1);
    }
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

void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n,
                           unsigned long long *total, void *temp, cudaStream_t s)
{
    run_scan(LoadU32{in}, ActStore{out}, nullptr, n, temp, total, nullptr, s);
}

size_t radix_temp_bytes(int64_t cap)
{
    const int64_t nb = (cap + SORT_TILE - 1) / SORT_TILE;
    const int64_t hist = (nb > 0 ? nb : 1) * RBINS;
    return (size_t)hist * sizeof(uint32_t) + scan_temp_bytes(hist);
}

int radix_passes(int key_bits)
{
    return key_bits <= 0 ? 0 : (key_bits + RB - 1) / RB;
}

void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *&keys_alt, uint32_t *&vals_alt,
                      const uint32_t *n_dev, int64_t cap, int key_bits, void *temp,
                      cudaStream_t s, uint32_t key_lo, uint32_t key_max, bool index_vals,
                      int bit_lo)
{
    if (cap <= 0) return;
    if (key_bits <= 0) {
        if (!index_vals) return; // all keys equal: already in stable order
        key_bits = 1;            // one pass still writes the index values
    }
    static const bool attr = cudaFuncSetAttribute(radix_scatter_kernel,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)SCATTER_SMEM) == cudaSuccess;
    (void)attr;
    const int64_t nb = (cap + SORT_TILE - 1) / SORT_TILE;
    uint32_t *hist = (uint32_t *)temp;
    void *scan_tmp = hist + nb * RBINS;
    const int passes = radix_passes(key_bits);
    const int width = (key_bits + passes - 1) / passes;
    for (int shift = bit_lo; shift < bit_lo + key_bits; shift += width) {
        const int wd = bit_lo + key_bits - shift < width ? bit_lo + key_bits - shift : width;
        radix_hist_kernel<<<(unsigned)((nb + HIST_TILES - 1) / HIST_TILES), SORT_THREADS, 0, s>>>(
            keys, n_dev, cap, key_lo, key_max, shift, wd, hist, nb);
        run_scan(LoadU32{hist}, ActStore{hist}, nullptr, nb << wd, scan_tmp, nullptr, nullptr, s);
        radix_scatter_kernel<<<(unsigned)nb, SORT_THREADS, SCATTER_SMEM, s>>>(
            keys, vals, keys_alt, vals_alt, n_dev, cap, key_lo, key_max, shift, wd, hist, nb,
            index_vals && shift == bit_lo);
        count_launches(2);
        uint32_t *tk = keys, *tv = vals;
        keys = keys_alt;
        vals = vals_alt;
        keys_alt = tk;
        vals_alt = tv;
    }
}

size_t emit_temp_bytes(int64_t cap_vis)
{
    return (size_t)(cap_vis > 0 ? cap_vis : 1) * 2 * sizeof(uint32_t) + scan_temp_bytes(cap_vis);
}

void launch_emit_pairs(const Batch &b, const DevOpts &o, const uint32_t *sorted_pv,
                       const uint32_t *n_vis, int64_t cap_vis, const uint32_t *ntiles,
                       const uint8_t *nt8, const uint4 *rect, uint32_t *keys, uint32_t *vals,
                       int64_t cap_pairs,
                       uint32_t *status, void *temp, cudaStream_t s)
{
    if (cap_vis <= 0) return;
    uint32_t *nt_sorted = (uint32_t *)temp;
    uint32_t *offs = nt_sorted + cap_vis;
    void *scan_tmp = offs + cap_vis;
    const unsigned nb = (unsigned)((cap_vis + 255) / 256);
    gather_counts_kernel<<<nb, 256, 0, s>>>(sorted_pv, ntiles, nt8, n_vis, cap_vis, nt_sorted);
    run_scan(LoadU32{nt_sorted}, ActStore{offs}, n_vis, cap_vis, scan_tmp, nullptr, status, s);
    auto emit = emit_pairs_kernel<16, 16>;
    if (o.tile_w == 8 && o.tile_h == 8) emit = emit_pairs_kernel<8, 8>;
    else if (o.tile_w == 16 && o.tile_h == 32) emit = emit_pairs_kernel<16, 32>;
    emit<<<nb, 256, 0, s>>>(b.views, b.n_views, sorted_pv, nt_sorted, offs, rect, n_vis,
                            cap_vis, keys, vals, cap_pairs, status);
    count_launches(2);
}

void launch_tile_ranges(const uint32_t *keys, const uint32_t *n_pairs, int64_t cap_pairs,
                        uint2 *ranges, uint32_t n_tiles, int shift, cudaStream_t s)
{
    if (cap_pairs <= 0) return;
    const int th = 256;
    const int64_t nb = ((cap_pairs + 3) / 4 + th - 1) / th;
    tile_ranges_kernel<<<(unsigned)nb, th, 0, s>>>(keys, n_pairs, cap_pairs, ranges, n_tiles,
                                                   shift);
    count_launches(1);
}

} // namespace pbr
