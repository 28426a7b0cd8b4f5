// Per-tile compositing of Sec. 3.2 and its adjoint.
//
// Per pixel centre u and listed point (records {px, py, rc^2, q'} {o, rgb}):
//   d2 = (ux - px)^2 + (uy - py)^2            (fp32, round-to-nearest, no FMA)
//   if d2 <= rc^2:                             (the cutoff of Sec. 3.2)
//     alpha = min(alpha_max, o * 2^(q' d2))    (Eq. 5, q' = -log2(e)/(2 s^2))
//     C += T alpha c ;  T *= (1 - alpha)       (Eqs. 6-7, front to back)
// stopping after the point that takes T below t_eps or reaches the count
// cap.  Outputs C + T bg, T and the list position just after the last
// composited point.
//
// The adjoint walks each pixel's list back to front from that position.  T
// before a point is recovered as T_after/(1-alpha); S accumulates the colour
// behind the point, so
//   dL/dc     = alpha T g
//   dL/dalpha = T (c.g) - S / (1 - alpha)
// and, below the alpha_max clamp,
//   dL/do = dL/dalpha G,  dL/dp = dL/dalpha alpha q (u - p),
//   dL/dq = -dL/dalpha alpha d2 / 2          (q = 1/s^2).
// The kernels sum {ca (u - p), ca d2} with ca = dL/dalpha alpha, without
// the per-point factors q and -1/2, which the point stage applies once per
// point-view: the terms are {ca dx, ca dy, ca d2, do, dr, dg, db}.
// The 7 per-point terms of a warp go to the per-(view, point) buffer with
// 16-byte atomics: straight from each contributing lane when few lanes
// contribute, else summed first with a transposed shuffle reduction (two
// atomics per warp and point) in the warp-streamed schedules.
//
// The pair keys carry the mask of the tile's 8 x 8 pixel blocks that hold a
// pixel including the point, so a warp takes from its tile's list only the
// entries of its own block, and it skips those whose cutoff disc misses its
// still active pixels.  Three schedules:
//   - warp-streamed (batch depth 0, default): a block covers one TW x TH
//     screen tile, each warp an 8 x 4 sub-block of it; every warp walks its
//     entries by itself, 32 per step, culls them with one ballot and stops
//     as soon as its own pixels have saturated.  No block barriers.
//   - persistent (batch depth 0, persistent): one launch; warps take (tile,
//     8 x 8 block) items longest list first from an atomic counter; a lane
//     owns two pixels of a column, four rows apart, and their arithmetic
//     runs packed (fp32x2).  The forward steps through each chunk's hits in
//     lockstep; the backward forms the adjoint at both pixels per hit.
//   - block-staged (batch depth > 0): the block stages `depth` records in
//     shared memory and each warp culls the batch into its own list; block
//     barriers between batches, per-block shared-memory gradient sums.
// Store mode (STORE): the forward also keeps T before each of a pixel's
// first store_depth composited points, and the backward reads it there
// instead of dividing.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t lanemask_lt_r()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int find_view_by_tile(const Batch &b, uint32_t tile)
{
    int lo = 0, hi = b.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The calling thread's pixel and its warp's 8 x 4 rectangle of pixel
// centres [xl, xh] x [yl, yh] inside tile `tile`.
struct PixelGeom {
    const DevView *V;
    int x, y;
    bool inside;
    float ux, uy, xl, xh, yl, yh;
};

// Pixel (sx0 + (lane & 7), sy0 + (lane >> 3)) of view V and the 8 x 4
// rectangle of pixel centres with corner (sx0, sy0).
__device__ __forceinline__ PixelGeom pixel_geom_at(const DevView *V, int sx0, int sy0, int lane)
{
    PixelGeom g;
    g.V = V;
    g.x = sx0 + (lane & 7);
    g.y = sy0 + (lane >> 3);
    g.inside = g.x < g.V->W && g.y < g.V->H;
    g.ux = (float)g.x + 0.5f;
    g.uy = (float)g.y + 0.5f;
    g.xl = (float)sx0 + 0.5f;
    g.xh = (float)sx0 + 7.5f;
    g.yl = (float)sy0 + 0.5f;
    g.yh = (float)sy0 + 3.5f;
    return g;
}

// Sub-block `w` of tile `tile` (sub-blocks numbered row-major, TW/8 per row).
template <int TW, int TH>
__device__ __forceinline__ PixelGeom pixel_geom(const Batch &b, uint32_t tile, int w, int lane)
{
    const DevView *V = &b.views[find_view_by_tile(b, tile)];
    const uint32_t local = tile - V->tile_base;
    const int tx = (int)(local % (uint32_t)V->tiles_x), ty = (int)(local / (uint32_t)V->tiles_x);
    return pixel_geom_at(V, tx * TW + (w % (TW / 8)) * 8, ty * TH + (w / (TW / 8)) * 4, lane);
}

// Culling test of one record against a rectangle of pixel centres: the
// per-pixel cutoff test (the same fp32 round-to-nearest operations) applied
// to the rectangle's pixel centre nearest the splat centre, floor(p) + 0.5
// clamped into the rectangle per axis.  Rounding is monotone, so that
// centre has the smallest fp32 squared distance of all the rectangle's
// centres: the test keeps exactly the points some pixel of the rectangle
// includes.
__device__ __forceinline__ bool disc_meets_rect(const float4 a, const PixelGeom &g)
{
    const float cx = fminf(fmaxf(floorf(a.x) + 0.5f, g.xl), g.xh);
    const float cy = fminf(fmaxf(floorf(a.y) + 0.5f, g.yl), g.yh);
    const float ex = __fsub_rn(cx, a.x), ey = __fsub_rn(cy, a.y);
    return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= a.z;
}

// Whether the cutoff disc of a record holds every pixel centre of the
// rectangle: the per-pixel fp32 test applied to the centre farthest from the
// splat centre (per axis the edge with the larger rounded offset), which by
// monotone rounding has the largest fp32 squared distance.
__device__ __forceinline__ bool disc_covers_rect(const float4 a, const PixelGeom &g)
{
    const float lx = __fsub_rn(g.xl, a.x), hx = __fsub_rn(g.xh, a.x);
    const float ly = __fsub_rn(g.yl, a.y), hy = __fsub_rn(g.yh, a.y);
    const float ex = fabsf(lx) > fabsf(hx) ? lx : hx;
    const float ey = fabsf(ly) > fabsf(hy) ? ly : hy;
    return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= a.z;
}

// The rectangle of pixel centres of the warp's lanes that are still
// active (g's own rectangle when every lane is).  Warp-wide reductions: all
// 32 lanes must call it together, outside any lane-dependent branch or
// short-circuit.
__device__ __forceinline__ PixelGeom active_rect(const PixelGeom &g, bool active)
{
    PixelGeom r = g;
    const uint32_t x = (uint32_t)g.x, y = (uint32_t)g.y;
    const uint32_t x0 = __reduce_min_sync(0xffffffffu, active ? x : 0xffffffffu);
    const uint32_t x1 = __reduce_max_sync(0xffffffffu, active ? x : 0u);
    const uint32_t y0 = __reduce_min_sync(0xffffffffu, active ? y : 0xffffffffu);
    const uint32_t y1 = __reduce_max_sync(0xffffffffu, active ? y : 0u);
    r.xl = (float)x0 + 0.5f;
    r.xh = (float)x1 + 0.5f;
    r.yl = (float)y0 + 0.5f;
    r.yh = (float)y1 + 0.5f;
    return r;
}

// active_rect for a warp that owns P pixels per lane, one column, rows 4
// apart (g[q] below g[q-1]): the rectangle of the centres of its still
// active pixels.  The same calling rule holds.
template <int P>
__device__ __forceinline__ PixelGeom active_rect_rows(const PixelGeom (&g)[P], const bool (&act)[P])
{
    PixelGeom r = g[0];
    bool any = false;
    uint32_t ylo = 0xffffffffu, yhi = 0u;
#pragma unroll
    for (int q = P - 1; q >= 0; --q) {
        any = any || act[q];
        if (act[q]) ylo = (uint32_t)g[q].y;
    }
#pragma unroll
    for (int q = 0; q < P; ++q)
        if (act[q]) yhi = (uint32_t)g[q].y;
    const uint32_t x = (uint32_t)g[0].x;
    const uint32_t x0 = __reduce_min_sync(0xffffffffu, any ? x : 0xffffffffu);
    const uint32_t x1 = __reduce_max_sync(0xffffffffu, any ? x : 0u);
    const uint32_t y0 = __reduce_min_sync(0xffffffffu, ylo);
    const uint32_t y1 = __reduce_max_sync(0xffffffffu, yhi);
    r.xl = (float)x0 + 0.5f;
    r.xh = (float)x1 + 0.5f;
    r.yl = (float)y0 + 0.5f;
    r.yh = (float)y1 + 0.5f;
    return r;
}

// Sum of 8 per-lane values over the warp; lane l returns the total of value
// (l >> 2) & 7.  Three halving exchanges then two butterfly steps.
__device__ __forceinline__ float warp_sum8_transposed(const float v[8], int lane)
{
    float a[4];
    bool hi = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = hi ? v[k] : v[k + 4];
        const float keep = hi ? v[k + 4] : v[k];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float c2[2];
    hi = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = hi ? a[k] : a[k + 2];
        const float keep = hi ? a[k + 2] : a[k];
        c2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    hi = lane & 4;
    float r;
    {
        const float send = hi ? c2[0] : c2[1];
        const float keep = hi ? c2[1] : c2[0];
        r = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// Adds the warp's 7 per-point terms to g2d[pv][0..6] with two 16-byte
// atomics: after the transposed reduction lane 4k holds term k; lanes 0 and
// 16 gather four terms each.
__device__ __forceinline__ void warp_add_terms(const float v[8], int lane, float *g2d, uint32_t pv)
{
    const float t = warp_sum8_transposed(v, lane);
    const float t1 = __shfl_down_sync(0xffffffffu, t, 4);
    const float t2 = __shfl_down_sync(0xffffffffu, t, 8);
    const float t3 = __shfl_down_sync(0xffffffffu, t, 12);
    if ((lane & 15) == 0) {
        float4 *dst = reinterpret_cast<float4 *>(g2d + 8 * (size_t)pv) + (lane >> 4);
        atomicAdd(dst, make_float4(t, t1, t2, lane ? 0.f : t3));
    }
}

// ------------------------------------------------------ block-mask queues
// The pair keys carry the mask of the 8 x 8 pixel blocks of the tile that
// hold a pixel including the point (pair key = tile << B | mask), so a warp
// working on one block takes from its tile's list only the entries with its
// block's bit: the queue below holds their list positions (relative to the
// tile's first entry) and point-view ids, in compositing order, and the
// compositing loops consume it 32 entries at a time.  bit == 0 (tiles of
// one block) takes every entry.
// The queue is a ring of QCAP entries read from `head`; a fill scans
// FILL_GROUPS groups of 32 list entries per step, their loads in flight
// together (a warp's block takes a fraction of its tile's entries, so a
// refill scans several groups).
constexpr int QCAP = 128;
constexpr int FILL_GROUPS = 3; // 32 + 3 x 32 entries fit the ring
struct WarpQueue {
    uint32_t pos[QCAP]; // list positions, relative to the tile's first entry
    uint32_t pv[QCAP];  // point-view ids
};

// Front to back: scans the list from position p (absolute, < e), appending
// the entries with `bit`, until the queue holds 32 or the list ends.
// Warp-uniform.
__device__ __forceinline__ void queue_fill_front(const uint32_t *__restrict__ keys,
                                                 const uint32_t *__restrict__ pv_list, uint32_t s,
                                                 uint32_t e, uint32_t bit, uint32_t &p, int &qn,
                                                 uint32_t qh, WarpQueue &q, int lane)
{
    const uint32_t lt = lanemask_lt_r();
    while (qn < 32 && p < e) {
        uint32_t k[FILL_GROUPS];
#pragma unroll
        for (int g = 0; g < FILL_GROUPS; ++g) {
            const uint32_t i = p + 32 * g + lane;
            k[g] = bit && i < e ? __ldg(keys + i) : 0u;
        }
#pragma unroll
        for (int g = 0; g < FILL_GROUPS; ++g) {
            const uint32_t i = p + 32 * g + lane;
            const bool take = i < e && (bit == 0 || (k[g] & bit) != 0);
            const uint32_t m = __ballot_sync(0xffffffffu, take);
            if (take) {
                const uint32_t slot = (qh + (uint32_t)qn + __popc(m & lt)) & (QCAP - 1);
                q.pos[slot] = i - s;
                q.pv[slot] = __ldg(pv_list + i);
            }
            qn += __popc(m);
        }
        p = e - p > 32u * FILL_GROUPS ? p + 32u * FILL_GROUPS : e;
    }
    __syncwarp();
}

// Back to front: scans the relative positions [0, c + 32) downwards from
// the aligned chunk c (c < 0: nothing left), entries below `lim` only,
// appending the entries with `bit` in descending position order.
__device__ __forceinline__ void queue_fill_back(const uint32_t *__restrict__ keys,
                                                const uint32_t *__restrict__ pv_list, uint32_t s,
                                                uint32_t lim, uint32_t bit, int64_t &c, int &qn,
                                                uint32_t qh, WarpQueue &q, int lane)
{
    const uint32_t gt = ~(lanemask_lt_r() | (1u << lane));
    while (qn < 32 && c >= 0) {
        uint32_t k[FILL_GROUPS];
#pragma unroll
        for (int g = 0; g < FILL_GROUPS; ++g) {
            const int64_t cg = c - 32 * g;
            const uint32_t i = (uint32_t)cg + lane;
            k[g] = bit && cg >= 0 && i < lim ? __ldg(keys + s + i) : 0u;
        }
#pragma unroll
        for (int g = 0; g < FILL_GROUPS; ++g) {
            const int64_t cg = c - 32 * g;
            const uint32_t i = (uint32_t)cg + lane;
            const bool take = cg >= 0 && i < lim && (bit == 0 || (k[g] & bit) != 0);
            const uint32_t m = __ballot_sync(0xffffffffu, take);
            if (take) {
                const uint32_t slot = (qh + (uint32_t)qn + __popc(m & gt)) & (QCAP - 1);
                q.pos[slot] = i;
                q.pv[slot] = __ldg(pv_list + s + i);
            }
            qn += __popc(m);
        }
        c -= 32 * FILL_GROUPS;
    }
    __syncwarp();
}

// Takes the next min(qn, 32) queued entries: lane l < the count receives
// entry l (its relative position and point-view).  Returns the count.
__device__ __forceinline__ int queue_take(WarpQueue &q, int &qn, uint32_t &qh, int lane,
                                          uint32_t &pos, uint32_t &pv)
{
    const int take = qn < 32 ? qn : 32;
    if (lane < take) {
        const uint32_t slot = (qh + (uint32_t)lane) & (QCAP - 1);
        pos = q.pos[slot];
        pv = q.pv[slot];
    }
    qh += (uint32_t)take;
    qn -= take;
    __syncwarp();
    return take;
}

// Keeps the compiler from fusing the product that produced v into a later
// add (a product feeding an add can be merged into one fused multiply-add
// even across __fmul_rn, which changes the rounding of a distance and with
// it the exact cutoff decision).
__device__ __forceinline__ float unfused1(float v)
{
    asm volatile("" : "+f"(v));
    return v;
}

// One composited point, front to back.  Returns true when the pixel stops.
// Every rounding is explicit: alpha = min(alpha_max, o 2^(q' d2)), weight
// alpha T, C += weight c (fused), T -= weight.
__device__ __forceinline__ bool pixel_blend(float d2, const float4 a, const float4 c,
                                            const DevOpts &o, float &T, float &C0, float &C1,
                                            float &C2, uint32_t &cnt)
{
    const float alpha = fminf(o.alpha_max, __fmul_rn(c.x, ex2_approx(__fmul_rn(d2, a.w))));
    const float wgt = __fmul_rn(alpha, T);
    C0 = fmaf(wgt, c.y, C0);
    C1 = fmaf(wgt, c.z, C1);
    C2 = fmaf(wgt, c.w, C2);
    T = __fsub_rn(T, wgt);
    ++cnt;
    return T < o.t_eps || cnt == (uint32_t)o.max_per_pixel;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Branch-free adjoint for a warp-uniform loop: `take` (0 or 1) says whether
// the point was composited at this pixel; with take = 0 every term is 0 and
// T, S are unchanged.
// With has_tb, tb is the stored transmittance before the point (store mode)
// instead of the one recovered by division.
__device__ __forceinline__ void pixel_adjoint_masked(float take, float d2, float dx, float dy,
                                                     const float4 a, const float4 c, float amax,
                                                     float g0, float g1, float g2, float &T,
                                                     float &S, float v[8], bool has_tb = false,
                                                     float tb = 0.0f)
{
    const float G = ex2_approx(d2 * a.w);
    const float raw = c.x * G;
    const float alpha = fminf(amax, raw) * take;
    const float rom = rcp_approx(1.0f - alpha);
    const float Tb = has_tb ? tb : T * rom;
    const float wgt = alpha * Tb;
    const float cg = c.y * g0 + c.z * g1 + c.w * g2;
    v[4] = wgt * g0;
    v[5] = wgt * g1;
    v[6] = wgt * g2;
    const float dalpha = (Tb * cg - S * rom) * take;
    S = fmaf(wgt, cg, S);
    T = Tb;
    const float ca = raw < amax ? dalpha * alpha : 0.0f; // clamped: no geometry terms
    v[0] = ca * dx;
    v[1] = ca * dy;
    v[2] = ca * d2;
    v[3] = raw < amax ? dalpha * G : 0.0f;
    v[7] = 0.0f;
}

// Per-pixel adjoint of one composited point (see the file comment).  On
// return v[0..6] = {ca dx, ca dy, ca d2, do, dr, dg, db}; T and S are
// updated.
__device__ __forceinline__ void pixel_adjoint(float d2, float dx, float dy, const float4 a,
                                              const float4 c, float amax, float g0, float g1,
                                              float g2, float &T, float &S, float v[8])
{
    const float G = ex2_approx(d2 * a.w);
    const float raw = c.x * G;
    const float alpha = fminf(amax, raw);
    const float rom = __frcp_rn(1.0f - alpha);
    const float Tb = T * rom;
    const float wgt = alpha * Tb;
    const float cg = c.y * g0 + c.z * g1 + c.w * g2;
    v[4] = wgt * g0;
    v[5] = wgt * g1;
    v[6] = wgt * g2;
    const float dalpha = Tb * cg - S * rom;
    S = fmaf(wgt, cg, S);
    T = Tb;
    if (raw < amax) {
        const float ca = dalpha * alpha;
        v[0] = ca * dx;
        v[1] = ca * dy;
        v[2] = ca * d2;
        v[3] = dalpha * G;
    }
}

__device__ __forceinline__ float pixel_d2(float ux, float uy, float px, float py, float &dx,
                                          float &dy)
{
    dx = __fsub_rn(ux, px);
    dy = __fsub_rn(uy, py);
    return __fadd_rn(unfused1(__fmul_rn(dx, dx)), unfused1(__fmul_rn(dy, dy)));
}

// Index of the pixel in the packed per-pixel arrays (valid when inside).
__device__ __forceinline__ int64_t pixel_index(const PixelGeom &g)
{
    return g.V->pix_base + (int64_t)g.y * g.V->W + g.x;
}

// Store mode: T before the cnt-th composited point of pixel pix.
__device__ __forceinline__ void store_T(const StoreBuf &sto, int64_t pix, uint32_t cnt, float T)
{
    if (sto.T && cnt < (uint32_t)sto.depth) sto.T[pix * sto.depth + cnt] = T;
}

__device__ __forceinline__ void write_pixel(const PixelGeom &g, const DevOpts &o, float T,
                                            float C0, float C1, float C2, uint32_t last,
                                            float *out_rgb, float *T_final, uint32_t *n_contrib)
{
    if (!g.inside) return;
    const int64_t local = (int64_t)g.y * g.V->W + g.x;
    const int64_t pix = g.V->pix_base + local;
    float *dst = g.V->out ? g.V->out + 3 * local : out_rgb + 3 * pix;
    dst[0] = C0 + T * o.bg[0];
    dst[1] = C1 + T * o.bg[1];
    dst[2] = C2 + T * o.bg[2];
    T_final[pix] = T;
    n_contrib[pix] = last;
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, uint32_t a, uint32_t b,
                                          int lane)
{
    if (!stats) return;
    const uint32_t wa = __reduce_add_sync(0xffffffffu, a);
    const uint32_t wb = __reduce_add_sync(0xffffffffu, b);
    if (lane == 0) {
        atomicAdd(stats, (unsigned long long)wa);
        atomicAdd(stats + 1, (unsigned long long)wb);
    }
}

// ======================================================= warp-streamed
// One warp composites its 8 x 4 sub-block of a tile.  Each step takes 32
// entries of the warp's 8 x 8 block from its queue, culls them against the
// warp's rectangle with one ballot and stages the hits in the warp's shared
// buffer; then
//   phase 1 (warp-uniform): for every hit, every lane runs its exact fp32
//            cutoff test and records the hit in its own bitmask;
//   phase 2 (per lane): each lane walks only its own included entries.
// wbuf: this warp's 64 float4 (a-parts, then b-parts of the chunk).
// g: the lane's pixel and the warp's rectangle; [s, e): the tile's list.
template <bool STATS, bool STORE>
__device__ __forceinline__ void fwd_stream_item(const PixelGeom &g, uint32_t s, uint32_t e,
                                                uint32_t bit, const DevOpts &o, int lane,
                                                const uint32_t *__restrict__ keys,
                                                const uint32_t *__restrict__ pv_list,
                                                const float4 *__restrict__ rec,
                                                float *__restrict__ out_rgb,
                                                float *__restrict__ T_final,
                                                uint32_t *__restrict__ n_contrib,
                                                uint32_t &examined_acc, uint32_t &composited_acc,
                                                float4 *wbuf, uint32_t *wpos, WarpQueue &q,
                                                const StoreBuf &sto)
{
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t cnt = 0, last = 0, examined = 0;
    bool done = !g.inside;
    const int64_t pix = STORE && g.inside ? pixel_index(g) : 0;
    uint32_t p = s;
    int qn = 0;
    uint32_t qh = 0;
    while (!__all_sync(0xffffffffu, done)) {
        queue_fill_front(keys, pv_list, s, e, bit, p, qn, qh, q, lane);
        if (qn == 0) break;
        uint32_t rel = 0, pv = 0;
        const int take = queue_take(q, qn, qh, lane, rel, pv);
        const bool valid = lane < take;
        float4 a = make_float4(0.f, 0.f, -1.f, 0.f);
        if (valid) a = __ldg(rec + 2 * (size_t)pv);
        // every lane takes part in the reductions, whatever its entry
        const PixelGeom ar = active_rect(g, !done);
        const bool hit = valid && disc_meets_rect(a, ar);
        const bool covers = hit && disc_covers_rect(a, ar);
        uint32_t m = __ballot_sync(0xffffffffu, hit);
        // entries whose disc holds every active pixel need no per-pixel test
        uint32_t mine = __ballot_sync(0xffffffffu, covers);
        if (hit) {
            wbuf[lane] = a;
            wbuf[32 + lane] = __ldg(rec + 2 * (size_t)pv + 1);
            wpos[lane] = rel;
        }
        __syncwarp();
        if (STATS && !done) examined += (uint32_t)__popc(m);
        m &= ~mine;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 aj = wbuf[j];
            float dx, dy;
            if (pixel_d2(g.ux, g.uy, aj.x, aj.y, dx, dy) <= aj.z) mine |= 1u << j;
        }
        if (done) mine = 0;
        while (mine) {
            const int j = __ffs(mine) - 1;
            mine &= mine - 1;
            const float4 aj = wbuf[j];
            float dx, dy;
            const float d2 = pixel_d2(g.ux, g.uy, aj.x, aj.y, dx, dy);
            last = wpos[j] + 1;
            if (STORE) store_T(sto, pix, cnt, T);
            if (pixel_blend(d2, aj, wbuf[32 + j], o, T, C0, C1, C2, cnt)) {
                done = true;
                break;
            }
        }
        __syncwarp(); // chunk consumed before the buffers are refilled
    }
    examined_acc += examined;
    composited_acc += cnt;
    if (STORE && g.inside) sto.n[pix] = cnt;
    write_pixel(g, o, T, C0, C1, C2, last, out_rgb, T_final, n_contrib);
}

// ------------------------------------------------- packed two-pixel math
// A lane of the 8 x 8-pixel warps owns two pixels of one column, rows 4
// apart (A above B); their per-point arithmetic runs in packed fp32x2
// operations (.x pixel A, .y pixel B), one instruction for both pixels.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Keeps the compiler from fusing the product that produced v into a later
// packed add (it merges a product feeding a packed add into one packed FMA,
// even across __fmul_rn, which changes the rounding of a distance and with it
// the exact cutoff decision).
__device__ __forceinline__ float2 unfused(float2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    asm volatile("" : "+l"(r));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// Squared fp32 distances from the lane's two pixel centres (ux, uy.x) and
// (ux, uy.y) to the splat centre, with the rounding of pixel_d2: dx =
// ux - px (shared), dy = uy - py, d2 = dx dx + dy dy, each operation rounded
// to nearest (no contraction).
__device__ __forceinline__ float2 pair_d2(float ux, float2 uy, float px, float py, float &dx,
                                          float2 &dy)
{
    dx = __fsub_rn(ux, px);
    dy = add2(uy, f2(-py));
    const float dx2 = __fmul_rn(dx, dx);
    return add2(unfused(f2(dx2)), unfused(mul2(dy, dy)));
}

// Forward of one 8 x 8 block by one warp, for the persistent schedule:
// lane l owns the pixels (l & 7, l >> 3) and (l & 7, 4 + (l >> 3)), gA and
// gB.  The warp takes the tile list's entries with its block's bit (`bit`)
// 32 at a time from its queue, culls them against the rectangle of its
// active pixels and stages the hits; then it steps through the hits in list
// order, every lane testing and blending the point at both of its pixels at
// once (packed fp32x2, .x pixel A, .y pixel B), with the blend of a pixel
// the point does not include (or that has stopped) masked to zero weight.
// Each pixel's blend sequence and roundings are the one-pixel walk's.
template <bool STATS, bool STORE>
__device__ __forceinline__ void fwd_pair_item(const PixelGeom &gA, const PixelGeom &gB,
                                              uint32_t s, uint32_t e, uint32_t bit,
                                              const DevOpts &o, int lane,
                                              const uint32_t *__restrict__ keys,
                                              const uint32_t *__restrict__ pv_list,
                                              const float4 *__restrict__ rec,
                                              float *__restrict__ out_rgb,
                                              float *__restrict__ T_final,
                                              uint32_t *__restrict__ n_contrib,
                                              uint32_t &examined_acc, uint32_t &composited_acc,
                                              float4 *wbuf, uint32_t *wpos, WarpQueue &q,
                                              const StoreBuf &sto)
{
    const int64_t pixA = STORE && gA.inside ? pixel_index(gA) : 0;
    const int64_t pixB = STORE && gB.inside ? pixel_index(gB) : 0;
    float2 T = f2(1.0f), C0 = f2(0.0f), C1 = f2(0.0f), C2 = f2(0.0f);
    uint32_t cntA = 0, cntB = 0, lastA = 0, lastB = 0, examined = 0;
    bool doneA = !gA.inside, doneB = !gB.inside;
    const PixelGeom g2[2] = {gA, gB};
    const float2 uy2 = make_float2(gA.uy, gB.uy);
    const uint32_t cmax = (uint32_t)o.max_per_pixel;
    uint32_t p = s;
    int qn = 0;
    uint32_t qh = 0;
    while (!__all_sync(0xffffffffu, doneA && doneB)) {
        queue_fill_front(keys, pv_list, s, e, bit, p, qn, qh, q, lane);
        if (qn == 0) break;
        uint32_t rel = 0, pv = 0;
        const int take = queue_take(q, qn, qh, lane, rel, pv);
        const bool valid = lane < take;
        float4 a = make_float4(0.f, 0.f, -1.f, 0.f);
        if (valid) a = __ldg(rec + 2 * (size_t)pv);
        // every lane takes part in the reductions, whatever its entry
        const bool act[2] = {!doneA, !doneB};
        const PixelGeom ar = active_rect_rows<2>(g2, act);
        const bool hit = valid && disc_meets_rect(a, ar);
        uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            wbuf[lane] = a;
            wbuf[32 + lane] = __ldg(rec + 2 * (size_t)pv + 1);
            wpos[lane] = rel;
        }
        __syncwarp();
        if (STATS) examined += (uint32_t)__popc(m) * ((uint32_t)!doneA + (uint32_t)!doneB);
        // the chunk's composited entries of each pixel, as bits of the chunk
        // (counts and the last position follow after the chunk)
        uint32_t incA = 0u, incB = 0u;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 aj = wbuf[j];
            float dx;
            float2 dy;
            const float2 d2 = pair_d2(gA.ux, uy2, aj.x, aj.y, dx, dy);
            const bool inA = !doneA && d2.x <= aj.z, inB = !doneB && d2.y <= aj.z;
            if (!__any_sync(0xffffffffu, inA || inB)) continue;
            const float4 cj = wbuf[32 + j];
            const float2 ea = mul2(d2, f2(aj.w));
            const float2 raw = mul2(f2(cj.x), make_float2(ex2_approx(ea.x), ex2_approx(ea.y)));
            const float2 alpha = make_float2(inA ? fminf(o.alpha_max, raw.x) : 0.0f,
                                             inB ? fminf(o.alpha_max, raw.y) : 0.0f);
            if (STORE) {
                if (inA) store_T(sto, pixA, cntA + __popc(incA), T.x);
                if (inB) store_T(sto, pixB, cntB + __popc(incB), T.y);
            }
            const float2 wgt = mul2(alpha, T);
            C0 = fma2(wgt, f2(cj.y), C0);
            C1 = fma2(wgt, f2(cj.z), C1);
            C2 = fma2(wgt, f2(cj.w), C2);
            T = add2(T, make_float2(-wgt.x, -wgt.y));
            const uint32_t bit_j = 1u << j;
            if (inA) {
                incA |= bit_j;
                doneA = T.x < o.t_eps;
            }
            if (inB) {
                incB |= bit_j;
                doneB = T.y < o.t_eps;
            }
            if (cmax) { // count cap (warp-uniform branch)
                doneA = doneA || (inA && cntA + __popc(incA) == cmax);
                doneB = doneB || (inB && cntB + __popc(incB) == cmax);
            }
        }
        if (incA) {
            cntA += __popc(incA);
            lastA = wpos[31 - __clz(incA)] + 1;
        }
        if (incB) {
            cntB += __popc(incB);
            lastB = wpos[31 - __clz(incB)] + 1;
        }
        __syncwarp(); // chunk consumed before the buffers are refilled
    }
    examined_acc += examined;
    composited_acc += cntA + cntB;
    if (STORE) {
        if (gA.inside) sto.n[pixA] = cntA;
        if (gB.inside) sto.n[pixB] = cntB;
    }
    write_pixel(gA, o, T.x, C0.x, C1.x, C2.x, lastA, out_rgb, T_final, n_contrib);
    write_pixel(gB, o, T.y, C0.y, C1.y, C2.y, lastB, out_rgb, T_final, n_contrib);
}

// Up to this many contributing pixels of a warp add their terms with their
// own vector atomics; more go through the transposed warp reduction.  The
// reduction costs some 35 instructions whatever the count, the atomics
// cost L2 throughput per pixel; measured on the batched 1M-point
// workload, the backward runs fastest between 12 and 16 (13.0 ms against
// 14.8 ms with the reduction for 2 or more and 22 ms with atomics only).
constexpr int BWD_DIRECT_MAX = 16;
// The same for the two-pixels-per-lane backward, whose lanes add the terms
// of both their pixels: fastest at 20-24 (11.1 ms; 11.4 ms at 16, 11.9 ms
// at 8, 15.8 ms with atomics only on the same workload; re-measured on a
// later version: 10.13 ms at 24, 10.14 at 20, 10.61 at 28 and 11.39 with
// the reduction for every point).
constexpr int BWD_PAIR_DIRECT_MAX = 24;
// The persistent backward runs 8 x 8-pixel warps (two pixels per lane):
// 8 x 16 (four pixels per lane) examined 41% more pairs through the coarser
// cull and needed 80 registers (13.4 ms against 11.1).

// One warp back-propagates through sub-block `sub` of tile `tile`, taking
// the entries of its 8 x 8 block (`bit`) from its queue, back to front.
template <int TW, int TH, bool STORE>
__device__ __forceinline__ void bwd_stream_item(const Batch &b, const DevOpts &o, uint32_t tile,
                                                int sub, uint32_t bit, int lane,
                                                const uint2 *__restrict__ ranges,
                                                const uint32_t *__restrict__ keys,
                                                const uint32_t *__restrict__ pv_list,
                                                const float4 *__restrict__ rec,
                                                const float *__restrict__ T_final,
                                                const uint32_t *__restrict__ n_contrib,
                                                const float *__restrict__ grad_rgb,
                                                float *__restrict__ g2d, uint32_t &examined,
                                                uint32_t &used, float4 *wbuf, uint32_t *wpv,
                                                uint32_t *wpos, WarpQueue &q, const StoreBuf &sto)
{
    const PixelGeom g = pixel_geom<TW, TH>(b, tile, sub, lane);
    const uint32_t s = ranges[tile].x;
    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t L = 0, k = 0; // k: composited points not yet visited (store mode)
    int64_t pix = 0;
    if (g.inside) {
        pix = g.V->pix_base + (int64_t)g.y * g.V->W + g.x;
        if (STORE) k = sto.n[pix];
        T = T_final[pix];
        L = n_contrib[pix];
        g0 = grad_rgb[3 * pix];
        g1 = grad_rgb[3 * pix + 1];
        g2 = grad_rgb[3 * pix + 2];
    }
    float S = T * (o.bg[0] * g0 + o.bg[1] * g1 + o.bg[2] * g2);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
    if (wmax == 0) return;
    int64_t c = (int64_t)((wmax - 1) & ~31u);
    int qn = 0;
    uint32_t qh = 0;
    while (true) {
        queue_fill_back(keys, pv_list, s, wmax, bit, c, qn, qh, q, lane);
        if (qn == 0) break;
        uint32_t rel = 0, pv = 0;
        const int take = queue_take(q, qn, qh, lane, rel, pv);
        const bool valid = lane < take;
        float4 a = make_float4(0.f, 0.f, -1.f, 0.f);
        if (valid) a = __ldg(rec + 2 * (size_t)pv);
        // lanes whose composited list reaches the chunk's nearest entry; every
        // lane takes part in the reductions, whatever its entry
        const uint32_t lowest = __shfl_sync(0xffffffffu, rel, take - 1);
        const PixelGeom ar = active_rect(g, L > lowest);
        const bool hit = valid && disc_meets_rect(a, ar);
        uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            wbuf[lane] = a;
            wbuf[32 + lane] = __ldg(rec + 2 * (size_t)pv + 1);
            wpv[lane] = pv;
            wpos[lane] = rel;
        }
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1; // back to front: queue order
            m &= m - 1;
            const float4 aj = wbuf[j];
            const float4 cj = wbuf[32 + j];
            const bool before = wpos[j] < L;
            float dx, dy;
            const float d2 = pixel_d2(g.ux, g.uy, aj.x, aj.y, dx, dy);
            const bool contrib = before && d2 <= aj.z;
            examined += before;
            used += contrib;
            const uint32_t cm = __ballot_sync(0xffffffffu, contrib);
            if (cm) {
                float v[8];
                bool has_tb = false;
                float tb = 0.0f;
                if (STORE && contrib && --k < (uint32_t)sto.depth) {
                    has_tb = true;
                    tb = sto.T[pix * sto.depth + k];
                }
                pixel_adjoint_masked(contrib ? 1.0f : 0.0f, d2, dx, dy, aj, cj, o.alpha_max, g0,
                                     g1, g2, T, S, v, has_tb, tb);
                if (__popc(cm) > BWD_DIRECT_MAX) {
                    warp_add_terms(v, lane, g2d, wpv[j]);
                } else if (contrib) { // few pixels: each adds its own terms
                    float4 *dst = reinterpret_cast<float4 *>(g2d) + 2 * (size_t)wpv[j];
                    atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
                    atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], 0.f));
                }
            }
        }
        __syncwarp(); // chunk consumed before the buffers are refilled
    }
}

// Adjoint state of one pixel: T after its last composited point, the colour
// behind (S, starting from the background term), dL/dC and the list length.
struct BwdPixel {
    float T, S, g0, g1, g2;
    uint32_t L;
};

__device__ __forceinline__ BwdPixel bwd_pixel(const PixelGeom &g, const DevOpts &o,
                                              const float *__restrict__ T_final,
                                              const uint32_t *__restrict__ n_contrib,
                                              const float *__restrict__ grad_rgb)
{
    BwdPixel p{1.0f, 0.f, 0.f, 0.f, 0.f, 0u};
    if (g.inside) {
        const int64_t pix = g.V->pix_base + (int64_t)g.y * g.V->W + g.x;
        p.T = T_final[pix];
        p.L = n_contrib[pix];
        p.g0 = grad_rgb[3 * pix];
        p.g1 = grad_rgb[3 * pix + 1];
        p.g2 = grad_rgb[3 * pix + 2];
    }
    p.S = p.T * (o.bg[0] * p.g0 + o.bg[1] * p.g1 + o.bg[2] * p.g2);
    return p;
}

// Adjoint state of a lane's two pixels (see BwdPixel), packed.
struct BwdPair {
    float2 T, S, g0, g1, g2;
    uint32_t LA, LB;
};

// The adjoint of one composited point at both pixels of a lane (the
// operations of pixel_adjoint_masked, packed): take.x / take.y (0 or 1) say
// whether the point was composited at pixel A / B (0: its terms are 0 and
// T, S stay).  Returns the sum over the two pixels of the terms {ca dx,
// ca dy, ca d2, do, dr, dg, db} in v[0..6].
// Bit 0 / 1 of has_tb: tb.x / .y is the stored transmittance before the
// point at pixel A / B (store mode) instead of the one recovered by
// division.
__device__ __forceinline__ void pair_adjoint(float2 take, float2 d2, float dx, float2 dy,
                                             const float4 a, const float4 c, float amax,
                                             BwdPair &p, float v[8], uint32_t has_tb = 0u,
                                             float2 tb = {0.0f, 0.0f})
{
    const float2 e = mul2(d2, f2(a.w));
    const float2 G = make_float2(ex2_approx(e.x), ex2_approx(e.y));
    const float2 raw = mul2(f2(c.x), G);
    const float2 alpha = mul2(make_float2(fminf(amax, raw.x), fminf(amax, raw.y)), take);
    const float2 om = fma2(alpha, f2(-1.0f), f2(1.0f));
    const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    float2 Tb = mul2(p.T, rom);
    if (has_tb & 1u) Tb.x = tb.x;
    if (has_tb & 2u) Tb.y = tb.y;
    const float2 wgt = mul2(alpha, Tb);
    const float2 cg = fma2(f2(c.w), p.g2, fma2(f2(c.z), p.g1, mul2(f2(c.y), p.g0)));
    const float2 t4 = mul2(wgt, p.g0), t5 = mul2(wgt, p.g1), t6 = mul2(wgt, p.g2);
    v[4] = t4.x + t4.y;
    v[5] = t5.x + t5.y;
    v[6] = t6.x + t6.y;
    const float2 dalpha = mul2(fma2(Tb, cg, mul2(p.S, mul2(rom, f2(-1.0f)))), take);
    p.S = fma2(wgt, cg, p.S);
    p.T = Tb;
    // clamped alpha: no geometry terms
    const float2 ca0 = mul2(dalpha, alpha), dg0 = mul2(dalpha, G);
    const float2 ca = make_float2(raw.x < amax ? ca0.x : 0.0f, raw.y < amax ? ca0.y : 0.0f);
    const float2 t1 = mul2(ca, dy), t2 = mul2(ca, d2);
    v[0] = (ca.x + ca.y) * dx;
    v[1] = t1.x + t1.y;
    v[2] = t2.x + t2.y;
    v[3] = (raw.x < amax ? dg0.x : 0.0f) + (raw.y < amax ? dg0.y : 0.0f);
    v[7] = 0.0f;
}

// Backward of one 8 x 8 block (blocks numbered row-major, TW/8 per row) by
// one warp, for the persistent schedule: lane l owns the pixels A = (l & 7,
// l >> 3) and B = (l & 7, 4 + (l >> 3)).  The warp takes the tile list's
// entries with its block's bit (`bit`) from its queue, back to front.  Per
// listed point the lane forms the adjoint at both pixels (packed fp32x2)
// and adds the two term vectors, so the per-point warp work (staging, cull,
// reduction or atomics) serves 64 pixels.  Each pixel's T and S recursions
// are the one-pixel walk's operations.
// V, (tx, ty): the tile's view and position; s: the start of its list.
template <int TW, int TH, bool STATS, bool STORE>
__device__ __forceinline__ void bwd_pair_item(const DevView *V, int tx, int ty, uint32_t s,
                                              uint32_t bit, const DevOpts &o, int sub, int lane,
                                              const uint32_t *__restrict__ keys,
                                              const uint32_t *__restrict__ pv_list,
                                              const float4 *__restrict__ rec,
                                              const float *__restrict__ T_final,
                                              const uint32_t *__restrict__ n_contrib,
                                              const float *__restrict__ grad_rgb,
                                              float *__restrict__ g2d, uint32_t &examined,
                                              uint32_t &used, float4 *wbuf, uint2 *wpp,
                                              WarpQueue &q, const StoreBuf &sto)
{
    const int sx0 = tx * TW + (sub % (TW / 8)) * 8, sy0 = ty * TH + (sub / (TW / 8)) * 8;
    PixelGeom g[2];
    g[0] = pixel_geom_at(V, sx0, sy0, lane);
    g[1] = pixel_geom_at(V, sx0, sy0 + 4, lane);
    const BwdPixel pa = bwd_pixel(g[0], o, T_final, n_contrib, grad_rgb);
    const BwdPixel pb = bwd_pixel(g[1], o, T_final, n_contrib, grad_rgb);
    BwdPair p;
    p.T = make_float2(pa.T, pb.T);
    p.S = make_float2(pa.S, pb.S);
    p.g0 = make_float2(pa.g0, pb.g0);
    p.g1 = make_float2(pa.g1, pb.g1);
    p.g2 = make_float2(pa.g2, pb.g2);
    p.LA = pa.L;
    p.LB = pb.L;
    // store mode: composited points not yet visited, per pixel
    const int64_t pixA = STORE && g[0].inside ? pixel_index(g[0]) : 0;
    const int64_t pixB = STORE && g[1].inside ? pixel_index(g[1]) : 0;
    uint32_t kA = 0, kB = 0;
    if (STORE) {
        if (g[0].inside) kA = sto.n[pixA];
        if (g[1].inside) kB = sto.n[pixB];
    }
    const float ux = g[0].ux;
    const float2 uy = make_float2(g[0].uy, g[1].uy);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(pa.L, pb.L));
    if (wmax == 0) return;
    int64_t c = (int64_t)((wmax - 1) & ~31u);
    int qn = 0;
    uint32_t qh = 0;
    while (true) {
        queue_fill_back(keys, pv_list, s, wmax, bit, c, qn, qh, q, lane);
        if (qn == 0) break;
        uint32_t rel = 0, pv = 0;
        const int take = queue_take(q, qn, qh, lane, rel, pv);
        const bool valid = lane < take;
        float4 a = make_float4(0.f, 0.f, -1.f, 0.f);
        if (valid) a = __ldg(rec + 2 * (size_t)pv);
        // pixels whose composited list reaches the chunk's nearest entry; every
        // lane takes part in the reductions, whatever its entry
        const uint32_t lowest = __shfl_sync(0xffffffffu, rel, take - 1);
        const bool act[2] = {p.LA > lowest, p.LB > lowest};
        const PixelGeom ar = active_rect_rows<2>(g, act);
        const bool hit = valid && disc_meets_rect(a, ar);
        uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            wbuf[lane] = a;
            wbuf[32 + lane] = __ldg(rec + 2 * (size_t)pv + 1);
            wpp[lane] = make_uint2(rel, pv);
        }
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1; // back to front: queue order
            m &= m - 1;
            const float4 aj = wbuf[j];
            const uint2 pp = wpp[j]; // list position, point-view
            const uint32_t idx = pp.x;
            float dx;
            float2 dy;
            const float2 d2 = pair_d2(ux, uy, aj.x, aj.y, dx, dy);
            const bool bA = idx < p.LA, bB = idx < p.LB;
            const bool cA = bA && d2.x <= aj.z, cB = bB && d2.y <= aj.z;
            if (STATS) {
                examined += (uint32_t)bA + (uint32_t)bB;
                used += (uint32_t)cA + (uint32_t)cB;
            }
            const bool any = cA || cB;
            const uint32_t cm = __ballot_sync(0xffffffffu, any);
            if (cm) {
                float v[8];
                uint32_t has_tb = 0u;
                float2 tb = make_float2(0.0f, 0.0f);
                if (STORE) {
                    if (cA && --kA < (uint32_t)sto.depth) {
                        has_tb |= 1u;
                        tb.x = sto.T[pixA * sto.depth + kA];
                    }
                    if (cB && --kB < (uint32_t)sto.depth) {
                        has_tb |= 2u;
                        tb.y = sto.T[pixB * sto.depth + kB];
                    }
                }
                pair_adjoint(make_float2(cA ? 1.0f : 0.0f, cB ? 1.0f : 0.0f), d2, dx, dy, aj,
                             wbuf[32 + j], o.alpha_max, p, v, has_tb, tb);
                if (__popc(cm) > BWD_PAIR_DIRECT_MAX) {
                    warp_add_terms(v, lane, g2d, pp.y);
                } else if (any) { // few lanes: each adds its own terms
                    float4 *dst = reinterpret_cast<float4 *>(g2d) + 2 * (size_t)pp.y;
                    atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
                    atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], 0.f));
                }
            }
        }
        __syncwarp(); // chunk consumed before the buffers are refilled
    }
}

// Bit of the 8 x 8 block holding the 8 x 4 sub-block w of a TW-wide tile
// in the pair keys' block masks (0 when a tile is a single block).
template <int TW, int TH>
__device__ __forceinline__ uint32_t stream_block_bit(int w)
{
    constexpr int BPR = TW / 8;
    return block_bits(TW, TH) ? 1u << (((w / BPR) >> 1) * BPR + w % BPR) : 0u;
}

template <int TW, int TH, bool STORE>
__global__ void __launch_bounds__(TW * TH)
raster_fwd_stream_kernel(Batch b, DevOpts o, const uint2 *__restrict__ ranges,
                         const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pv_list,
                         const float4 *__restrict__ rec, float *__restrict__ out_rgb,
                         float *__restrict__ T_final, uint32_t *__restrict__ n_contrib,
                         unsigned long long *__restrict__ stats, StoreBuf sto)
{
    constexpr int NW = TW * TH / 32;
    __shared__ float4 s_buf[NW][64];
    __shared__ uint32_t s_pos[NW][32];
    __shared__ WarpQueue s_q[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ex = 0, co = 0;
    const uint2 rg = ranges[blockIdx.x];
    fwd_stream_item<true, STORE>(pixel_geom<TW, TH>(b, blockIdx.x, w, lane), rg.x,
                    rg.y > rg.x ? rg.y : rg.x,
                    stream_block_bit<TW, TH>(w), o, lane, keys, pv_list, rec, out_rgb, T_final,
                    n_contrib, ex, co, s_buf[w], s_pos[w], s_q[w], sto);
    add_stats(stats, ex, co, lane);
}

template <int TW, int TH, bool STORE>
__global__ void __launch_bounds__(TW * TH)
raster_bwd_stream_kernel(Batch b, DevOpts o, const uint2 *__restrict__ ranges,
                         const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pv_list,
                         const float4 *__restrict__ rec, const float *__restrict__ T_final,
                         const uint32_t *__restrict__ n_contrib, const float *__restrict__ grad_rgb,
                         float *__restrict__ g2d, unsigned long long *__restrict__ stats,
                         StoreBuf sto)
{
    constexpr int NW = TW * TH / 32;
    __shared__ float4 s_buf[NW][64];
    __shared__ uint32_t s_pv[NW][32];
    __shared__ uint32_t s_pos[NW][32];
    __shared__ WarpQueue s_q[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ex = 0, us = 0;
    bwd_stream_item<TW, TH, STORE>(b, o, blockIdx.x, w, stream_block_bit<TW, TH>(w), lane,
                                   ranges, keys,
                            pv_list, rec, T_final, n_contrib, grad_rgb, g2d, ex, us, s_buf[w],
                            s_pv[w], s_pos[w], s_q[w], sto);
    add_stats(stats ? stats + 2 : nullptr, ex, us, lane);
}

// ------------------------------------------------------------ persistent
// Persistent warps: each warp takes (tile, sub-block) items from an atomic
// counter over `order` (tiles sorted longest list first), so long tiles
// start early and no warp idles while work remains.
constexpr int PERSIST_THREADS = 256;
constexpr int FWD_PERSIST_BLOCKS = 5; // forward blocks per SM (see the kernel)

__device__ __forceinline__ uint32_t next_item(uint32_t *work, int lane)
{
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(work, 1u);
    return __shfl_sync(0xffffffffu, it, 0);
}

// Tile descriptor of the persistent order: {view, tx | ty << 16, list start,
// list end}, so that a warp starting an item needs one load, not a search
// of the view table, a division and the ranges.
__device__ __forceinline__ uint4 tile_desc(const Batch &b, const uint2 *ranges, uint32_t tile)
{
    const int v = find_view_by_tile(b, tile);
    const DevView &V = b.views[v];
    const uint32_t local = tile - V.tile_base;
    const uint32_t tx = local % (uint32_t)V.tiles_x, ty = local / (uint32_t)V.tiles_x;
    const uint2 r = ranges[tile];
    return make_uint4((uint32_t)v, tx | (ty << 16), r.x, r.y > r.x ? r.y : r.x);
}

// STATS: count examined / composited pairs into stats (which must then be
// non-null); without, the loops carry no counting.  The forward's 8 x 8
// warps run five blocks per SM (48 registers): 5.47 ms on the 1M-point,
// 64-view step against 5.66 at four (six spill).  The backward runs best at
// its natural four blocks (five: 11.1 -> 11.9 ms).
template <int TW, int TH, bool STATS, bool STORE>
__global__ void __launch_bounds__(PERSIST_THREADS, FWD_PERSIST_BLOCKS)
raster_fwd_persist_kernel(Batch b, DevOpts o, const uint2 *__restrict__ ranges,
                          const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pv_list,
                          const float4 *__restrict__ rec, float *__restrict__ out_rgb,
                          float *__restrict__ T_final, uint32_t *__restrict__ n_contrib,
                          unsigned long long *__restrict__ stats, const uint4 *__restrict__ order,
                          uint32_t *work, StoreBuf sto)
{
    constexpr uint32_t SUBS = (TW / 8) * (TH / 8);
    constexpr int NW = PERSIST_THREADS / 32;
    __shared__ float4 s_buf[NW][64];
    __shared__ uint32_t s_pos[NW][32];
    __shared__ WarpQueue s_q[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t n_items = b.n_tiles * SUBS;
    uint32_t ex = 0, co = 0;
    for (uint32_t it = next_item(work, lane); it < n_items; it = next_item(work, lane)) {
        const uint4 d = order[it / SUBS];
        const int sub = (int)(it % SUBS);
        const DevView *V = &b.views[d.x];
        const int sx0 = (int)(d.y & 0xffffu) * TW + (sub % (TW / 8)) * 8;
        const int sy0 = (int)(d.y >> 16) * TH + (sub / (TW / 8)) * 8;
        const uint32_t bit = block_bits(TW, TH) ? 1u << sub : 0u;
        fwd_pair_item<STATS, STORE>(pixel_geom_at(V, sx0, sy0, lane),
                                    pixel_geom_at(V, sx0, sy0 + 4, lane),
                             d.z, d.w, bit, o, lane, keys, pv_list, rec, out_rgb, T_final,
                             n_contrib, ex, co, s_buf[w], s_pos[w], s_q[w], sto);
    }
    if (STATS) add_stats(stats, ex, co, lane);
}

template <int TW, int TH, bool STATS, bool STORE>
__global__ void __launch_bounds__(PERSIST_THREADS)
raster_bwd_persist_kernel(Batch b, DevOpts o, const uint2 *__restrict__ ranges,
                          const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pv_list,
                          const float4 *__restrict__ rec, const float *__restrict__ T_final,
                          const uint32_t *__restrict__ n_contrib,
                          const float *__restrict__ grad_rgb, float *__restrict__ g2d,
                          unsigned long long *__restrict__ stats, const uint4 *__restrict__ order,
                          uint32_t *work, StoreBuf sto)
{
    // 8 x 8 blocks, numbered like the key masks
    constexpr uint32_t SUBS = (TW / 8) * (TH / 8);
    constexpr int NW = PERSIST_THREADS / 32;
    __shared__ float4 s_buf[NW][64];
    __shared__ uint2 s_pp[NW][32];
    __shared__ WarpQueue s_q[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t n_items = b.n_tiles * SUBS;
    uint32_t ex = 0, us = 0;
    for (uint32_t it = next_item(work, lane); it < n_items; it = next_item(work, lane)) {
        const uint4 d = order[it / SUBS];
        const int sub = (int)(it % SUBS);
        const uint32_t bit = block_bits(TW, TH) ? 1u << sub : 0u;
        bwd_pair_item<TW, TH, STATS, STORE>(&b.views[d.x], (int)(d.y & 0xffffu), (int)(d.y >> 16),
                                            d.z,
                                     bit, o, sub, lane, keys, pv_list, rec, T_final, n_contrib,
                                     grad_rgb, g2d, ex, us, s_buf[w], s_pp[w], s_q[w],
                                     sto);
    }
    if (STATS) add_stats(stats + 2, ex, us, lane);
}

// Tile order, longest list first: bucket = floor(log2(length)), buckets in
// descending order (order inside a bucket is arbitrary; it only affects
// scheduling).  work[0] = forward item counter, work[1] = backward item
// counter, work[2..34) = bucket counts / offsets.
__global__ void tile_bucket_count_kernel(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                         uint32_t *work)
{
    __shared__ uint32_t s_c[32];
    if (threadIdx.x < 32) s_c[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        atomicAdd(&s_c[31 - (len ? __clz(len) : 31)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32 && s_c[threadIdx.x]) atomicAdd(work + 2 + threadIdx.x, s_c[threadIdx.x]);
}

__global__ void tile_bucket_scan_kernel(uint32_t *work)
{
    if (threadIdx.x == 0) {
        work[0] = 0;
        work[1] = 0;
        uint32_t run = 0;
        for (int bkt = 31; bkt >= 0; --bkt) { // longest first
            const uint32_t c = work[2 + bkt];
            work[2 + bkt] = run;
            run += c;
        }
    }
}

// Stable inside a block: the block's tiles of one bucket keep their id
// order and take one contiguous range of the bucket (one atomic per block
// and bucket), so neighbouring tiles of similar length run close together
// in time and share their records through L2.
__global__ void __launch_bounds__(256)
tile_bucket_scatter_kernel(Batch b, const uint2 *__restrict__ ranges, uint32_t n_tiles,
                           uint32_t *work, uint4 *__restrict__ order)
{
    __shared__ uint32_t s_w[8][33]; // per warp and bucket: count, then offset
    __shared__ uint32_t s_base[32];
    const int w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < 8 * 33; j += 256) (&s_w[0][0])[j] = 0;
    __syncthreads();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bkt = 32; // none
    if (t < n_tiles) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        bkt = 31 - (len ? __clz(len) : 31);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, bkt);
    const uint32_t rank = __popc(peers & lanemask_lt_r());
    if (bkt < 32 && rank == 0) s_w[w][bkt] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 32) {
        const int b = threadIdx.x;
        uint32_t run = 0;
        for (int v = 0; v < 8; ++v) {
            const uint32_t c = s_w[v][b];
            s_w[v][b] = run;
            run += c;
        }
        s_base[b] = run ? atomicAdd(work + 2 + b, run) : 0u;
    }
    __syncthreads();
    if (bkt < 32) order[s_base[bkt] + s_w[w][bkt] + rank] = tile_desc(b, ranges, t);
}

// ========================================================= block-staged
// Builds, in shared memory, the ascending list of batch entries whose cutoff
// disc reaches the warp's rectangle.  Returns the count.
__device__ __forceinline__ int warp_cull(const float4 *s_a, int nb, const PixelGeom &g,
                                         uint16_t *list, int lane)
{
    int cnt = 0;
    const uint32_t lt = lanemask_lt_r();
    for (int k0 = 0; k0 < nb; k0 += 32) {
        const int k = k0 + lane;
        const bool hit = k < nb && disc_meets_rect(s_a[k], g);
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[cnt + __popc(m & lt)] = (uint16_t)k;
        cnt += __popc(m);
    }
    __syncwarp();
    return cnt;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
raster_fwd_staged_kernel(Batch b, DevOpts o, int depth, const uint2 *__restrict__ ranges,
                         const uint32_t *__restrict__ pv_list, const float4 *__restrict__ rec,
                         float *__restrict__ out_rgb, float *__restrict__ T_final,
                         uint32_t *__restrict__ n_contrib, unsigned long long *__restrict__ stats)
{
    constexpr int NT = TW * TH;
    extern __shared__ float4 s_rec[]; // [depth] a-part, [depth] b-part, per-warp lists
    float4 *s_a = s_rec, *s_b = s_rec + depth;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint16_t *s_list = (uint16_t *)(s_rec + 2 * depth) + w * depth;
    const uint32_t tile = blockIdx.x;
    const PixelGeom g = pixel_geom<TW, TH>(b, tile, w, lane);
    const uint2 rg = ranges[tile];
    const uint32_t s = rg.x, e = rg.y > rg.x ? rg.y : rg.x;

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t cnt = 0, last = 0, examined = 0;
    bool done = !g.inside;
    for (uint32_t base = s; base < e; base += depth) {
        if (__syncthreads_count(!done) == 0) break;
        const int nb = (int)min((uint32_t)depth, e - base);
        for (int k = threadIdx.x; k < nb; k += NT) {
            const uint32_t pv = pv_list[base + k];
            s_a[k] = rec[2 * (size_t)pv];
            s_b[k] = rec[2 * (size_t)pv + 1];
        }
        __syncthreads();
        if (!__any_sync(0xffffffffu, !done)) continue;
        const int nl = warp_cull(s_a, nb, g, s_list, lane);
        if (done) continue;
        int j = 0;
        for (; j < nl; ++j) {
            const int k = s_list[j];
            const float4 a = s_a[k];
            float dx, dy;
            const float d2 = pixel_d2(g.ux, g.uy, a.x, a.y, dx, dy);
            if (d2 <= a.z) {
                last = base + k - s + 1;
                if (pixel_blend(d2, a, s_b[k], o, T, C0, C1, C2, cnt)) {
                    done = true;
                    ++j;
                    break;
                }
            }
        }
        examined += j;
    }
    add_stats(stats, examined, cnt, lane);
    write_pixel(g, o, T, C0, C1, C2, last, out_rgb, T_final, n_contrib);
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
raster_bwd_staged_kernel(Batch b, DevOpts o, int depth, const uint2 *__restrict__ ranges,
                         const uint32_t *__restrict__ pv_list, const float4 *__restrict__ rec,
                         const float *__restrict__ T_final, const uint32_t *__restrict__ n_contrib,
                         const float *__restrict__ grad_rgb, float *__restrict__ g2d,
                         unsigned long long *__restrict__ stats)
{
    constexpr int NT = TW * TH;
    extern __shared__ float4 s_rec[];
    float4 *s_a = s_rec, *s_b = s_rec + depth;
    float *s_acc = (float *)(s_rec + 2 * depth); // [depth][8] block sums of the terms
    uint32_t *s_pv = (uint32_t *)(s_acc + 8 * depth);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint16_t *s_list = (uint16_t *)(s_pv + depth) + w * depth;
    __shared__ uint32_t s_max[NT / 32];
    const uint32_t tile = blockIdx.x;
    const PixelGeom g = pixel_geom<TW, TH>(b, tile, w, lane);
    const uint32_t s = ranges[tile].x;

    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t L = 0;
    if (g.inside) {
        const int64_t pix = g.V->pix_base + (int64_t)g.y * g.V->W + g.x;
        T = T_final[pix];
        L = n_contrib[pix];
        g0 = grad_rgb[3 * pix];
        g1 = grad_rgb[3 * pix + 1];
        g2 = grad_rgb[3 * pix + 2];
    }
    float S = T * (o.bg[0] * g0 + o.bg[1] * g1 + o.bg[2] * g2);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
    if (lane == 0) s_max[w] = wmax;
    __syncthreads();
    uint32_t maxL = 0;
#pragma unroll
    for (int j = 0; j < NT / 32; ++j) maxL = max(maxL, s_max[j]);

    uint32_t examined = 0, used = 0;
    for (int64_t bend = maxL; bend > 0; bend -= depth) {
        const uint32_t bstart = (uint32_t)(bend > depth ? bend - depth : 0);
        const int nb = (int)(bend - bstart);
        __syncthreads(); // previous batch fully consumed
        for (int k = threadIdx.x; k < nb; k += NT) {
            const uint32_t pv = pv_list[s + bstart + k];
            s_pv[k] = pv;
            s_a[k] = rec[2 * (size_t)pv];
            s_b[k] = rec[2 * (size_t)pv + 1];
            reinterpret_cast<float4 *>(s_acc)[2 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4 *>(s_acc)[2 * k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        // warps whose pixels all stop before this batch skip it
        const int nwb = bstart < wmax ? (int)min((uint32_t)nb, wmax - bstart) : 0;
        const int nl = nwb > 0 ? warp_cull(s_a, nwb, g, s_list, lane) : 0;
        for (int j = nl - 1; j >= 0; --j) {
            const int k = s_list[j];
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (bstart + k < L) {
                ++examined;
                const float4 a = s_a[k];
                float dx, dy;
                const float d2 = pixel_d2(g.ux, g.uy, a.x, a.y, dx, dy);
                if (d2 <= a.z) {
                    contrib = true;
                    ++used;
                    pixel_adjoint(d2, dx, dy, a, s_b[k], o.alpha_max, g0, g1, g2, T, S, v);
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float tot = warp_sum8_transposed(v, lane);
                const int which = (lane >> 2) & 7;
                if ((lane & 3) == 0 && which < 7) atomicAdd(s_acc + 8 * k + which, tot);
            }
        }
        __syncthreads();
        // one global atomic per (block, point, term)
        for (int t = threadIdx.x; t < nb * 7; t += NT) {
            const int k = t / 7, cc = t - 7 * k;
            const float val = s_acc[8 * k + cc];
            if (val != 0.f) atomicAdd(g2d + 8 * (size_t)s_pv[k] + cc, val);
        }
    }
    add_stats(stats ? stats + 2 : nullptr, examined, used, lane);
}

// ------------------------------------------------------------ dispatch
int persist_grid(const void *kernel)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, PERSIST_THREADS, 0);
    return sms * (per_sm > 0 ? per_sm : 1);
}

template <int TW, int TH, bool STATS, bool STORE>
void fwd_persist_launch(const Batch &b, const DevOpts &o, const uint2 *ranges,
                        const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                        float *out_rgb, float *T_final, uint32_t *n_contrib,
                        unsigned long long *stats, const uint4 *order, uint32_t *work,
                        cudaStream_t s, const StoreBuf &sto)
{
    static const int grid =
        persist_grid((const void *)raster_fwd_persist_kernel<TW, TH, STATS, STORE>);
    raster_fwd_persist_kernel<TW, TH, STATS, STORE><<<grid, PERSIST_THREADS, 0, s>>>(
        b, o, ranges, keys, pv_list, rec, out_rgb, T_final, n_contrib, stats, order, work, sto);
}

template <int TW, int TH, bool STATS, bool STORE>
void bwd_persist_launch(const Batch &b, const DevOpts &o, const uint2 *ranges,
                        const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                        const float *T_final, const uint32_t *n_contrib, const float *grad_rgb,
                        float4 *g2d, unsigned long long *stats, const uint4 *order, uint32_t *work,
                        cudaStream_t s, const StoreBuf &sto)
{
    static const int grid =
        persist_grid((const void *)raster_bwd_persist_kernel<TW, TH, STATS, STORE>);
    raster_bwd_persist_kernel<TW, TH, STATS, STORE><<<grid, PERSIST_THREADS, 0, s>>>(
        b, o, ranges, keys, pv_list, rec, T_final, n_contrib, grad_rgb, (float *)g2d, stats,
        order, work + 1, sto);
}

// The kernels are instantiated with and without pair counting (STATS) and
// store mode (STORE), so that the variants the graphs run carry neither.
template <int TW, int TH>
void fwd_dispatch(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                  const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                  float *out_rgb, float *T_final,
                  uint32_t *n_contrib, unsigned long long *stats, const uint4 *order,
                  uint32_t *work, cudaStream_t s, const StoreBuf &sto)
{
    const bool store = sto.T != nullptr;
    if (depth == 0 && order) {
        auto f = stats ? (store ? fwd_persist_launch<TW, TH, true, true>
                                : fwd_persist_launch<TW, TH, true, false>)
                       : (store ? fwd_persist_launch<TW, TH, false, true>
                                : fwd_persist_launch<TW, TH, false, false>);
        f(b, o, ranges, keys, pv_list, rec, out_rgb, T_final, n_contrib, stats, order, work, s,
          sto);
    } else if (depth == 0) {
        auto k = store ? raster_fwd_stream_kernel<TW, TH, true>
                       : raster_fwd_stream_kernel<TW, TH, false>;
        k<<<b.n_tiles, TW * TH, 0, s>>>(b, o, ranges, keys, pv_list, rec, out_rgb, T_final,
                                        n_contrib, stats, sto);
    } else {
        const size_t smem =
            (size_t)depth * (2 * sizeof(float4) + (TW * TH / 32) * sizeof(uint16_t));
        static const bool attr = cudaFuncSetAttribute(raster_fwd_staged_kernel<TW, TH>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      160 * 1024) == cudaSuccess;
        (void)attr;
        raster_fwd_staged_kernel<TW, TH><<<b.n_tiles, TW * TH, smem, s>>>(
            b, o, depth, ranges, pv_list, rec, out_rgb, T_final, n_contrib, stats);
    }
    count_launches(1);
}

template <int TW, int TH>
void bwd_dispatch(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                  const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                  const float *T_final,
                  const uint32_t *n_contrib, const float *grad_rgb, float4 *g2d,
                  unsigned long long *stats, const uint4 *order, uint32_t *work,
                  cudaStream_t s, const StoreBuf &sto)
{
    const bool store = sto.T != nullptr;
    if (depth == 0 && order) {
        auto f = stats ? (store ? bwd_persist_launch<TW, TH, true, true>
                                : bwd_persist_launch<TW, TH, true, false>)
                       : (store ? bwd_persist_launch<TW, TH, false, true>
                                : bwd_persist_launch<TW, TH, false, false>);
        f(b, o, ranges, keys, pv_list, rec, T_final, n_contrib, grad_rgb, g2d, stats, order, work,
          s, sto);
    } else if (depth == 0) {
        auto k = store ? raster_bwd_stream_kernel<TW, TH, true>
                       : raster_bwd_stream_kernel<TW, TH, false>;
        k<<<b.n_tiles, TW * TH, 0, s>>>(b, o, ranges, keys, pv_list, rec, T_final, n_contrib,
                                        grad_rgb, (float *)g2d, stats, sto);
    } else {
        const size_t smem = (size_t)depth * (4 * sizeof(float4) + sizeof(uint32_t) +
                                             (TW * TH / 32) * sizeof(uint16_t));
        static const bool attr = cudaFuncSetAttribute(raster_bwd_staged_kernel<TW, TH>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      160 * 1024) == cudaSuccess;
        (void)attr;
        raster_bwd_staged_kernel<TW, TH><<<b.n_tiles, TW * TH, smem, s>>>(
            b, o, depth, ranges, pv_list, rec, T_final, n_contrib, grad_rgb, (float *)g2d, stats);
    }
    count_launches(1);
}

} // namespace

void launch_tile_order(const Batch &b, const uint2 *ranges, uint32_t n_tiles, uint4 *order,
                       uint32_t *work, cudaStream_t s)
{
    cudaMemsetAsync(work, 0, 34 * sizeof(uint32_t), s);
    if (n_tiles == 0) return;
    const unsigned nb = (n_tiles + 255) / 256;
    tile_bucket_count_kernel<<<nb, 256, 0, s>>>(ranges, n_tiles, work);
    tile_bucket_scan_kernel<<<1, 32, 0, s>>>(work);
    tile_bucket_scatter_kernel<<<nb, 256, 0, s>>>(b, ranges, n_tiles, work, order);
    count_launches(3);
}

void reset_work_counters(uint32_t *work, cudaStream_t s)
{
    cudaMemsetAsync(work, 0, 2 * sizeof(uint32_t), s);
}

void launch_raster_fwd(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                       const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                       float *out_rgb, float *T_final, uint32_t *n_contrib,
                       unsigned long long *stats, cudaStream_t s, const uint4 *order,
                       uint32_t *work, const StoreBuf &sto)
{
    if (b.n_tiles == 0) return;
    if (o.tile_w == 8 && o.tile_h == 8)
        fwd_dispatch<8, 8>(b, o, depth, ranges, keys, pv_list, rec, out_rgb, T_final, n_contrib,
                           stats, order, work, s, sto);
    else if (o.tile_w == 16 && o.tile_h == 32)
        fwd_dispatch<16, 32>(b, o, depth, ranges, keys, pv_list, rec, out_rgb, T_final,
                             n_contrib, stats, order, work, s, sto);
    else
        fwd_dispatch<16, 16>(b, o, depth, ranges, keys, pv_list, rec, out_rgb, T_final,
                             n_contrib, stats, order, work, s, sto);
}

void launch_raster_bwd(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                       const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                       const float *T_final, const uint32_t *n_contrib, const float *grad_rgb,
                       float4 *g2d, unsigned long long *stats, cudaStream_t s,
                       const uint4 *order, uint32_t *work, const StoreBuf &sto)
{
    if (b.n_tiles == 0) return;
    if (o.tile_w == 8 && o.tile_h == 8)
        bwd_dispatch<8, 8>(b, o, depth, ranges, keys, pv_list, rec, T_final, n_contrib, grad_rgb,
                           g2d, stats, order, work, s, sto);
    else if (o.tile_w == 16 && o.tile_h == 32)
        bwd_dispatch<16, 32>(b, o, depth, ranges, keys, pv_list, rec, T_final, n_contrib,
                             grad_rgb, g2d, stats, order, work, s, sto);
    else
        bwd_dispatch<16, 16>(b, o, depth, ranges, keys, pv_list, rec, T_final, n_contrib,
                             grad_rgb, g2d, stats, order, work, s, sto);
}

} // namespace pbr
