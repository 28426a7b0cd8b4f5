// Per-tile compositing of Sec. 3.2 and its adjoint.
//
// raster_fwd: one block per screen tile, one thread per pixel.  The tile's
// list (already ordered by depth, then point id) is staged through shared
// memory in batches of `depth` records.  Per pixel centre u and listed point
//   d2 = (ux - px)^2 + (uy - py)^2            (fp32, round-to-nearest, no FMA)
//   if d2 <= rc^2:                             (the cutoff of Sec. 3.2)
//     alpha = min(alpha_max, o * 2^(q' d2))    (Eq. 5, q' = -log2(e)/(2 s^2))
//     C += T alpha c ;  T *= (1 - alpha)       (Eqs. 6-7, front to back)
// stopping after the point that takes T below t_eps or reaches the count
// cap.  A block leaves the list as soon as every pixel in it has stopped
// (__syncthreads_count).  Writes C + T bg, T and the list position just
// after the last composited point.
//
// raster_bwd: same tiling, walking each pixel's list back to front from its
// last composited point.  T before a point is recovered as T_after/(1-alpha);
// S accumulates the colour behind the point, so
//   dL/dc     = alpha T g
//   dL/dalpha = T (c.g) - S / (1 - alpha)
// and, below the alpha_max clamp,
//   dL/do = dL/dalpha G,  dL/dp = dL/dalpha alpha q (u - p),
//   dL/dq = -dL/dalpha alpha d2 / 2          (q = 1/s^2).
// The 7 per-point terms of a warp are summed with a transposed shuffle
// reduction (9 shuffles) and added with one atomic per term per warp.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
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

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
raster_fwd_kernel(Batch b, DevOpts o, int depth, const uint2 *__restrict__ ranges,
                  const uint32_t *__restrict__ pv_list, const float4 *__restrict__ rec,
                  float *__restrict__ out_rgb, float *__restrict__ T_final,
                  uint32_t *__restrict__ n_contrib, unsigned long long *__restrict__ stats)
{
    extern __shared__ float4 s_rec[]; // [depth] a-part, then [depth] b-part
    float4 *s_a = s_rec, *s_b = s_rec + depth;
    const uint32_t tile = blockIdx.x;
    const DevView &V = b.views[find_view_by_tile(b, tile)];
    const uint32_t local = tile - V.tile_base;
    const int tx = (int)(local % (uint32_t)V.tiles_x), ty = (int)(local / (uint32_t)V.tiles_x);
    const int x = tx * TW + (int)(threadIdx.x % TW), y = ty * TH + (int)(threadIdx.x / TW);
    const bool inside = x < V.W && y < V.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const uint2 rg = ranges[tile];
    const uint32_t s = rg.x, e = rg.y > rg.x ? rg.y : rg.x;

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t cnt = 0, last = 0, examined = 0;
    bool done = !inside;
    const uint32_t maxpp = (uint32_t)o.max_per_pixel;
    for (uint32_t base = s; base < e; base += depth) {
        if (__syncthreads_count(!done) == 0) break;
        const int nb = (int)min((uint32_t)depth, e - base);
        for (int k = threadIdx.x; k < nb; k += TW * TH) {
            const uint32_t pv = pv_list[base + k];
            s_a[k] = rec[2 * (size_t)pv];
            s_b[k] = rec[2 * (size_t)pv + 1];
        }
        __syncthreads();
        if (!done) {
            int k = 0;
            for (; k < nb; ++k) {
                const float4 a = s_a[k];
                const float dx = __fsub_rn(ux, a.x), dy = __fsub_rn(uy, a.y);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                const float4 c = s_b[k];
                if (d2 <= c.w) {
                    const float alpha = fminf(o.alpha_max, a.w * ex2_approx(d2 * a.z));
                    const float w = alpha * T;
                    C0 = fmaf(w, c.x, C0);
                    C1 = fmaf(w, c.y, C1);
                    C2 = fmaf(w, c.z, C2);
                    T = T - w;
                    ++cnt;
                    last = base + k - s + 1;
                    if (T < o.t_eps || cnt == maxpp) {
                        done = true;
                        ++k;
                        break;
                    }
                }
            }
            examined += k;
        }
    }
    if (stats) { // pair counts for the ALU roofline: [0] examined, [1] composited
        const uint32_t we = __reduce_add_sync(0xffffffffu, examined);
        const uint32_t wc = __reduce_add_sync(0xffffffffu, cnt);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(stats, (unsigned long long)we);
            atomicAdd(stats + 1, (unsigned long long)wc);
        }
    }
    if (inside) {
        const int64_t pix = V.pix_base + (int64_t)y * V.W + x;
        out_rgb[3 * pix] = C0 + T * o.bg[0];
        out_rgb[3 * pix + 1] = C1 + T * o.bg[1];
        out_rgb[3 * pix + 2] = C2 + T * o.bg[2];
        T_final[pix] = T;
        n_contrib[pix] = last;
    }
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

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH)
raster_bwd_kernel(Batch b, DevOpts o, int depth, const uint2 *__restrict__ ranges,
                  const uint32_t *__restrict__ pv_list, const float4 *__restrict__ rec,
                  const float *__restrict__ T_final, const uint32_t *__restrict__ n_contrib,
                  const float *__restrict__ grad_rgb, float *__restrict__ g2d,
                  unsigned long long *__restrict__ stats)
{
    extern __shared__ float4 s_rec[];
    float4 *s_a = s_rec, *s_b = s_rec + depth;
    uint32_t *s_pv = (uint32_t *)(s_rec + 2 * depth);
    __shared__ uint32_t s_max[TW * TH / 32];
    const int lane = threadIdx.x & 31;
    const uint32_t tile = blockIdx.x;
    const DevView &V = b.views[find_view_by_tile(b, tile)];
    const uint32_t local = tile - V.tile_base;
    const int tx = (int)(local % (uint32_t)V.tiles_x), ty = (int)(local / (uint32_t)V.tiles_x);
    const int x = tx * TW + (int)(threadIdx.x % TW), y = ty * TH + (int)(threadIdx.x / TW);
    const bool inside = x < V.W && y < V.H;
    const float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    const uint2 rg = ranges[tile];
    const uint32_t s = rg.x;

    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t L = 0;
    if (inside) {
        const int64_t pix = V.pix_base + (int64_t)y * V.W + x;
        T = T_final[pix];
        L = n_contrib[pix];
        g0 = grad_rgb[3 * pix];
        g1 = grad_rgb[3 * pix + 1];
        g2 = grad_rgb[3 * pix + 2];
    }
    float S = T * (o.bg[0] * g0 + o.bg[1] * g1 + o.bg[2] * g2);
    // longest list prefix any pixel of the block needs
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
    if (lane == 0) s_max[threadIdx.x >> 5] = wmax;
    __syncthreads();
    uint32_t maxL = 0;
#pragma unroll
    for (int j = 0; j < TW * TH / 32; ++j) maxL = max(maxL, s_max[j]);

    uint32_t examined = 0, used = 0;
    for (int64_t bend = maxL; bend > 0; bend -= depth) {
        const uint32_t bstart = (uint32_t)(bend > depth ? bend - depth : 0);
        const int nb = (int)(bend - bstart);
        __syncthreads(); // previous batch fully consumed
        for (int k = threadIdx.x; k < nb; k += TW * TH) {
            const uint32_t pv = pv_list[s + bstart + k];
            s_pv[k] = pv;
            s_a[k] = rec[2 * (size_t)pv];
            s_b[k] = rec[2 * (size_t)pv + 1];
        }
        __syncthreads();
        for (int k = nb - 1; k >= 0; --k) {
            const uint32_t idx = bstart + k;
            float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (idx < L) {
                ++examined;
                const float4 a = s_a[k];
                const float dx = __fsub_rn(ux, a.x), dy = __fsub_rn(uy, a.y);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                const float4 c = s_b[k];
                if (d2 <= c.w) {
                    contrib = true;
                    ++used;
                    const float G = ex2_approx(d2 * a.z);
                    const float raw = a.w * G;
                    const float alpha = fminf(o.alpha_max, raw);
                    const float om = 1.0f - alpha;
                    const float Tb = __fdividef(T, om);
                    const float wgt = alpha * Tb;
                    const float cg = c.x * g0 + c.y * g1 + c.z * g2;
                    v[4] = wgt * g0;
                    v[5] = wgt * g1;
                    v[6] = wgt * g2;
                    const float dalpha = Tb * cg - __fdividef(S, om);
                    S = fmaf(wgt, cg, S);
                    T = Tb;
                    if (raw < o.alpha_max) {
                        const float q = a.z * QP_TO_Q;
                        const float ca = dalpha * alpha;
                        v[0] = ca * q * dx;
                        v[1] = ca * q * dy;
                        v[2] = -0.5f * ca * d2;
                        v[3] = dalpha * G;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float tot = warp_sum8_transposed(v, lane);
                const int which = (lane >> 2) & 7;
                if ((lane & 3) == 0 && which < 7) atomicAdd(g2d + 8 * (size_t)s_pv[k] + which, tot);
            }
        }
    }
    if (stats) { // [2] examined, [3] contributing
        const uint32_t we = __reduce_add_sync(0xffffffffu, examined);
        const uint32_t wu = __reduce_add_sync(0xffffffffu, used);
        if (lane == 0) {
            atomicAdd(stats + 2, (unsigned long long)we);
            atomicAdd(stats + 3, (unsigned long long)wu);
        }
    }
}

template <int TW, int TH>
void fwd_dispatch(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                  const uint32_t *pv_list, const float4 *rec, float *out_rgb, float *T_final,
                  uint32_t *n_contrib, unsigned long long *stats, cudaStream_t s)
{
    const size_t smem = (size_t)depth * 2 * sizeof(float4);
    raster_fwd_kernel<TW, TH><<<b.n_tiles, TW * TH, smem, s>>>(b, o, depth, ranges, pv_list, rec,
                                                              out_rgb, T_final, n_contrib, stats);
    count_launches(1);
}

template <int TW, int TH>
void bwd_dispatch(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                  const uint32_t *pv_list, const float4 *rec, const float *T_final,
                  const uint32_t *n_contrib, const float *grad_rgb, float4 *g2d,
                  unsigned long long *stats, cudaStream_t s)
{
    const size_t smem = (size_t)depth * (2 * sizeof(float4) + sizeof(uint32_t));
    raster_bwd_kernel<TW, TH><<<b.n_tiles, TW * TH, smem, s>>>(
        b, o, depth, ranges, pv_list, rec, T_final, n_contrib, grad_rgb, (float *)g2d, stats);
    count_launches(1);
}

} // namespace

void launch_raster_fwd(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                       const uint32_t *pv_list, const float4 *rec, float *out_rgb,
                       float *T_final, uint32_t *n_contrib, unsigned long long *stats,
                       cudaStream_t s)
{
    if (b.n_tiles == 0) return;
    if (o.tile_w == 8 && o.tile_h == 8)
        fwd_dispatch<8, 8>(b, o, depth, ranges, pv_list, rec, out_rgb, T_final, n_contrib, stats, s);
    else if (o.tile_w == 16 && o.tile_h == 32)
        fwd_dispatch<16, 32>(b, o, depth, ranges, pv_list, rec, out_rgb, T_final, n_contrib, stats, s);
    else
        fwd_dispatch<16, 16>(b, o, depth, ranges, pv_list, rec, out_rgb, T_final, n_contrib, stats, s);
}

void launch_raster_bwd(const Batch &b, const DevOpts &o, int depth, const uint2 *ranges,
                       const uint32_t *pv_list, const float4 *rec, const float *T_final,
                       const uint32_t *n_contrib, const float *grad_rgb, float4 *g2d,
                       unsigned long long *stats, cudaStream_t s)
{
    if (b.n_tiles == 0) return;
    if (o.tile_w == 8 && o.tile_h == 8)
        bwd_dispatch<8, 8>(b, o, depth, ranges, pv_list, rec, T_final, n_contrib, grad_rgb, g2d,
                           stats, s);
    else if (o.tile_w == 16 && o.tile_h == 32)
        bwd_dispatch<16, 32>(b, o, depth, ranges, pv_list, rec, T_final, n_contrib, grad_rgb, g2d,
                             stats, s);
    else
        bwd_dispatch<16, 16>(b, o, depth, ranges, pv_list, rec, T_final, n_contrib, grad_rgb, g2d,
                             stats, s);
}

} // namespace pbr
