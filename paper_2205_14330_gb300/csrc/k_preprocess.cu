// Per-point stages of the renderer.
//
// preprocess_fwd (Sec. 3.1 Eqs. 1-4, Sec. 3.2 cutoff): one thread per point,
// looping over every view of the point's scene, so position, radius,
// opacity and the [K,3] SH block are read from HBM once per batch.  For each
// (view, point) it writes a 32-byte record {px, py, rc^2, q'} {o, r, g, b},
// the fp32 depth bits (0xffffffff when the point-view lists no tile), the
// tile box with the mask of its listed tiles (one 16-byte record) and the
// tile count.
//
// The discrete decisions (cull, cutoff radius, pixel box, tile rectangle,
// depth key) use IEEE fp32 round-to-nearest operations with no
// contraction, in a fixed order, so they can be reproduced exactly:
//   X_a = ((R_a0 P0 + R_a1 P1) + R_a2 P2) + t_a
//   px = fx (X0 / X2) + cx,   py = fy (X1 / X2) + cy
//   s  = (fx r) / X2  (radius_mode 0)  or  (r min(W,H)) 0.5  (mode 1)
//   rc = cutoff_k s,  rc2 = rc rc
//   pixel box: [floor(px - rc) - 1, ceil(px + rc)] clamped to the image;
//   listed tiles: those holding a pixel (inside the image) whose centre
//   passes the per-pixel test d2 <= rc2 -- decided at the tile's pixel
//   centre nearest the splat centre (rect_reached).
//
// preprocess_bwd (Sec. 3.3): one thread per point; per view it chains the
// screen-space adjoint {dpx, dpy, dq, do, dr, dg, db} (q = 1/s^2; the
// compositing kernels leave dpx = q t0, dpy = q t1 and dq = -t2 / 2 to this
// stage, which applies the factors once per point-view) through the
// kernel width, the projection, the direction normalisation and the SH basis
// back to the point position, SH coefficients and opacity.  Views are
// visited in a fixed order, so the result does not depend on scheduling.
#include "pbr_internal.cuh"
#include "sh.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ int find_scene(const Batch &b, int64_t block)
{
    int s = 0;
    for (int j = 1; j < b.n_scenes; ++j)
        if (b.scenes[j].block_begin <= block) s = j;
    return s;
}

// Cooperative, coalesced copy of the block's SH coefficients into shared
// memory (the per-thread slice is then read with a stride of K*3 floats).
// The block's SH coefficients in shared memory, transposed and padded:
// coefficient j of the block's point p at s_sh[j * SH_STRIDE + p].  A
// thread walking its own point's coefficients then touches consecutive
// banks across the warp (a row-per-point layout of 48 floats puts threads
// two apart on the same bank), and the coalesced global read maps to
// consecutive banks too (SH_STRIDE = 1 mod 32).
constexpr int SH_STRIDE = PRE_THREADS + 1;

// f / K3 for 0 <= f <= 48 * PRE_THREADS by a multiply-high: with
// M = floor(2^32 / K3) + 1 = (2^32 + e) / K3, 0 < e <= K3, the product
// f M / 2^32 exceeds f / K3 by f e / (K3 2^32) < 1 / K3, so its floor is
// exact while f < 2^32 / K3.
__device__ __forceinline__ uint32_t div_k3(uint32_t f, uint32_t magic)
{
    return __umulhi(f, magic);
}

__device__ __forceinline__ uint32_t k3_magic(int K3)
{
    return 0xffffffffu / (uint32_t)K3 + 1u;
}

__device__ __forceinline__ void stage_sh(const float *__restrict__ sh, int64_t first, int count,
                                         int K3, float *s_sh)
{
    const int64_t base = first * K3;
    const int total = count * K3;
    const uint32_t magic = k3_magic(K3);
    for (int f = threadIdx.x; f < total; f += blockDim.x) {
        const int p = (int)div_k3((uint32_t)f, magic);
        s_sh[(f - p * K3) * SH_STRIDE + p] = __ldg(sh + base + f);
    }
}

template <int DEG>
__device__ void pre_fwd_point(const Batch &b, const DevOpts &o, const DevScene &sc, int64_t i,
                              const float *hs, float4 *__restrict__ rec,
                              uint32_t *__restrict__ zbits, uint32_t *__restrict__ ntiles,
                              uint8_t *__restrict__ nt8,
                              uint4 *__restrict__ rect, uint32_t &vis_cnt, uint32_t &pair_cnt,
                              uint32_t &zlo, uint32_t &zhi)
{
    constexpr int K = SH<DEG>::K;
    const float P0 = __ldg(sc.pos + 3 * i), P1 = __ldg(sc.pos + 3 * i + 1),
                P2 = __ldg(sc.pos + 3 * i + 2);
    const float r = __ldg(sc.radius + i);
    const float op = __ldg(sc.opacity + i);
    const int tws = __ffs(o.tile_w) - 1, ths = __ffs(o.tile_h) - 1;

    for (int vv = 0; vv < sc.view_count; ++vv) {
        const int v = b.view_list[sc.view_begin + vv];
        const DevView &V = b.views[v];
        const int64_t pv = V.pv_base + i;
        float X[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s = __fmul_rn(V.R[3 * a], P0);
            s = __fadd_rn(s, __fmul_rn(V.R[3 * a + 1], P1));
            s = __fadd_rn(s, __fmul_rn(V.R[3 * a + 2], P2));
            X[a] = __fadd_rn(s, V.t[a]);
        }
        const float z = X[2];
        uint32_t nt = 0;
        if (z > o.z_near) {
            const float px = __fadd_rn(__fmul_rn(V.fx, __fdiv_rn(X[0], z)), V.cx);
            const float py = __fadd_rn(__fmul_rn(V.fy, __fdiv_rn(X[1], z)), V.cy);
            float sg;
            if (o.radius_mode == 0)
                sg = __fdiv_rn(__fmul_rn(V.fx, r), z);
            else
                sg = __fmul_rn(__fmul_rn(r, (float)min(V.W, V.H)), 0.5f);
            const float rc = __fmul_rn(o.cutoff_k, sg);
            const float rc2 = __fmul_rn(rc, rc);
            int x0, x1, y0, y1;
            if (sg > 0.0f && pixel_box(px, py, rc, V.W, V.H, x0, x1, y0, y1)) do {
                // tile sizes are powers of two and the box is non-negative
                const int tx0 = x0 >> tws, tx1 = x1 >> tws;
                const int ty0 = y0 >> ths, ty1 = y1 >> ths;
                const int wx = tx1 - tx0 + 1, wy = ty1 - ty0 + 1;
                // listed tiles: those holding a pixel that passes the cutoff
                // test (rect_reached on the tile's pixels inside the image)
                uint32_t w = 0;
                if (wx * wy <= 32) {
                    int bit = 0;
                    for (int ty = ty0; ty <= ty1; ++ty) {
                        const int ya = ty << ths, yb = min(ya + o.tile_h, V.H) - 1;
                        for (int tx = tx0; tx <= tx1; ++tx, ++bit) {
                            const int xa = tx << tws, xb = min(xa + o.tile_w, V.W) - 1;
                            if (rect_reached(px, py, rc2, xa, xb, ya, yb)) w |= 1u << bit;
                        }
                    }
                    nt = (uint32_t)__popc(w);
                } else {
                    // wide box: per tile row, the listed tiles are one run
                    // around the column nearest the splat centre (the nearest
                    // pixel's distance grows away from it); walk it out
                    const int xn = (int)fminf(fmaxf(floorf(px), (float)x0), (float)x1);
                    const int tc = xn >> tws;
                    for (int ty = ty0; ty <= ty1; ++ty) {
                        const int ya = ty << ths, yb = min(ya + o.tile_h, V.H) - 1;
                        auto reached = [&](int tx) {
                            const int xa = tx << tws;
                            return rect_reached(px, py, rc2, xa, min(xa + o.tile_w, V.W) - 1, ya,
                                                yb);
                        };
                        if (!reached(tc)) continue;
                        int lo = tc, hi = tc;
                        while (lo > tx0 && reached(lo - 1)) --lo;
                        while (hi < tx1 && reached(hi + 1)) ++hi;
                        nt += (uint32_t)(hi - lo + 1);
                    }
                    w = nt;
                }
                if (nt == 0) break; // no pixel within reach: not visible
                ++vis_cnt;
                pair_cnt += nt;
                zlo = min(zlo, __float_as_uint(z));
                zhi = max(zhi, __float_as_uint(z));
                if (!rec) break; // counting only
                // view direction (Eq. 3) and colour (Eq. 4)
                const float inv = rsqrtf(X[0] * X[0] + X[1] * X[1] + z * z);
                float dx = X[0] * inv, dy = X[1] * inv, dz = z * inv;
                if (o.dir_frame == 1) {
                    const float wx = V.R[0] * dx + V.R[3] * dy + V.R[6] * dz;
                    const float wy = V.R[1] * dx + V.R[4] * dy + V.R[7] * dz;
                    const float wz = V.R[2] * dx + V.R[5] * dy + V.R[8] * dz;
                    dx = wx;
                    dy = wy;
                    dz = wz;
                }
                float Y[K];
                sh_basis<DEG>(dx, dy, dz, Y);
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    c0 = fmaf(hs[(3 * k) * SH_STRIDE], Y[k], c0);
                    c1 = fmaf(hs[(3 * k + 1) * SH_STRIDE], Y[k], c1);
                    c2 = fmaf(hs[(3 * k + 2) * SH_STRIDE], Y[k], c2);
                }
                const float qp = -0.5f * LOG2E / (sg * sg);
                rec[2 * pv] = make_float4(px, py, rc2, qp);
                rec[2 * pv + 1] = make_float4(op, c0, c1, c2);
                zbits[pv] = __float_as_uint(z);
                rect[pv] = make_uint4(__float_as_uint(px), __float_as_uint(py),
                                      __float_as_uint(rc), w);
            } while (0);
        }
        if (!rec) continue; // counting only: nothing is written
        ntiles[pv] = nt;
        nt8[pv] = (uint8_t)(nt < 255u ? nt : 255u);
        if (nt == 0) zbits[pv] = 0xffffffffu; // not visible: sorts behind every depth
    }
}

__global__ void __launch_bounds__(PRE_THREADS, 6)
preprocess_fwd_kernel(Batch b, DevOpts o, float4 *__restrict__ rec, uint32_t *__restrict__ zbits,
                      uint32_t *__restrict__ ntiles, uint8_t *__restrict__ nt8,
                      uint4 *__restrict__ rect,
                      unsigned long long *__restrict__ counters)
{
    __shared__ float s_sh[48 * SH_STRIDE];
    const int s = find_scene(b, blockIdx.x);
    const DevScene sc = b.scenes[s];
    const int64_t first = (int64_t)(blockIdx.x - sc.block_begin) * PRE_THREADS;
    const int count = (int)(sc.n - first < PRE_THREADS ? sc.n - first : PRE_THREADS);
    if (count <= 0) return; // whole block past the scene (uniform)
    const int K3 = sc.K * 3;
    stage_sh(sc.sh, first, count, K3, s_sh);
    __syncthreads();
    uint32_t vis = 0, pairs = 0, zlo = 0xffffffffu, zhi = 0u;
    if ((int)threadIdx.x < count) {
        const int64_t i = first + threadIdx.x;
        const float *hs = s_sh + threadIdx.x; // coefficient j at hs[j * SH_STRIDE]
        switch (sc.deg) {
        case 0: pre_fwd_point<0>(b, o, sc, i, hs, rec, zbits, ntiles, nt8, rect, vis, pairs, zlo, zhi); break;
        case 1: pre_fwd_point<1>(b, o, sc, i, hs, rec, zbits, ntiles, nt8, rect, vis, pairs, zlo, zhi); break;
        case 2: pre_fwd_point<2>(b, o, sc, i, hs, rec, zbits, ntiles, nt8, rect, vis, pairs, zlo, zhi); break;
        default: pre_fwd_point<3>(b, o, sc, i, hs, rec, zbits, ntiles, nt8, rect, vis, pairs, zlo, zhi); break;
        }
    }
    // per-warp totals, one atomic per warp: counters[0] pairs, [1] visible,
    // 32-bit words 12 / 13: smallest / largest depth bits of a visible pv
    vis = __reduce_add_sync(0xffffffffu, vis);
    pairs = __reduce_add_sync(0xffffffffu, pairs);
    zlo = __reduce_min_sync(0xffffffffu, zlo);
    zhi = __reduce_max_sync(0xffffffffu, zhi);
    if ((threadIdx.x & 31) == 0) {
        if (pairs) atomicAdd(counters, (unsigned long long)pairs);
        if (vis) {
            atomicAdd(counters + 1, (unsigned long long)vis);
            atomicMin((unsigned int *)counters + 12, zlo);
            atomicMax((unsigned int *)counters + 13, zhi);
        }
    }
}

// ------------------------------------------------------------- backward
// The screen-space terms of a point's views are fetched BWD_AHEAD views
// ahead with per-thread asynchronous copies into shared memory, so that
// their reads are in flight while earlier views are computed.
// BWD_AHEAD + 1 slots per thread: a slot is refilled one view after its
// contents were read.  Measured on the 1M-point, 64-view step: 1.27-1.29 ms
// at one or two views ahead, 1.37 ms at three or four (the deeper buffer
// takes shared memory from the L1 cache).
constexpr int BWD_AHEAD = 2;
constexpr int BWD_SLOTS = BWD_AHEAD + 1;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Starts the copy of view slot `vv`'s two float4 terms of point i into the
// thread's slot.  sg: this thread's slots, [slot][half] with a stride of
// PRE_THREADS float4 between entries.
__device__ __forceinline__ void fetch_view_terms(const Batch &b, const DevScene &sc, int64_t i,
                                                 int vv, const float4 *__restrict__ g2d,
                                                 float4 *sg)
{
    const int64_t pv = b.views[b.view_list[sc.view_begin + vv]].pv_base + i;
    float4 *dst = sg + (vv % BWD_SLOTS) * 2 * PRE_THREADS;
    cp_async16(dst, g2d + 2 * pv);
    cp_async16(dst + PRE_THREADS, g2d + 2 * pv + 1);
}

template <int DEG>
__device__ void pre_bwd_point(const Batch &b, const DevOpts &o, const DevScene &sc, int64_t i,
                              float *hs, float4 *sg, const float4 *__restrict__ g2d,
                              float *__restrict__ grad_pos, float *__restrict__ grad_opacity)
{
    constexpr int K = SH<DEG>::K;
    float dh[K * 3];
#pragma unroll
    for (int j = 0; j < K * 3; ++j) dh[j] = 0.0f;
    const float P0 = __ldg(sc.pos + 3 * i), P1 = __ldg(sc.pos + 3 * i + 1),
                P2 = __ldg(sc.pos + 3 * i + 2);
    const float r = __ldg(sc.radius + i);
    float dP0 = 0.f, dP1 = 0.f, dP2 = 0.f, dop = 0.f;

    const int nv = sc.view_count;
#pragma unroll
    for (int d = 0; d < BWD_AHEAD; ++d) {
        if (d < nv) fetch_view_terms(b, sc, i, d, g2d, sg);
        cp_async_commit(); // one group per view slot, empty past the end
    }
    for (int vv = 0; vv < nv; ++vv) {
        const int v = b.view_list[sc.view_begin + vv];
        const DevView &V = b.views[v];
        cp_async_wait<BWD_AHEAD - 1>(); // the copies of views 0..vv have landed
        const float4 *slot = sg + (vv % BWD_SLOTS) * 2 * PRE_THREADS;
        const float4 ga = slot[0];           // t0, t1, t2, do
        const float4 gb = slot[PRE_THREADS]; // dr, dg, db, -
        if (vv + BWD_AHEAD < nv) fetch_view_terms(b, sc, i, vv + BWD_AHEAD, g2d, sg);
        cp_async_commit();
        if (ga.x == 0.f && ga.y == 0.f && ga.z == 0.f && ga.w == 0.f && gb.x == 0.f &&
            gb.y == 0.f && gb.z == 0.f)
            continue; // culled or never composited
        float X[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            X[a] = V.R[3 * a] * P0 + V.R[3 * a + 1] * P1 + V.R[3 * a + 2] * P2 + V.t[a];
        const float z = X[2];
        float iz; // 1/z, approximate (gradient factors only)
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iz) : "f"(z));
        // the kernel width of this point-view and q = 1/s^2
        const float s = o.radius_mode == 0 ? V.fx * r * iz : r * (float)min(V.W, V.H) * 0.5f;
        float q; // 1/s^2, approximate as well
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(s * s));
        const float gpx = ga.x * q, gpy = ga.y * q, gq = -0.5f * ga.z;
        float dX0 = 0.f, dX1 = 0.f, dX2 = 0.f;
        // p = (fx X0/z + cx, fy X1/z + cy)
        dX0 += gpx * V.fx * iz;
        dX2 -= gpx * V.fx * X[0] * iz * iz;
        dX1 += gpy * V.fy * iz;
        dX2 -= gpy * V.fy * X[1] * iz * iz;
        // q = 1/s^2 = z^2 / (fx r)^2  =>  dq/dz = 2 q / z  (radius_mode 0)
        if (o.radius_mode == 0) dX2 += gq * 2.0f * iz * q;
        dop += ga.w;
        // colour: c = sum_k h_k Y_k(v)
        const float nrm2 = X[0] * X[0] + X[1] * X[1] + z * z;
        const float inv = rsqrtf(nrm2);
        const float vx = X[0] * inv, vy = X[1] * inv, vz = z * inv;
        float ux = vx, uy = vy, uz = vz;
        if (o.dir_frame == 1) {
            ux = V.R[0] * vx + V.R[3] * vy + V.R[6] * vz;
            uy = V.R[1] * vx + V.R[4] * vy + V.R[7] * vz;
            uz = V.R[2] * vx + V.R[5] * vy + V.R[8] * vz;
        }
        float Y[K], w[K];
        sh_basis<DEG>(ux, uy, uz, Y);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dh[3 * k] = fmaf(Y[k], gb.x, dh[3 * k]);
            dh[3 * k + 1] = fmaf(Y[k], gb.y, dh[3 * k + 1]);
            dh[3 * k + 2] = fmaf(Y[k], gb.z, dh[3 * k + 2]);
            w[k] = hs[(3 * k) * SH_STRIDE] * gb.x + hs[(3 * k + 1) * SH_STRIDE] * gb.y +
                   hs[(3 * k + 2) * SH_STRIDE] * gb.z;
        }
        if (DEG > 0) {
            float gx = 0.f, gy = 0.f, gz = 0.f;
            sh_grad_accum<DEG>(ux, uy, uz, w, gx, gy, gz);
            if (o.dir_frame == 1) { // u = R^T v  =>  dv = R du
                const float ax = V.R[0] * gx + V.R[1] * gy + V.R[2] * gz;
                const float ay = V.R[3] * gx + V.R[4] * gy + V.R[5] * gz;
                const float az = V.R[6] * gx + V.R[7] * gy + V.R[8] * gz;
                gx = ax;
                gy = ay;
                gz = az;
            }
            // v = X/|X|  =>  dX = (dv - v (v . dv)) / |X|
            const float vd = vx * gx + vy * gy + vz * gz;
            dX0 += (gx - vx * vd) * inv;
            dX1 += (gy - vy * vd) * inv;
            dX2 += (gz - vz * vd) * inv;
        }
        // X = R P + t  =>  dP = R^T dX
        dP0 += V.R[0] * dX0 + V.R[3] * dX1 + V.R[6] * dX2;
        dP1 += V.R[1] * dX0 + V.R[4] * dX1 + V.R[7] * dX2;
        dP2 += V.R[2] * dX0 + V.R[5] * dX1 + V.R[8] * dX2;
    }
    const int64_t gi = sc.point_base + i;
    grad_pos[3 * gi] = dP0;
    grad_pos[3 * gi + 1] = dP1;
    grad_pos[3 * gi + 2] = dP2;
    if (grad_opacity) grad_opacity[gi] = dop;
#pragma unroll
    for (int j = 0; j < K * 3; ++j) hs[j * SH_STRIDE] = dh[j];
}

__global__ void __launch_bounds__(PRE_THREADS)
preprocess_bwd_kernel(Batch b, DevOpts o, const float4 *__restrict__ g2d,
                      float *__restrict__ grad_pos, float *__restrict__ grad_sh,
                      float *__restrict__ grad_opacity)
{
    __shared__ float s_sh[48 * SH_STRIDE];
    __shared__ float4 s_g[BWD_SLOTS * 2 * PRE_THREADS]; // [slot][half][thread]
    const int s = find_scene(b, blockIdx.x);
    const DevScene sc = b.scenes[s];
    const int64_t first = (int64_t)(blockIdx.x - sc.block_begin) * PRE_THREADS;
    const int count = (int)(sc.n - first < PRE_THREADS ? sc.n - first : PRE_THREADS);
    if (count <= 0) return;
    const int K3 = sc.K * 3;
    stage_sh(sc.sh, first, count, K3, s_sh);
    __syncthreads();
    if ((int)threadIdx.x < count) {
        const int64_t i = first + threadIdx.x;
        float *hs = s_sh + threadIdx.x; // coefficient j at hs[j * SH_STRIDE]
        float4 *sg = s_g + threadIdx.x;
        switch (sc.deg) {
        case 0: pre_bwd_point<0>(b, o, sc, i, hs, sg, g2d, grad_pos, grad_opacity); break;
        case 1: pre_bwd_point<1>(b, o, sc, i, hs, sg, g2d, grad_pos, grad_opacity); break;
        case 2: pre_bwd_point<2>(b, o, sc, i, hs, sg, g2d, grad_pos, grad_opacity); break;
        default: pre_bwd_point<3>(b, o, sc, i, hs, sg, g2d, grad_pos, grad_opacity); break;
        }
    }
    __syncthreads();
    // coalesced write-back of the SH gradient slice
    float *dst = grad_sh + sc.sh_base + first * K3;
    const int total = count * K3;
    const uint32_t magic = k3_magic(K3);
    for (int f = threadIdx.x; f < total; f += blockDim.x) {
        const int p = (int)div_k3((uint32_t)f, magic);
        dst[f] = s_sh[(f - p * K3) * SH_STRIDE + p];
    }
}

} // namespace

void launch_preprocess_fwd(const Batch &b, const DevOpts &o, float4 *rec, uint32_t *zbits,
                           uint32_t *ntiles, uint8_t *nt8, uint4 *rect,
                           unsigned long long *counters, cudaStream_t s)
{
    if (b.n_point_blocks <= 0) return;
    preprocess_fwd_kernel<<<(unsigned)b.n_point_blocks, PRE_THREADS, 0, s>>>(
        b, o, rec, zbits, ntiles, nt8, rect, counters);
    count_launches(1);
}

void launch_preprocess_bwd(const Batch &b, const DevOpts &o, const float4 *g2d, float *grad_pos,
                           float *grad_sh, float *grad_opacity, cudaStream_t s)
{
    if (b.n_point_blocks <= 0) return;
    preprocess_bwd_kernel<<<(unsigned)b.n_point_blocks, PRE_THREADS, 0, s>>>(
        b, o, g2d, grad_pos, grad_sh, grad_opacity);
    count_launches(1);
}

} // namespace pbr
