// C entry points of the visual-hull initialisation and the consistency
// check (Sec. 3.1 and the appendix).
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_internal.h"

using namespace pbr;

namespace {

constexpr uint64_t SH_STREAM = 0x5DEECE66Dull; // SH draws: stream seed ^ this

// Views of the check on the device; validates cameras and z_near.
int upload_views(TempBufs &tb, const pbr_camera *cams, int32_t n_cams, float z_near,
                 HullView **d_views, cudaStream_t s)
{
    if (!cams || n_cams < 1 || !(z_near >= 0.0f) || !std::isfinite(z_near))
        return set_error(PBR_ERR_INVALID_ARG, "consistency check: bad cameras or z_near");
    std::vector<HullView> v(n_cams);
    int64_t base = 0;
    for (int i = 0; i < n_cams; ++i) {
        const pbr_camera &c = cams[i];
        if (c.width <= 0 || c.height <= 0)
            return set_error(PBR_ERR_INVALID_ARG, "camera %d: size", i);
        HullView &h = v[i];
        h.fx = c.fx;
        h.fy = c.fy;
        h.cx = c.cx;
        h.cy = c.cy;
        for (int k = 0; k < 9; ++k) h.R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) h.t[k] = c.t[k];
        h.W = c.width;
        h.H = c.height;
        h.pix_base = base;
        base += (int64_t)c.width * c.height;
    }
    PBR_TRY(tb.alloc(d_views, sizeof(HullView) * n_cams));
    PBR_CUDA(cudaMemcpyAsync(*d_views, v.data(), sizeof(HullView) * n_cams,
                             cudaMemcpyHostToDevice, s));
    return PBR_OK;
}

int read_u64(const unsigned long long *dev, unsigned long long *out, cudaStream_t s)
{
    PBR_CUDA(cudaMemcpyAsync(out, dev, sizeof(*out), cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    return PBR_OK;
}

} // namespace

extern "C" int pbr_consistency_check(pbr_ctx *ctx, const float *pos, int64_t n,
                                     const pbr_camera *cams, int32_t n_cams,
                                     const uint8_t *masks, float z_near, uint8_t *keep,
                                     pbr_stream_t stream)
{
    if (!ctx || n < 0 || (n > 0 && (!pos || !masks || !keep)))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_consistency_check: bad arguments");
    if (n == 0) return PBR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    TempBufs tb(s);
    HullView *views;
    PBR_TRY(upload_views(tb, cams, n_cams, z_near, &views, s));
    launch_consistency(pos, n, views, n_cams, masks, z_near, keep, nullptr, s);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_consistency_filter(pbr_ctx *ctx, const pbr_points *in, const pbr_camera *cams,
                                      int32_t n_cams, const uint8_t *masks, float z_near,
                                      float *out_pos, float *out_sh, float *out_opacity,
                                      float *out_radius, int64_t *n_out, pbr_stream_t stream)
{
    if (!ctx || !in || !n_out || in->n < 0 || in->n > 0x7fffffffLL || in->sh_degree < 0 ||
        in->sh_degree > 3)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_consistency_filter: bad arguments");
    *n_out = 0;
    const int64_t n = in->n;
    if (n == 0) return PBR_OK;
    if (!in->pos || !in->sh || !in->opacity || !in->radius || !masks || !out_pos || !out_sh ||
        !out_opacity || !out_radius)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_consistency_filter: null array");
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    const int nsh = 3 * (in->sh_degree + 1) * (in->sh_degree + 1);
    TempBufs tb(s);
    HullView *views;
    PBR_TRY(upload_views(tb, cams, n_cams, z_near, &views, s));
    uint32_t *keep, *newpos;
    void *stmp;
    unsigned long long *tot;
    PBR_TRY(tb.alloc(&keep, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&newpos, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&stmp, scan_temp_bytes(n)));
    PBR_TRY(tb.alloc(&tot, sizeof(unsigned long long)));
    launch_consistency(in->pos, n, views, n_cams, masks, z_near, nullptr, keep, s);
    launch_exclusive_scan(keep, newpos, n, tot, stmp, s);
    launch_compact_points(keep, newpos, n,
                          PointArrays{in->pos, in->sh, in->opacity, in->radius, nsh},
                          PointArraysOut{out_pos, out_sh, out_opacity, out_radius, nsh}, s);
    unsigned long long m = 0;
    PBR_TRY(read_u64(tot, &m, s));
    *n_out = (int64_t)m;
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_visual_hull_init(pbr_ctx *ctx, const float lo[3], const float hi[3],
                                    const pbr_camera *cams, int32_t n_cams, const uint8_t *masks,
                                    float z_near, uint64_t seed, int64_t n_target,
                                    int64_t max_candidates, int32_t sh_degree, float *out_pos,
                                    float *out_sh, int64_t *n_out, int64_t *n_drawn,
                                    pbr_stream_t stream)
{
    if (!ctx || !lo || !hi || !masks || !n_out || !n_drawn || n_target < 0 ||
        n_target > 0x7fffffffLL || max_candidates < 0 || sh_degree < 0 || sh_degree > 3 ||
        (n_target > 0 && !out_pos))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_visual_hull_init: bad arguments");
    float ext[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] >= lo[a]))
            return set_error(PBR_ERR_INVALID_ARG, "pbr_visual_hull_init: bad box");
        ext[a] = hi[a] - lo[a];
    }
    *n_out = 0;
    *n_drawn = 0;
    if (max_candidates == 0) max_candidates = 1ll << 40;
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    TempBufs tb(s);
    HullView *views;
    PBR_TRY(upload_views(tb, cams, n_cams, z_near, &views, s));
    constexpr int64_t BATCH = 1ll << 22;
    float *cand;
    uint32_t *flags, *rank;
    void *stmp;
    unsigned long long *tot, *last;
    PBR_TRY(tb.alloc(&cand, sizeof(float) * 3 * BATCH));
    PBR_TRY(tb.alloc(&flags, sizeof(uint32_t) * BATCH));
    PBR_TRY(tb.alloc(&rank, sizeof(uint32_t) * BATCH));
    PBR_TRY(tb.alloc(&stmp, scan_temp_bytes(BATCH)));
    PBR_TRY(tb.alloc(&tot, sizeof(unsigned long long)));
    PBR_TRY(tb.alloc(&last, sizeof(unsigned long long)));

    // batches of candidates in counter order; the first n_target accepted
    int64_t done = 0, drawn = 0;
    while (done < n_target && drawn < max_candidates) {
        const int64_t cnt = std::min<int64_t>(BATCH, max_candidates - drawn);
        launch_hull_candidates(seed, (uint64_t)drawn, cnt, lo, ext, views, n_cams, masks, z_near,
                               cand, flags, s);
        launch_exclusive_scan(flags, rank, cnt, tot, stmp, s);
        const uint32_t need = (uint32_t)(n_target - done);
        launch_hull_take(cand, flags, rank, cnt, need, out_pos, done, last, s);
        unsigned long long acc = 0;
        PBR_TRY(read_u64(tot, &acc, s));
        if ((int64_t)acc >= (int64_t)need) {
            unsigned long long li = 0;
            PBR_TRY(read_u64(last, &li, s));
            drawn += (int64_t)li + 1;
            done = n_target;
        } else {
            drawn += cnt;
            done += (int64_t)acc;
        }
    }
    // SH of the kept points: standard normals
    if (out_sh && done > 0) {
        const int64_t coef = 3ll * (sh_degree + 1) * (sh_degree + 1);
        launch_sh_normals(seed ^ SH_STREAM, 0, done * coef, out_sh, s);
    }
    *n_out = done;
    *n_drawn = drawn;
    PBR_CUDA(cudaGetLastError());
    PBR_CUDA(cudaStreamSynchronize(s));
    return PBR_OK;
}
