// C ABI of libpbr (declared in include/pbr.h): argument checking, batch
// layout, workspace management and the launch sequence of the forward and
// backward passes of the point-splat renderer (Sec. 3.1-3.3).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pbr.h"
#include "pbr_internal.cuh"
#include "api_internal.h"

using namespace pbr;

// --------------------------------------------------- launches and timing
static std::atomic<unsigned long long> g_launches{0};
void pbr::count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }
unsigned long long pbr::launches_total() { return g_launches.load(); }
extern "C" unsigned long long pbr_kernel_launches(void) { return g_launches.load(); }

static cudaEvent_t take_event(pbr_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

pbr::StageScope::StageScope(pbr_ctx *c, int stage, cudaStream_t s) : c_(c), stage_(stage), s_(s)
{
    if (!c_ || !c_->timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s_, &cs);
    if (cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> g(c_->timing_mu);
    a_ = take_event(c_);
    cudaEventRecord(a_, s_);
}

pbr::StageScope::~StageScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> g(c_->timing_mu);
    cudaEvent_t b = take_event(c_);
    cudaEventRecord(b, s_);
    c_->pending.push_back({stage_, a_, b});
}

extern "C" int pbr_set_stage_timing(pbr_ctx *c, int enable)
{
    if (!c) return PBR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(c->timing_mu);
    c->timing = enable != 0;
    return PBR_OK;
}

extern "C" int pbr_stage_times(pbr_ctx *c, double *ms, long long *calls, int n)
{
    if (!c) return PBR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(c->timing_mu);
    for (auto &r : c->pending) {
        cudaEventSynchronize(r.b);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            c->stage_ms[r.stage] += t;
            c->stage_calls[r.stage] += 1;
        }
        c->event_pool.push_back(r.a);
        c->event_pool.push_back(r.b);
    }
    c->pending.clear();
    for (int i = 0; i < n && i < STG_COUNT; ++i) {
        if (ms) ms[i] = c->stage_ms[i];
        if (calls) calls[i] = c->stage_calls[i];
        c->stage_ms[i] = 0.0;
        c->stage_calls[i] = 0;
    }
    return PBR_OK;
}

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int pbr::set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

extern "C" const char *pbr_last_error(const pbr_ctx *) { return g_err.c_str(); }

extern "C" const char *pbr_version(void) { return "pbr 0.1 (sm_103a)"; }

extern "C" void pbr_default_opts(pbr_render_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->radius_mode = 0;
    o->dir_frame = 0;
    o->cutoff_k = 3.0f;
    o->alpha_max = 0.99f;
    o->t_eps = 1e-5f;
    o->max_per_pixel = 0;
    o->z_near = 0.01f;
    o->tile_w = 16;
    o->tile_h = 16;
    o->batch_depth = 0;
}

// ---------------------------------------------------------------- context
extern "C" int pbr_create(pbr_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return set_error(PBR_ERR_INVALID_ARG, "pbr_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_create: no CUDA device %d", device);
    PBR_CUDA(cudaSetDevice(device));
    pbr_ctx *c = new pbr_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    c->hbm_budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    // keep freed stream-ordered allocations cached in the device pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMallocHost(&c->host_counters, 64) != cudaSuccess) {
        delete c;
        return set_error(PBR_ERR_OOM, "pbr_create: pinned host buffer");
    }
    *out = c;
    return PBR_OK;
}

extern "C" int pbr_destroy(pbr_ctx *c)
{
    if (!c) return PBR_OK;
    serve_shutdown(c);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->host_counters) cudaFreeHost(c->host_counters);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return PBR_OK;
}

// ----------------------------------------------------------- validation
int pbr::check_opts(const pbr_render_opts *o)
{
    if (!o) return set_error(PBR_ERR_INVALID_ARG, "opts is NULL");
    const bool tile_ok = (o->tile_w == 8 && o->tile_h == 8) || (o->tile_w == 16 && o->tile_h == 16) ||
                         (o->tile_w == 16 && o->tile_h == 32);
    if (!tile_ok) return set_error(PBR_ERR_INVALID_ARG, "tile must be 8x8, 16x16 or 16x32");
    if (o->batch_depth != 0 && (o->batch_depth < 32 || o->batch_depth > 1024 || (o->batch_depth & 31)))
        return set_error(PBR_ERR_INVALID_ARG,
                         "batch_depth must be 0 (warp-streamed) or a multiple of 32 in [32,1024]");
    if (!(o->alpha_max > 0.f && o->alpha_max < 1.f))
        return set_error(PBR_ERR_INVALID_ARG, "alpha_max must be in (0,1)");
    if (!(o->t_eps >= 0.f) || !(o->cutoff_k > 0.f) || o->max_per_pixel < 0)
        return set_error(PBR_ERR_INVALID_ARG, "t_eps >= 0, cutoff_k > 0, max_per_pixel >= 0");
    if (o->radius_mode < 0 || o->radius_mode > 1 || o->dir_frame < 0 || o->dir_frame > 1)
        return set_error(PBR_ERR_INVALID_ARG, "radius_mode and dir_frame are 0 or 1");
    if (o->no_pair_stats < 0 || o->no_pair_stats > 1)
        return set_error(PBR_ERR_INVALID_ARG, "no_pair_stats is 0 or 1");
    if (o->bwd_mode < 0 || o->bwd_mode > 2 || o->store_depth < 0 || o->store_depth > 255)
        return set_error(PBR_ERR_INVALID_ARG, "bwd_mode in 0..2, store_depth in 0..255");
    return PBR_OK;
}

DevOpts pbr::dev_opts(const pbr_render_opts *o)
{
    DevOpts d;
    d.radius_mode = o->radius_mode;
    d.dir_frame = o->dir_frame;
    d.cutoff_k = o->cutoff_k;
    d.alpha_max = o->alpha_max;
    // Compositing stops once T falls below t_eps, and never lets T leave the
    // normal fp32 range: the backward recovers T before each point by
    // dividing by (1 - alpha), which fails once T has been flushed to zero
    // (after a few thousand faint layers at t_eps = 0).  What is left behind
    // T < 1e-30 weighs less than 1e-30 of the colour scale.
    d.t_eps = o->t_eps > T_EPS_FLOOR ? o->t_eps : T_EPS_FLOOR;
    d.max_per_pixel = o->max_per_pixel;
    for (int i = 0; i < 3; ++i) d.bg[i] = o->bg[i];
    d.z_near = o->z_near;
    d.tile_w = o->tile_w;
    d.tile_h = o->tile_h;
    return d;
}

int pbr::build_layout(const pbr_points *scenes, int32_t n_scenes, const int32_t *scene_of_view,
                      const pbr_camera *cams, int32_t n_cams, const pbr_render_opts *o,
                      HostLayout &L)
{
    if (n_scenes <= 0 || !scenes) return set_error(PBR_ERR_INVALID_ARG, "no scenes");
    if (n_cams <= 0 || !cams) return set_error(PBR_ERR_INVALID_ARG, "no cameras");
    L.views.resize(n_cams);
    L.scenes.resize(n_scenes);
    int64_t pbase = 0, shbase = 0, blk = 0;
    for (int s = 0; s < n_scenes; ++s) {
        const pbr_points &p = scenes[s];
        if (p.n < 0 || p.sh_degree < 0 || p.sh_degree > 3)
            return set_error(PBR_ERR_INVALID_ARG, "scene %d: n >= 0 and sh_degree in 0..3", s);
        if (p.n > 0 && (!p.pos || !p.sh || !p.opacity || !p.radius))
            return set_error(PBR_ERR_INVALID_ARG, "scene %d: NULL point array", s);
        DevScene &d = L.scenes[s];
        d.pos = p.pos;
        d.sh = p.sh;
        d.opacity = p.opacity;
        d.radius = p.radius;
        d.n = p.n;
        d.deg = p.sh_degree;
        d.K = (p.sh_degree + 1) * (p.sh_degree + 1);
        d.point_base = pbase;
        d.sh_base = shbase;
        d.block_begin = blk;
        d.view_begin = 0;
        d.view_count = 0;
        pbase += p.n;
        shbase += p.n * d.K * 3;
    }
    std::vector<int32_t> sov(n_cams, 0);
    for (int v = 0; v < n_cams; ++v) {
        sov[v] = scene_of_view ? scene_of_view[v] : 0;
        if (sov[v] < 0 || sov[v] >= n_scenes)
            return set_error(PBR_ERR_INVALID_ARG, "scene_of_view[%d] out of range", v);
    }
    // view list grouped by scene (stable)
    L.view_list.resize(n_cams);
    for (int v = 0; v < n_cams; ++v) L.view_list[v] = v;
    std::stable_sort(L.view_list.begin(), L.view_list.end(),
                     [&](int a, int b) { return sov[a] < sov[b]; });
    for (int j = 0; j < n_cams; ++j) {
        DevScene &d = L.scenes[sov[L.view_list[j]]];
        if (d.view_count == 0) d.view_begin = j;
        d.view_count++;
    }
    // point-parallel grid: every scene with views gets ceil(n/PRE_THREADS) blocks
    for (int s = 0; s < n_scenes; ++s) {
        DevScene &d = L.scenes[s];
        d.block_begin = blk;
        if (d.view_count > 0) blk += (d.n + PRE_THREADS - 1) / PRE_THREADS;
    }
    L.n_point_blocks = blk;
    int64_t pv = 0, pix = 0;
    uint64_t tiles = 0;
    for (int v = 0; v < n_cams; ++v) {
        const pbr_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 32768 || c.height > 32768)
            return set_error(PBR_ERR_INVALID_ARG, "camera %d: size %dx%d", v, c.width, c.height);
        DevView &d = L.views[v];
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        std::memcpy(d.R, c.R, sizeof d.R);
        std::memcpy(d.t, c.t, sizeof d.t);
        d.W = c.width;
        d.H = c.height;
        d.tiles_x = (c.width + o->tile_w - 1) / o->tile_w;
        d.tiles_y = (c.height + o->tile_h - 1) / o->tile_h;
        d.tile_base = (uint32_t)tiles;
        d.scene = sov[v];
        d.pix_base = pix;
        d.pv_base = pv;
        d.out = nullptr;
        tiles += (uint64_t)d.tiles_x * d.tiles_y;
        pix += (int64_t)c.width * c.height;
        pv += scenes[sov[v]].n;
    }
    // tile ids and their 8 x 8 block masks share the 32-bit pair keys
    const int sb = block_bits(o->tile_w, o->tile_h);
    if (pv >= (int64_t)UINT32_MAX || tiles >= (UINT32_MAX >> sb))
        return set_error(PBR_ERR_CAPACITY, "batch too large: %lld point-views, %llu tiles",
                         (long long)pv, (unsigned long long)tiles);
    L.n_pv = pv;
    L.n_pix = pix;
    L.n_tiles = (uint32_t)tiles;
    L.n_points_total = pbase;
    L.n_sh_total = shbase;
    return PBR_OK;
}

// ------------------------------------------------------------ allocation
int pbr::dalloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PBR_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    return PBR_OK;
}

void pbr::dfree(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

static int key_bits_for(uint32_t n_keys)
{
    int b = 0;
    while (b < 32 && (n_keys - 1) >> b) ++b;
    return b < 1 ? 1 : b;
}

int32_t pbr::resolve_store_depth(const pbr_ctx *c, const pbr_render_opts *o, int64_t n_pix,
                                 bool keep_state)
{
    if (!keep_state || o->bwd_mode == 1 || o->batch_depth != 0) return 0;
    const int32_t depth = o->store_depth > 0 ? o->store_depth : 32;
    if (o->bwd_mode == 2) return depth;
    return store_bytes(depth, n_pix) <= c->hbm_budget / 8 ? depth : 0;
}

size_t pbr::store_bytes(int32_t store_depth, int64_t n_pix)
{
    return store_depth > 0 ? (size_t)(4 * (int64_t)store_depth + 4) * (size_t)n_pix : 0;
}

void pbr_state::release()
{
    void **all[] = {(void **)&d_views, (void **)&d_scenes, (void **)&d_view_list, (void **)&rec,
                    (void **)&ntiles, (void **)&counters, (void **)&tile_keys,
                    (void **)&tile_vals, (void **)&ranges, (void **)&T_final,
                    (void **)&n_contrib, (void **)&tile_order, (void **)&work,
                    (void **)&T_store, (void **)&n_comp};
    for (void **p : all) {
        dfree(*p, stream);
        *p = nullptr;
    }
}

// Runs the forward chain into the state's buffers.  Exact-size workspaces:
// one host synchronisation after the per-point stage reads the pair count.
int pbr::forward_eager(pbr_ctx *c, pbr_state *st, float *out_rgb, cudaStream_t s)
{
    HostLayout &L = st->layout;
    const DevOpts &o = st->dopts;
    // tables
    PBR_TRY(dalloc((void **)&st->d_views, sizeof(DevView) * L.views.size(), s));
    PBR_TRY(dalloc((void **)&st->d_scenes, sizeof(DevScene) * L.scenes.size(), s));
    PBR_TRY(dalloc((void **)&st->d_view_list, sizeof(int32_t) * L.view_list.size(), s));
    PBR_CUDA(cudaMemcpyAsync(st->d_views, L.views.data(), sizeof(DevView) * L.views.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(st->d_scenes, L.scenes.data(), sizeof(DevScene) * L.scenes.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(st->d_view_list, L.view_list.data(),
                             sizeof(int32_t) * L.view_list.size(), cudaMemcpyHostToDevice, s));
    Batch b = st->batch();
    const int64_t npv = L.n_pv;
    PBR_TRY(dalloc((void **)&st->rec, sizeof(float4) * 2 * npv, s));
    PBR_TRY(dalloc((void **)&st->ntiles, sizeof(uint32_t) * npv, s));
    PBR_TRY(dalloc((void **)&st->counters, 128, s));
    TempBufs tmp(s);
    uint32_t *zbits = nullptr;
    uint4 *rect = nullptr;
    uint8_t *nt8 = nullptr;
    PBR_TRY(tmp.alloc(&zbits, sizeof(uint32_t) * npv));
    PBR_TRY(tmp.alloc(&rect, sizeof(uint4) * npv));
    PBR_TRY(tmp.alloc(&nt8, (size_t)npv));
    PBR_CUDA(cudaMemsetAsync(st->counters, 0, 128, s));
    PBR_CUDA(cudaMemsetAsync((char *)st->counters + 48, 0xff, 4, s)); // depth-bits minimum
    {
        StageScope t(c, STG_PREPROCESS_FWD, s);
        launch_preprocess_fwd(b, o, st->rec, zbits, st->ntiles, nt8, rect, st->counters, s);
    }
    PBR_CUDA(cudaGetLastError());
    // size the lists (pinned read-back buffer per host thread: the serving
    // thread and callers may run forward passes concurrently)
    static thread_local unsigned long long *host = nullptr;
    if (!host) PBR_CUDA(cudaMallocHost((void **)&host, 64));
    PBR_CUDA(cudaMemcpyAsync(host, st->counters, 64, cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    const uint64_t n_pairs = host[0], n_vis = host[1];
    const uint32_t zlo = ((const uint32_t *)host)[12];
    const uint32_t zhi = ((const uint32_t *)host)[13];
    // With most point-views visible, all of them are sorted by depth
    // directly: the invisible ones (key 0xffffffff, clamped to one above the
    // deepest visible key) land behind the visible ones, and no compaction
    // pass is needed.  Otherwise the visible ones are compacted first.
    const bool direct = n_vis > 0 && 4 * n_vis >= 3 * (uint64_t)npv;
    const uint32_t marker = n_vis > 0 ? zhi - zlo + 1 : 0u;
    const int depth_bits = direct ? 32 - __builtin_clz(marker)
                                  : (n_vis > 0 && zhi > zlo) ? 32 - __builtin_clz(zhi - zlo) : 0;
    const int64_t n_sort = direct ? npv : (int64_t)n_vis;
    if (n_pairs >= UINT32_MAX) {
        return set_error(PBR_ERR_CAPACITY, "%llu (tile, point-view) pairs exceed 2^32-1",
                         (unsigned long long)n_pairs);
    }
    st->n_vis = (int64_t)n_vis;
    st->n_pairs = (int64_t)n_pairs;
    uint32_t *vk = nullptr, *vv = nullptr, *vk2 = nullptr, *vv2 = nullptr;
    uint32_t *pk2 = nullptr, *pv2 = nullptr;
    void *temp = nullptr;
    const int64_t cap_sort = std::max<int64_t>(n_sort, n_pairs);
    const size_t temp_bytes = std::max(std::max(scan_temp_bytes(npv), radix_temp_bytes(cap_sort)),
                                       emit_temp_bytes((int64_t)n_vis));
    if (!direct) PBR_TRY(tmp.alloc(&vk, sizeof(uint32_t) * n_sort));
    PBR_TRY(tmp.alloc(&vv, sizeof(uint32_t) * n_sort));
    PBR_TRY(tmp.alloc(&vk2, sizeof(uint32_t) * n_sort));
    PBR_TRY(tmp.alloc(&vv2, sizeof(uint32_t) * n_sort));
    PBR_TRY(dalloc((void **)&st->tile_keys, sizeof(uint32_t) * n_pairs, s));
    PBR_TRY(dalloc((void **)&st->tile_vals, sizeof(uint32_t) * n_pairs, s));
    PBR_TRY(tmp.alloc(&pk2, sizeof(uint32_t) * n_pairs));
    PBR_TRY(tmp.alloc(&pv2, sizeof(uint32_t) * n_pairs));
    PBR_TRY(dalloc((void **)&st->ranges, sizeof(uint2) * L.n_tiles, s));
    PBR_TRY(dalloc((void **)&st->T_final, sizeof(float) * L.n_pix, s));
    PBR_TRY(dalloc((void **)&st->n_contrib, sizeof(uint32_t) * L.n_pix, s));
    PBR_TRY(tmp.alloc(&temp, temp_bytes));
    uint32_t *status = (uint32_t *)((char *)st->counters + 64);
    const uint32_t *n_vis_dev = (const uint32_t *)(st->counters + 1);  // low word (< 2^32)
    const uint32_t *n_pairs_dev = (const uint32_t *)(st->counters + 0); // low word (< 2^32)
    // 1. visible point-views with their depth keys, in point-view order
    if (!direct) {
        StageScope t(c, STG_COMPACT, s);
        launch_compact_visible(st->ntiles, zbits, npv, vk, vv, nullptr, temp, s);
    }
    // 2. stable sort by fp32 depth bits (ties keep point-view order)
    {
        StageScope t(c, STG_DEPTH_SORT, s);
        if (direct)
            radix_sort_pairs(zbits, vv, vk2, vv2, nullptr, npv, depth_bits, temp, s, zlo, marker,
                             true);
        else
            radix_sort_pairs(vk, vv, vk2, vv2, n_vis_dev, (int64_t)n_vis, depth_bits, temp, s,
                             zlo);
    }
    // 3. duplicate per covered tile, in depth order
    uint32_t *tk = st->tile_keys, *tv = st->tile_vals;
    {
        StageScope t(c, STG_EMIT, s);
        launch_emit_pairs(b, o, vv, n_vis_dev, (int64_t)n_vis, st->ntiles, nt8, rect, tk, tv,
                          (int64_t)n_pairs, status, temp, s);
    }
    // 4. stable sort by tile id
    {
        StageScope t(c, STG_TILE_SORT, s);
        radix_sort_pairs(tk, tv, pk2, pv2, n_pairs_dev, (int64_t)n_pairs,
                         key_bits_for(L.n_tiles), temp, s, 0, 0xffffffffu, false,
                         block_bits(o.tile_w, o.tile_h));
    }
    if (tk != st->tile_keys) { // result landed in the alternate buffers: swap ownership
        for (void *&p : tmp.ptrs) {
            if (p == (void *)tk) p = (void *)st->tile_keys;
            else if (p == (void *)tv) p = (void *)st->tile_vals;
        }
        st->tile_keys = tk;
        st->tile_vals = tv;
    }
    // 5. per-tile ranges
    {
        StageScope t(c, STG_RANGES, s);
        PBR_CUDA(cudaMemsetAsync(st->ranges, 0, sizeof(uint2) * L.n_tiles, s));
        launch_tile_ranges(st->tile_keys, n_pairs_dev, (int64_t)n_pairs, st->ranges, L.n_tiles,
                           block_bits(o.tile_w, o.tile_h), s);
    }
    // 6. composite (optionally as one persistent launch over a longest-first tile order)
    const bool persist = st->opts.persistent && st->batch_depth == 0;
    if (persist) {
        PBR_TRY(dalloc((void **)&st->tile_order, sizeof(uint4) * L.n_tiles, s));
        PBR_TRY(dalloc((void **)&st->work, 64 * sizeof(uint32_t), s));
    }
    if (st->store_depth > 0) {
        PBR_TRY(dalloc((void **)&st->T_store,
                       sizeof(float) * (size_t)st->store_depth * (size_t)L.n_pix, s));
        PBR_TRY(dalloc((void **)&st->n_comp, sizeof(uint32_t) * L.n_pix, s));
    }
    {
        StageScope t(c, STG_RASTER_FWD, s);
        if (persist) launch_tile_order(b, st->ranges, L.n_tiles, st->tile_order, st->work, s);
        launch_raster_fwd(b, o, st->batch_depth, st->ranges, st->tile_keys, st->tile_vals,
                          st->rec, out_rgb,
                          st->T_final, st->n_contrib,
                          st->opts.no_pair_stats ? nullptr : st->counters + 2, s, st->tile_order,
                          st->work, st->store());
    }
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

// The bytes forward_eager allocates (each allocation at least 16 bytes), all
// alive at its end: the state's buffers, the call's temporaries and, in store
// mode, the transmittance list.
size_t pbr::forward_bytes(const HostLayout &L, int64_t n_vis, int64_t n_pairs,
                          const pbr_render_opts *o, int32_t store_depth)
{
    auto al = [](size_t b) { return b ? b : (size_t)16; };
    const int64_t npv = L.n_pv;
    const bool direct = n_vis > 0 && 4 * n_vis >= 3 * npv;
    const int64_t n_sort = direct ? npv : n_vis;
    const int64_t cap_sort = std::max<int64_t>(n_sort, n_pairs);
    const size_t temp = std::max(std::max(scan_temp_bytes(npv), radix_temp_bytes(cap_sort)),
                                 emit_temp_bytes(n_vis));
    size_t b = al(sizeof(DevView) * L.views.size()) + al(sizeof(DevScene) * L.scenes.size()) +
               al(sizeof(int32_t) * L.view_list.size());
    b += al(32 * (size_t)npv) + al(4 * (size_t)npv) + 128;         // records, tile counts, counters
    b += al(4 * (size_t)npv) + al(16 * (size_t)npv) + al((size_t)npv); // depth bits, rectangles,
                                                                         // one-byte counts
    b += (direct ? 0 : al(4 * (size_t)n_sort)) + 3 * al(4 * (size_t)n_sort); // depth sort
    b += 4 * al(4 * (size_t)n_pairs);                              // pair lists, sort buffers
    b += al(8 * (size_t)L.n_tiles) + 2 * al(4 * (size_t)L.n_pix);  // ranges, T_final, n_contrib
    b += al(temp);
    if (o->persistent && o->batch_depth == 0) b += al(16 * (size_t)L.n_tiles) + 256;
    if (store_depth > 0)
        b += al(4 * (size_t)store_depth * (size_t)L.n_pix) + al(4 * (size_t)L.n_pix);
    return b;
}

extern "C" int pbr_forward_workspace_size(pbr_ctx *c, const pbr_points *scenes, int32_t n_scenes,
                                          const int32_t *scene_of_view, const pbr_camera *cams,
                                          int32_t n_cams, const pbr_render_opts *opts,
                                          int32_t keep_state, size_t *bytes, size_t *store_out,
                                          pbr_stream_t stream)
{
    if (!c || !bytes) return set_error(PBR_ERR_INVALID_ARG, "ctx or bytes is NULL");
    PBR_TRY(check_opts(opts));
    PBR_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    HostLayout L;
    PBR_TRY(build_layout(scenes, n_scenes, scene_of_view, cams, n_cams, opts, L));
    // the per-point stage, counting only: visible point-views and pairs
    TempBufs tmp(s);
    DevView *dv = nullptr;
    DevScene *ds = nullptr;
    int32_t *dl = nullptr;
    unsigned long long *counters = nullptr;
    PBR_TRY(tmp.alloc(&dv, sizeof(DevView) * L.views.size()));
    PBR_TRY(tmp.alloc(&ds, sizeof(DevScene) * L.scenes.size()));
    PBR_TRY(tmp.alloc(&dl, sizeof(int32_t) * L.view_list.size()));
    PBR_TRY(tmp.alloc(&counters, 128));
    PBR_CUDA(cudaMemcpyAsync(dv, L.views.data(), sizeof(DevView) * L.views.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(ds, L.scenes.data(), sizeof(DevScene) * L.scenes.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(dl, L.view_list.data(), sizeof(int32_t) * L.view_list.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemsetAsync(counters, 0, 128, s));
    PBR_CUDA(cudaMemsetAsync((char *)counters + 48, 0xff, 4, s));
    Batch b;
    b.views = dv;
    b.scenes = ds;
    b.view_list = dl;
    b.n_views = (int32_t)L.views.size();
    b.n_scenes = (int32_t)L.scenes.size();
    b.n_pv = L.n_pv;
    b.n_tiles = L.n_tiles;
    b.n_pix = L.n_pix;
    b.n_point_blocks = L.n_point_blocks;
    launch_preprocess_fwd(b, dev_opts(opts), nullptr, nullptr, nullptr, nullptr, nullptr, counters,
                          s);
    PBR_CUDA(cudaGetLastError());
    unsigned long long host[2] = {0, 0};
    PBR_CUDA(cudaMemcpyAsync(host, counters, sizeof host, cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    const int32_t depth = resolve_store_depth(c, opts, L.n_pix, keep_state != 0);
    *bytes = forward_bytes(L, (int64_t)host[1], (int64_t)host[0], opts, depth);
    if (store_out) *store_out = store_bytes(depth, L.n_pix);
    return PBR_OK;
}

extern "C" int pbr_render_forward(pbr_ctx *c, const pbr_points *scenes, int32_t n_scenes,
                                  const int32_t *scene_of_view, const pbr_camera *cams,
                                  int32_t n_cams, const pbr_render_opts *opts, float *out_rgb,
                                  pbr_state **state_out, pbr_stream_t stream)
{
    if (state_out) *state_out = nullptr;
    if (!c) return set_error(PBR_ERR_INVALID_ARG, "ctx is NULL");
    PBR_TRY(check_opts(opts));
    if (!out_rgb) return set_error(PBR_ERR_INVALID_ARG, "out_rgb is NULL");
    PBR_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    pbr_state *st = new pbr_state();
    st->stream = s;
    st->opts = *opts;
    st->dopts = dev_opts(opts);
    st->batch_depth = opts->batch_depth;
    int rc = build_layout(scenes, n_scenes, scene_of_view, cams, n_cams, opts, st->layout);
    st->store_depth = resolve_store_depth(c, opts, st->layout.n_pix, state_out != nullptr);
    if (rc == PBR_OK) rc = forward_eager(c, st, out_rgb, s);
    if (rc != PBR_OK || !state_out) {
        st->release();
        delete st;
        return rc;
    }
    *state_out = st;
    return PBR_OK;
}

void pbr::zero_unviewed_grads(const HostLayout &L, float *grad_pos, float *grad_sh,
                              float *grad_opacity, cudaStream_t s)
{
    for (const DevScene &d : L.scenes) {
        if (d.view_count > 0 || d.n == 0) continue;
        cudaMemsetAsync(grad_pos + 3 * d.point_base, 0, sizeof(float) * 3 * (size_t)d.n, s);
        cudaMemsetAsync(grad_sh + d.sh_base, 0, sizeof(float) * 3 * (size_t)d.K * d.n, s);
        if (grad_opacity)
            cudaMemsetAsync(grad_opacity + d.point_base, 0, sizeof(float) * (size_t)d.n, s);
    }
}

extern "C" int pbr_render_backward(pbr_ctx *c, pbr_state *st, const float *grad_rgb,
                                   float *grad_pos, float *grad_sh, float *grad_opacity,
                                   pbr_stream_t stream)
{
    if (!c || !st) return set_error(PBR_ERR_INVALID_ARG, "ctx or state is NULL");
    if (!grad_rgb || !grad_pos || !grad_sh)
        return set_error(PBR_ERR_INVALID_ARG, "grad_rgb, grad_pos and grad_sh are required");
    PBR_CUDA(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const HostLayout &L = st->layout;
    Batch b = st->batch();
    float4 *g2d = nullptr;
    PBR_TRY(dalloc((void **)&g2d, sizeof(float4) * 2 * L.n_pv, s));
    {
        StageScope t(c, STG_RASTER_BWD, s);
        PBR_CUDA(cudaMemsetAsync(g2d, 0, sizeof(float4) * 2 * L.n_pv, s));
        if (st->work) reset_work_counters(st->work, s);
        launch_raster_bwd(b, st->dopts, st->batch_depth, st->ranges, st->tile_keys,
                          st->tile_vals, st->rec,
                          st->T_final, st->n_contrib, grad_rgb, g2d,
                          st->opts.no_pair_stats ? nullptr : st->counters + 2, s,
                          st->tile_order, st->work, st->store());
    }
    {
        StageScope t(c, STG_PREPROCESS_BWD, s);
        launch_preprocess_bwd(b, st->dopts, g2d, grad_pos, grad_sh, grad_opacity, s);
        zero_unviewed_grads(L, grad_pos, grad_sh, grad_opacity, s);
    }
    cudaError_t e = cudaGetLastError();
    dfree(g2d, s);
    if (e != cudaSuccess)
        return set_error(PBR_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
    return PBR_OK;
}

extern "C" int pbr_state_free(pbr_ctx *c, pbr_state *st)
{
    (void)c;
    if (!st) return PBR_OK;
    st->release();
    delete st;
    return PBR_OK;
}

extern "C" int pbr_state_info(pbr_state *st, pbr_state_info_t *info)
{
    if (!st || !info) return set_error(PBR_ERR_INVALID_ARG, "state or info is NULL");
    PBR_CUDA(cudaStreamSynchronize(st->stream));
    uint32_t status = 0;
    PBR_CUDA(cudaMemcpy(&status, (char *)st->counters + 64, 4, cudaMemcpyDeviceToHost));
    std::memset(info, 0, sizeof *info);
    info->n_point_views = st->layout.n_pv;
    info->n_visible = st->n_vis;
    info->n_pairs = st->n_pairs;
    info->n_tiles = st->layout.n_tiles;
    info->n_pixels = st->layout.n_pix;
    info->tile_keys = st->tile_keys;
    info->tile_vals = st->tile_vals;
    info->ranges = (const uint32_t *)st->ranges;
    info->records = (const float *)st->rec;
    info->ntiles = st->ntiles;
    info->T_final = st->T_final;
    info->n_contrib = st->n_contrib;
    if (status) return set_error(PBR_ERR_DEVICE_STATUS, "device status 0x%x", status);
    return PBR_OK;
}

extern "C" int pbr_state_read(pbr_state *st, int32_t which, void *host_dst, size_t cap_bytes,
                              size_t *size_bytes)
{
    if (!st) return set_error(PBR_ERR_INVALID_ARG, "state is NULL");
    const void *src = nullptr;
    size_t n = 0;
    const HostLayout &L = st->layout;
    switch (which) {
    case 0: src = st->tile_keys; n = 4 * (size_t)st->n_pairs; break;
    case 1: src = st->tile_vals; n = 4 * (size_t)st->n_pairs; break;
    case 2: src = st->ranges; n = 8 * (size_t)L.n_tiles; break;
    case 3: src = st->rec; n = 32 * (size_t)L.n_pv; break;
    case 4: src = st->ntiles; n = 4 * (size_t)L.n_pv; break;
    case 5: src = st->T_final; n = 4 * (size_t)L.n_pix; break;
    case 6: src = st->n_contrib; n = 4 * (size_t)L.n_pix; break;
    case 7: src = st->T_store; n = 4 * (size_t)st->store_depth * (size_t)L.n_pix; break;
    case 8: src = st->n_comp; n = st->n_comp ? 4 * (size_t)L.n_pix : 0; break;
    default: return set_error(PBR_ERR_INVALID_ARG, "pbr_state_read: unknown array %d", which);
    }
    if (size_bytes) *size_bytes = n;
    PBR_CUDA(cudaStreamSynchronize(st->stream));
    const size_t m = n < cap_bytes ? n : cap_bytes;
    if (m && host_dst && src) PBR_CUDA(cudaMemcpy(host_dst, src, m, cudaMemcpyDeviceToHost));
    return PBR_OK;
}

extern "C" int pbr_state_stats(pbr_state *st, unsigned long long *out4)
{
    if (!st || !out4) return set_error(PBR_ERR_INVALID_ARG, "state or out is NULL");
    PBR_CUDA(cudaStreamSynchronize(st->stream));
    PBR_CUDA(cudaMemcpy(out4, st->counters + 2, 4 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost));
    return PBR_OK;
}

extern "C" int pbr_image_loss(int32_t kind, const float *pred, const float *target, int64_t n,
                              float *grad, double *loss_dev, pbr_stream_t stream)
{
    if ((kind != 0 && kind != 1) || n < 0 || (n > 0 && (!pred || !target || !grad || !loss_dev)))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_image_loss: bad arguments");
    launch_image_loss(kind, pred, target, n, grad, loss_dev, (cudaStream_t)stream);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" void pbr_default_optimizer(pbr_optimizer_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->kind = 1;
    c->lr_pos = 8e-4f;
    c->lr_sh = 3e-3f;
    c->lr_opacity = 0.0f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->lambda_tv = 0.01f;
    c->loss_kind = 0;
}

extern "C" int pbr_image_loss_tv(const pbr_camera *cams, int32_t n_cams, const float *pred,
                                 const float *target, int32_t loss_kind, float lambda_tv,
                                 float *grad, double *loss_dev, pbr_stream_t stream)
{
    if (!cams || n_cams <= 0 || !pred || !target || !grad || !loss_dev ||
        (loss_kind != 0 && loss_kind != 1) || !(lambda_tv >= 0.f))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_image_loss_tv: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<DevView> views(n_cams);
    int64_t pix = 0, max_pix = 0;
    for (int v = 0; v < n_cams; ++v) {
        if (cams[v].width <= 0 || cams[v].height <= 0)
            return set_error(PBR_ERR_INVALID_ARG, "camera %d: size", v);
        std::memset(&views[v], 0, sizeof(DevView));
        views[v].W = cams[v].width;
        views[v].H = cams[v].height;
        views[v].pix_base = pix;
        const int64_t np = (int64_t)cams[v].width * cams[v].height;
        pix += np;
        max_pix = std::max(max_pix, np);
    }
    TempBufs tmp(s);
    DevView *d = nullptr;
    PBR_TRY(tmp.alloc(&d, sizeof(DevView) * n_cams));
    PBR_CUDA(cudaMemcpyAsync(d, views.data(), sizeof(DevView) * n_cams, cudaMemcpyHostToDevice, s));
    launch_loss_tv(d, n_cams, max_pix, loss_kind, lambda_tv, pred, target, grad, loss_dev, s);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_optimizer_step(int32_t kind, float *param, const float *grad, float *m,
                                  float *v, int64_t n, float lr, float beta1, float beta2,
                                  float eps, int32_t step, pbr_stream_t stream)
{
    if ((kind != 0 && kind != 1) || n < 0 || (n > 0 && (!param || !grad)) ||
        (kind == 1 && n > 0 && (!m || !v || step < 1)))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_optimizer_step: bad arguments");
    OptParams prm{kind, lr, beta1, beta2, eps, step};
    launch_optimizer(prm, nullptr, 0, param, grad, m, v, n, (cudaStream_t)stream);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_measure_alu_peaks(int device, double *fp32_flops, double *ex2_ops)
{
    if (measure_alu_peaks(device, fp32_flops, ex2_ops) != 0)
        return set_error(PBR_ERR_CUDA, "microbenchmark failed");
    return PBR_OK;
}
