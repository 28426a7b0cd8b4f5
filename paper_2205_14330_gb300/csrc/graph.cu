// Batched rendering as CUDA graphs, and the schedule autotuner.
//
// pbr_graph_create plans one batch of views (possibly of several scenes or
// frames): an eager forward pass measures the visible point-views, the
// number of (tile, point-view) pairs and the depth range; buffers are then
// allocated once with headroom and the whole chain -- per-point stage, both
// sorts, emission, ranges, compositing, optionally the image loss and the
// backward pass -- is captured into CUDA graphs.  Nothing inside a replay
// synchronises with the host: every kernel reads its element counts from
// device memory and grids are sized by capacity.  A replay that outgrows a
// capacity (more pairs than planned, depths outside the planned key range)
// raises a bit in the device status word; pbr_graph_check reports it and
// pbr_graph_replan re-plans and re-captures.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "api_internal.h"

using namespace pbr;

namespace {

constexpr uint32_t ST_DEPTH_RANGE = 1u << 3;

// Raises ST_DEPTH_RANGE when a visible depth falls outside the planned key
// range [lo, lo + span).
__global__ void check_depth_range_kernel(const unsigned long long *counters, uint32_t lo,
                                         uint64_t span, uint32_t *status)
{
    const uint32_t *w = (const uint32_t *)counters;
    if (counters[1] == 0) return;
    const uint32_t zmin = w[12], zmax = w[13];
    if (zmin < lo || (uint64_t)(zmax - lo) >= span) atomicOr(status, ST_DEPTH_RANGE);
}

float bits_to_float(uint32_t b)
{
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

uint32_t float_to_bits(float f)
{
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

int bit_width(uint32_t x)
{
    int b = 0;
    while (b < 32 && (x >> b)) ++b;
    return b;
}

} // namespace

struct pbr_graph {
    pbr_ctx *ctx = nullptr;
    // creation parameters (kept for re-planning)
    std::vector<pbr_points> scenes;
    std::vector<int32_t> sov;
    std::vector<pbr_camera> cams;
    pbr_render_opts opts{};
    float *out_rgb = nullptr;
    const float *target = nullptr;
    int32_t loss_kind = 0;
    double *loss_out = nullptr;
    const float *grad_rgb = nullptr;
    float *grad_pos = nullptr, *grad_sh = nullptr, *grad_opacity = nullptr;
    double headroom = 0.25;
    // plan
    DevOpts dopts{};
    HostLayout layout;
    int64_t cap_vis = 0, cap_pairs = 0;
    uint32_t depth_lo = 0;
    int depth_bits = 32;
    // all point-views sorted by depth, the invisible ones behind (key clamped
    // to depth_marker), instead of compacting the visible ones first
    bool direct_depth = false;
    uint32_t depth_marker = 0xffffffffu;
    // buffers (cudaMalloc, stable addresses for the graphs)
    std::vector<void *> allocs;
    DevView *d_views = nullptr;
    DevScene *d_scenes = nullptr;
    int32_t *d_view_list = nullptr;
    float4 *rec = nullptr, *g2d = nullptr;
    uint32_t *ntiles = nullptr, *zbits = nullptr;
    uint8_t *nt8 = nullptr;
    uint4 *rect = nullptr;
    uint2 *ranges = nullptr;
    unsigned long long *counters = nullptr;
    uint32_t *vk = nullptr, *vv = nullptr, *vk2 = nullptr, *vv2 = nullptr;
    uint32_t *tk = nullptr, *tv = nullptr, *tk2 = nullptr, *tv2 = nullptr;
    float *T_final = nullptr;
    uint32_t *n_contrib = nullptr, *work = nullptr;
    uint4 *order = nullptr; // persistent raster: tile descriptors, longest list first
    void *temp = nullptr;
    float *own_grad = nullptr;
    double *own_loss = nullptr;
    uint32_t *keys_final = nullptr, *vals_final = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr}; // fwd, bwd, step, train
    int kernels[4] = {0, 0, 0, 0};
    // training phase: optimiser settings, device rates / step, moments
    bool has_opt = false;
    pbr_optimizer_cfg opt{};
    std::vector<void *> opt_allocs; // survive re-planning
    OptState *d_opt = nullptr;
    float *m_pos = nullptr, *v_pos = nullptr, *m_sh = nullptr, *v_sh = nullptr;
    float *m_op = nullptr, *v_op = nullptr;
    unsigned long long *host = nullptr; // pinned status read-back

    Batch batch() const
    {
        Batch b;
        b.views = d_views;
        b.scenes = d_scenes;
        b.view_list = d_view_list;
        b.n_views = (int32_t)layout.views.size();
        b.n_scenes = (int32_t)layout.scenes.size();
        b.n_pv = layout.n_pv;
        b.n_tiles = layout.n_tiles;
        b.n_pix = layout.n_pix;
        b.n_point_blocks = layout.n_point_blocks;
        return b;
    }
    template <class T> int alloc(T **p, size_t bytes)
    {
        *p = nullptr;
        const cudaError_t e = cudaMalloc((void **)p, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(PBR_ERR_OOM, "graph buffer of %zu bytes: %s", bytes,
                             cudaGetErrorString(e));
        }
        allocs.push_back((void *)*p);
        return PBR_OK;
    }
    void release()
    {
        for (auto &e : exec)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
    }
};

namespace {

// The forward chain on planned capacities.  Pointer ping-pong of the sorts
// happens at capture time; the final pair-list buffers are recorded.
void enqueue_forward(pbr_graph *g, cudaStream_t s)
{
    const Batch b = g->batch();
    const DevOpts &o = g->dopts;
    const HostLayout &L = g->layout;
    uint32_t *status = (uint32_t *)((char *)g->counters + 64);
    const uint32_t *n_vis_dev = (const uint32_t *)(g->counters + 1);
    const uint32_t *n_pairs_dev = (const uint32_t *)(g->counters + 0);
    cudaMemsetAsync(g->counters, 0, 128, s);
    cudaMemsetAsync((char *)g->counters + 48, 0xff, 4, s);
    launch_preprocess_fwd(b, o, g->rec, g->zbits, g->ntiles, g->nt8, g->rect, g->counters, s);
    // visible keys must lie below the marker (direct) or inside the bits
    const uint64_t span = g->direct_depth ? (uint64_t)g->depth_marker
                          : g->depth_bits >= 32 ? (1ull << 32) : (1ull << g->depth_bits);
    check_depth_range_kernel<<<1, 1, 0, s>>>(g->counters, g->depth_lo, span, status);
    count_launches(1);
    uint32_t *vk = g->vk, *vv = g->vv, *vk2 = g->vk2, *vv2 = g->vv2;
    if (g->direct_depth) {
        vk = g->zbits;
        radix_sort_pairs(vk, vv, vk2, vv2, nullptr, L.n_pv, g->depth_bits, g->temp, s,
                         g->depth_lo, g->depth_marker, true);
    } else {
        launch_compact_visible(g->ntiles, g->zbits, L.n_pv, g->vk, g->vv, nullptr, g->temp, s);
        radix_sort_pairs(vk, vv, vk2, vv2, n_vis_dev, g->cap_vis, g->depth_bits, g->temp, s,
                         g->depth_lo);
    }
    uint32_t *tk = g->tk, *tv = g->tv, *tk2 = g->tk2, *tv2 = g->tv2;
    launch_emit_pairs(b, o, vv, n_vis_dev, g->cap_vis, g->ntiles, g->nt8, g->rect, tk, tv,
                      g->cap_pairs, status, g->temp, s);
    int key_bits = bit_width(L.n_tiles > 0 ? L.n_tiles - 1 : 0);
    if (key_bits < 1) key_bits = 1;
    const int sb = block_bits(o.tile_w, o.tile_h);
    radix_sort_pairs(tk, tv, tk2, tv2, n_pairs_dev, g->cap_pairs, key_bits, g->temp, s, 0,
                     0xffffffffu, false, sb);
    g->keys_final = tk;
    g->vals_final = tv;
    cudaMemsetAsync(g->ranges, 0, sizeof(uint2) * L.n_tiles, s);
    launch_tile_ranges(tk, n_pairs_dev, g->cap_pairs, g->ranges, L.n_tiles, sb, s);
    const bool persist = g->opts.persistent && g->opts.batch_depth == 0;
    if (persist) launch_tile_order(b, g->ranges, L.n_tiles, g->order, g->work, s);
    launch_raster_fwd(b, o, g->opts.batch_depth, g->ranges, tk, tv, g->rec, g->out_rgb, g->T_final,
                      g->n_contrib, nullptr, s, persist ? g->order : nullptr, g->work);
}

void enqueue_backward(pbr_graph *g, const float *grad_rgb, cudaStream_t s)
{
    const Batch b = g->batch();
    const HostLayout &L = g->layout;
    cudaMemsetAsync(g->g2d, 0, sizeof(float4) * 2 * L.n_pv, s);
    const bool persist = g->opts.persistent && g->opts.batch_depth == 0;
    if (persist) reset_work_counters(g->work, s);
    launch_raster_bwd(b, g->dopts, g->opts.batch_depth, g->ranges, g->keys_final, g->vals_final,
                      g->rec,
                      g->T_final, g->n_contrib, grad_rgb, g->g2d, nullptr, s,
                      persist ? g->order : nullptr, g->work);
    launch_preprocess_bwd(b, g->dopts, g->g2d, g->grad_pos, g->grad_sh, g->grad_opacity, s);
    zero_unviewed_grads(L, g->grad_pos, g->grad_sh, g->grad_opacity, s);
}

// Optimiser update of every scene's parameters from the packed gradients.
void enqueue_optimizer(pbr_graph *g, cudaStream_t s)
{
    launch_step_counter(g->d_opt, s);
    const OptParams prm{g->opt.kind, 0.0f, g->opt.beta1, g->opt.beta2, g->opt.eps, 1};
    for (const DevScene &sc : g->layout.scenes) {
        const int64_t n = sc.n;
        launch_optimizer(prm, g->d_opt, 0, const_cast<float *>(sc.pos), g->grad_pos + 3 * sc.point_base,
                         g->m_pos + 3 * sc.point_base, g->v_pos + 3 * sc.point_base, 3 * n, s);
        launch_optimizer(prm, g->d_opt, 1, const_cast<float *>(sc.sh), g->grad_sh + sc.sh_base,
                         g->m_sh + sc.sh_base, g->v_sh + sc.sh_base, n * sc.K * 3, s);
        if (g->grad_opacity)
            launch_optimizer(prm, g->d_opt, 2, const_cast<float *>(sc.opacity),
                             g->grad_opacity + sc.point_base, g->m_op + sc.point_base,
                             g->v_op + sc.point_base, n, s);
    }
}

int capture(pbr_graph *g, int which, cudaStream_t s)
{
    cudaGraph_t graph = nullptr;
    const unsigned long long l0 = launches_total();
    PBR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const float *grad = g->grad_rgb ? g->grad_rgb : g->own_grad;
    if (which == 0 || which == 2 || which == 3) enqueue_forward(g, s);
    double *loss = g->loss_out ? g->loss_out : g->own_loss;
    if (which == 2) {
        cudaMemsetAsync(loss, 0, sizeof(double), s);
        launch_image_loss(g->loss_kind, g->out_rgb, g->target, g->layout.n_pix * 3, g->own_grad,
                          loss, s);
        grad = g->own_grad;
    }
    if (which == 3) {
        int64_t max_pix = 0;
        for (const DevView &v : g->layout.views) max_pix = std::max<int64_t>(max_pix, (int64_t)v.W * v.H);
        cudaMemsetAsync(loss, 0, sizeof(double), s);
        launch_loss_tv(g->d_views, (int)g->layout.views.size(), max_pix, g->opt.loss_kind,
                       g->opt.lambda_tv, g->out_rgb, g->target, g->own_grad, loss, s);
        grad = g->own_grad;
    }
    if (which == 1 || which == 2 || which == 3) enqueue_backward(g, grad, s);
    if (which == 3) enqueue_optimizer(g, s);
    const cudaError_t e1 = cudaStreamEndCapture(s, &graph);
    const unsigned long long l1 = launches_total();
    if (e1 != cudaSuccess) {
        cudaGetLastError();
        return set_error(PBR_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e1));
    }
    const cudaError_t e2 = cudaGraphInstantiate(&g->exec[which], graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
        cudaGetLastError();
        return set_error(PBR_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e2));
    }
    g->kernels[which] = (int)(l1 - l0);
    // the captured launches ran no kernel yet: do not count them twice
    count_launches(-(int)(l1 - l0));
    return PBR_OK;
}

int plan_and_capture(pbr_graph *g, cudaStream_t user_stream)
{
    pbr_ctx *c = g->ctx;
    g->release();
    PBR_TRY(check_opts(&g->opts));
    g->dopts = dev_opts(&g->opts);
    g->layout = HostLayout();
    PBR_TRY(build_layout(g->scenes.data(), (int32_t)g->scenes.size(),
                         g->sov.empty() ? nullptr : g->sov.data(), g->cams.data(),
                         (int32_t)g->cams.size(), &g->opts, g->layout));
    const HostLayout &L = g->layout;
    // 1. planning pass (eager, exact sizes)
    {
        pbr_state st;
        st.stream = user_stream;
        st.opts = g->opts;
        st.dopts = g->dopts;
        st.batch_depth = g->opts.batch_depth;
        st.layout = L;
        const int rc = forward_eager(c, &st, g->out_rgb, user_stream);
        if (rc == PBR_OK) {
            PBR_CUDA(cudaMemcpyAsync(g->host, st.counters, 64, cudaMemcpyDeviceToHost, user_stream));
        }
        st.release();
        PBR_CUDA(cudaStreamSynchronize(user_stream));
        if (rc != PBR_OK) return rc;
    }
    const uint64_t n_pairs = g->host[0], n_vis = g->host[1];
    const uint32_t zlo = ((uint32_t *)g->host)[12], zhi = ((uint32_t *)g->host)[13];
    g->cap_vis = L.n_pv;
    g->cap_pairs = (int64_t)std::ceil((double)n_pairs * (1.0 + g->headroom)) + 4096;
    if (g->cap_pairs >= (int64_t)UINT32_MAX) g->cap_pairs = (int64_t)UINT32_MAX - 1;
    g->direct_depth = n_vis > 0 && 4 * n_vis >= 3 * (uint64_t)L.n_pv;
    if (n_vis > 0 && zhi >= zlo) {
        // key range with a factor-2 margin in depth on both sides
        const uint32_t lo = float_to_bits(bits_to_float(zlo) * 0.5f);
        const uint32_t hi = float_to_bits(std::min(bits_to_float(zhi) * 2.0f, 3.0e38f));
        g->depth_lo = lo;
        // direct sort: one key value above the range is the invisible marker
        g->depth_bits = bit_width(g->direct_depth ? hi - lo + 1 : hi - lo);
    } else {
        g->depth_lo = 0;
        g->depth_bits = 32;
    }
    if (g->direct_depth)
        g->depth_marker = g->depth_bits >= 32 ? 0xffffffffu : (1u << g->depth_bits) - 1u;
    // 2. buffers
    const int64_t npv = L.n_pv;
    PBR_TRY(g->alloc(&g->d_views, sizeof(DevView) * L.views.size()));
    PBR_TRY(g->alloc(&g->d_scenes, sizeof(DevScene) * L.scenes.size()));
    PBR_TRY(g->alloc(&g->d_view_list, sizeof(int32_t) * L.view_list.size()));
    PBR_TRY(g->alloc(&g->counters, 128));
    PBR_TRY(g->alloc(&g->rec, sizeof(float4) * 2 * npv));
    PBR_TRY(g->alloc(&g->ntiles, sizeof(uint32_t) * npv));
    PBR_TRY(g->alloc(&g->zbits, sizeof(uint32_t) * npv));
    PBR_TRY(g->alloc(&g->rect, sizeof(uint4) * npv));
    PBR_TRY(g->alloc(&g->nt8, (size_t)npv));
    if (!g->direct_depth) PBR_TRY(g->alloc(&g->vk, 4 * (size_t)g->cap_vis));
    PBR_TRY(g->alloc(&g->vv, 4 * (size_t)g->cap_vis));
    PBR_TRY(g->alloc(&g->vk2, 4 * (size_t)g->cap_vis));
    PBR_TRY(g->alloc(&g->vv2, 4 * (size_t)g->cap_vis));
    PBR_TRY(g->alloc(&g->tk, 4 * (size_t)g->cap_pairs));
    PBR_TRY(g->alloc(&g->tv, 4 * (size_t)g->cap_pairs));
    PBR_TRY(g->alloc(&g->tk2, 4 * (size_t)g->cap_pairs));
    PBR_TRY(g->alloc(&g->tv2, 4 * (size_t)g->cap_pairs));
    PBR_TRY(g->alloc(&g->ranges, sizeof(uint2) * L.n_tiles));
    PBR_TRY(g->alloc(&g->T_final, sizeof(float) * L.n_pix));
    PBR_TRY(g->alloc(&g->n_contrib, sizeof(uint32_t) * L.n_pix));
    PBR_TRY(g->alloc(&g->order, sizeof(uint4) * (L.n_tiles ? L.n_tiles : 1)));
    PBR_TRY(g->alloc(&g->work, 64 * sizeof(uint32_t)));
    const size_t temp = std::max(std::max(scan_temp_bytes(npv),
                                          radix_temp_bytes(std::max(g->cap_vis, g->cap_pairs))),
                                 emit_temp_bytes(g->cap_vis));
    PBR_TRY(g->alloc(&g->temp, temp));
    const bool want_bwd = g->grad_pos && g->grad_sh;
    if (want_bwd) PBR_TRY(g->alloc(&g->g2d, sizeof(float4) * 2 * npv));
    if (want_bwd && g->target) {
        PBR_TRY(g->alloc(&g->own_grad, sizeof(float) * 3 * L.n_pix));
        PBR_TRY(g->alloc(&g->own_loss, sizeof(double)));
    }
    PBR_CUDA(cudaMemcpy(g->d_views, L.views.data(), sizeof(DevView) * L.views.size(),
                        cudaMemcpyHostToDevice));
    PBR_CUDA(cudaMemcpy(g->d_scenes, L.scenes.data(), sizeof(DevScene) * L.scenes.size(),
                        cudaMemcpyHostToDevice));
    PBR_CUDA(cudaMemcpy(g->d_view_list, L.view_list.data(), sizeof(int32_t) * L.view_list.size(),
                        cudaMemcpyHostToDevice));
    // 3. capture: forward, backward (from the caller's dL/dimage), training step
    PBR_TRY(capture(g, 0, g->cap_stream));
    if (want_bwd && (g->grad_rgb || g->target)) PBR_TRY(capture(g, 1, g->cap_stream));
    if (want_bwd && g->target) PBR_TRY(capture(g, 2, g->cap_stream));
    if (want_bwd && g->target && g->has_opt) PBR_TRY(capture(g, 3, g->cap_stream));
    return PBR_OK;
}

} // namespace

extern "C" int pbr_graph_create(pbr_ctx *c, const pbr_points *scenes, int32_t n_scenes,
                                const int32_t *scene_of_view, const pbr_camera *cams,
                                int32_t n_cams, const pbr_render_opts *opts, float *out_rgb,
                                const float *target, int32_t loss_kind, double *loss_out,
                                const float *grad_rgb, float *grad_pos, float *grad_sh,
                                float *grad_opacity, double headroom, pbr_stream_t stream,
                                pbr_graph **out)
{
    if (!out) return set_error(PBR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!c || !scenes || n_scenes <= 0 || !cams || n_cams <= 0 || !opts || !out_rgb)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_graph_create: missing argument");
    if (loss_kind != 0 && loss_kind != 1)
        return set_error(PBR_ERR_INVALID_ARG, "loss_kind must be 0 (L2) or 1 (L1)");
    if (!(headroom >= 0.0 && headroom <= 10.0))
        return set_error(PBR_ERR_INVALID_ARG, "headroom must be in [0, 10]");
    PBR_CUDA(cudaSetDevice(c->device));
    pbr_graph *g = new pbr_graph();
    g->ctx = c;
    g->scenes.assign(scenes, scenes + n_scenes);
    if (scene_of_view) g->sov.assign(scene_of_view, scene_of_view + n_cams);
    g->cams.assign(cams, cams + n_cams);
    g->opts = *opts;
    g->out_rgb = out_rgb;
    g->target = target;
    g->loss_kind = loss_kind;
    g->loss_out = loss_out;
    g->grad_rgb = grad_rgb;
    g->grad_pos = grad_pos;
    g->grad_sh = grad_sh;
    g->grad_opacity = grad_opacity;
    g->headroom = headroom;
    if (cudaMallocHost(&g->host, 128) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (g->host) cudaFreeHost(g->host);
        delete g;
        return set_error(PBR_ERR_CUDA, "graph set-up failed");
    }
    const int rc = plan_and_capture(g, (cudaStream_t)stream);
    if (rc != PBR_OK) {
        g->release();
        cudaStreamDestroy(g->cap_stream);
        cudaFreeHost(g->host);
        delete g;
        return rc;
    }
    *out = g;
    return PBR_OK;
}

extern "C" int pbr_graph_set_optimizer(pbr_graph *g, const pbr_optimizer_cfg *cfg,
                                       pbr_stream_t stream)
{
    if (!g || !cfg || (cfg->kind != 0 && cfg->kind != 1) || (cfg->loss_kind != 0 && cfg->loss_kind != 1))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_graph_set_optimizer: bad arguments");
    if (!g->target || !g->grad_pos || !g->grad_sh)
        return set_error(PBR_ERR_INVALID_ARG,
                         "the training phase needs a graph created with a target and gradients");
    PBR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (void *p : g->opt_allocs) cudaFree(p);
    g->opt_allocs.clear();
    const int64_t np = g->layout.n_points_total, nsh = g->layout.n_sh_total;
    auto al = [&](float **p, int64_t n) -> int {
        if (cudaMalloc((void **)p, sizeof(float) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(PBR_ERR_OOM, "optimiser state");
        }
        g->opt_allocs.push_back(*p);
        cudaMemset(*p, 0, sizeof(float) * (size_t)(n > 0 ? n : 1));
        return PBR_OK;
    };
    PBR_TRY(al(&g->m_pos, 3 * np));
    PBR_TRY(al(&g->v_pos, 3 * np));
    PBR_TRY(al(&g->m_sh, nsh));
    PBR_TRY(al(&g->v_sh, nsh));
    PBR_TRY(al(&g->m_op, np));
    PBR_TRY(al(&g->v_op, np));
    if (cudaMalloc((void **)&g->d_opt, sizeof(OptState)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(PBR_ERR_OOM, "optimiser state");
    }
    g->opt_allocs.push_back(g->d_opt);
    OptState st{{cfg->lr_pos, cfg->lr_sh, cfg->lr_opacity}, 0};
    PBR_CUDA(cudaMemcpy(g->d_opt, &st, sizeof st, cudaMemcpyHostToDevice));
    g->opt = *cfg;
    g->has_opt = true;
    if (g->exec[3]) {
        cudaGraphExecDestroy(g->exec[3]);
        g->exec[3] = nullptr;
    }
    return capture(g, 3, g->cap_stream);
}

extern "C" int pbr_graph_set_lr(pbr_graph *g, float lr_pos, float lr_sh, float lr_opacity)
{
    if (!g || !g->d_opt) return set_error(PBR_ERR_INVALID_ARG, "no optimiser on this graph");
    const float lr[3] = {lr_pos, lr_sh, lr_opacity};
    PBR_CUDA(cudaMemcpy(g->d_opt, lr, sizeof lr, cudaMemcpyHostToDevice));
    return PBR_OK;
}

extern "C" int pbr_graph_launch(pbr_graph *g, int32_t phase, pbr_stream_t stream)
{
    if (!g || phase < 0 || phase > 3) return set_error(PBR_ERR_INVALID_ARG, "bad graph or phase");
    if (!g->exec[phase])
        return set_error(PBR_ERR_INVALID_ARG, "graph phase %d was not captured (backward needs "
                                              "gradient buffers, the step needs a target)", phase);
    PBR_CUDA(cudaGraphLaunch(g->exec[phase], (cudaStream_t)stream));
    count_launches(g->kernels[phase]);
    return PBR_OK;
}

extern "C" int pbr_graph_check(pbr_graph *g, pbr_stream_t stream, int64_t *n_pairs,
                               int64_t *cap_pairs)
{
    if (!g) return set_error(PBR_ERR_INVALID_ARG, "graph is NULL");
    PBR_CUDA(cudaMemcpyAsync(g->host, g->counters, 128, cudaMemcpyDeviceToHost,
                             (cudaStream_t)stream));
    PBR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (n_pairs) *n_pairs = (int64_t)g->host[0];
    if (cap_pairs) *cap_pairs = g->cap_pairs;
    const uint32_t status = ((uint32_t *)g->host)[16];
    if (status)
        return set_error(PBR_ERR_CAPACITY,
                         "graph replay outgrew its plan (status 0x%x: %llu pairs, capacity %lld); "
                         "call pbr_graph_replan", status, (unsigned long long)g->host[0],
                         (long long)g->cap_pairs);
    return PBR_OK;
}

extern "C" int pbr_graph_replan(pbr_graph *g, pbr_stream_t stream)
{
    if (!g) return set_error(PBR_ERR_INVALID_ARG, "graph is NULL");
    PBR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return plan_and_capture(g, (cudaStream_t)stream);
}

extern "C" int pbr_graph_set_cameras(pbr_graph *g, const pbr_camera *cams, int32_t n_cams,
                                     pbr_stream_t stream)
{
    if (!g || !cams || n_cams != (int32_t)g->cams.size())
        return set_error(PBR_ERR_INVALID_ARG, "camera count must match the graph's");
    for (int v = 0; v < n_cams; ++v)
        if (cams[v].width != g->cams[v].width || cams[v].height != g->cams[v].height)
            return set_error(PBR_ERR_INVALID_ARG, "camera %d: image size differs from the plan", v);
    for (int v = 0; v < n_cams; ++v) {
        g->cams[v] = cams[v];
        DevView &d = g->layout.views[v];
        d.fx = cams[v].fx;
        d.fy = cams[v].fy;
        d.cx = cams[v].cx;
        d.cy = cams[v].cy;
        std::memcpy(d.R, cams[v].R, sizeof d.R);
        std::memcpy(d.t, cams[v].t, sizeof d.t);
    }
    PBR_CUDA(cudaMemcpyAsync(g->d_views, g->layout.views.data(),
                             sizeof(DevView) * g->layout.views.size(), cudaMemcpyHostToDevice,
                             (cudaStream_t)stream));
    PBR_CUDA(cudaStreamSynchronize((cudaStream_t)stream)); // host copy must outlive the transfer
    return PBR_OK;
}

extern "C" int pbr_graph_destroy(pbr_graph *g)
{
    if (!g) return PBR_OK;
    cudaDeviceSynchronize();
    g->release();
    for (void *p : g->opt_allocs) cudaFree(p);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->host) cudaFreeHost(g->host);
    delete g;
    return PBR_OK;
}

// ------------------------------------------------------------ autotuner
// Candidate schedules: tile size x {warp-streamed, persistent warp-streamed,
// block-staged with 128 / 256 / 512 points per batch}.  Each candidate runs
// the eager forward (and backward, mode 1) `reps` times after one warm-up;
// the fastest is written into *opts and cached in the context under the
// batch's shape class.
extern "C" int pbr_autotune(pbr_ctx *c, const pbr_points *scenes, int32_t n_scenes,
                            const int32_t *scene_of_view, const pbr_camera *cams, int32_t n_cams,
                            pbr_render_opts *opts, int32_t mode, int32_t reps, double *ms_out,
                            int32_t *n_candidates, pbr_stream_t stream)
{
    if (!c || !opts || reps < 1) return set_error(PBR_ERR_INVALID_ARG, "pbr_autotune: bad args");
    PBR_TRY(check_opts(opts));
    HostLayout L;
    PBR_TRY(build_layout(scenes, n_scenes, scene_of_view, cams, n_cams, opts, L));
    // shape class: views, log2 pixels, log2 point-views, degrees
    int64_t key_deg = 0;
    for (int s = 0; s < n_scenes; ++s) key_deg = key_deg * 4 + scenes[s].sh_degree;
    const auto key = std::make_tuple((int64_t)n_cams, (int64_t)std::log2((double)L.n_pix + 1),
                                     (int64_t)std::log2((double)L.n_pv + 1), key_deg, (int64_t)mode);
    {
        auto it = c->tuned.find(key);
        if (it != c->tuned.end() && !ms_out) {
            opts->tile_w = it->second[0];
            opts->tile_h = it->second[1];
            opts->batch_depth = it->second[2];
            opts->persistent = it->second[3];
            if (n_candidates) *n_candidates = 0;
            return PBR_OK;
        }
    }
    static const int tiles[3][2] = {{16, 16}, {8, 8}, {16, 32}};
    static const int scheds[5][2] = {{0, 0}, {0, 1}, {128, 0}, {256, 0}, {512, 0}};
    cudaStream_t s = (cudaStream_t)stream;
    float *img = nullptr, *grad = nullptr, *gpos = nullptr, *gsh = nullptr;
    int64_t n_tot = 0, n_sh = 0;
    for (int q = 0; q < n_scenes; ++q) {
        n_tot += scenes[q].n;
        n_sh += scenes[q].n * (scenes[q].sh_degree + 1) * (scenes[q].sh_degree + 1) * 3;
    }
    PBR_CUDA(cudaMalloc(&img, sizeof(float) * 3 * (L.n_pix ? L.n_pix : 1)));
    if (mode == 1) {
        PBR_CUDA(cudaMalloc(&grad, sizeof(float) * 3 * (L.n_pix ? L.n_pix : 1)));
        PBR_CUDA(cudaMemset(grad, 0, sizeof(float) * 3 * L.n_pix));
        PBR_CUDA(cudaMalloc(&gpos, sizeof(float) * 3 * (n_tot ? n_tot : 1)));
        PBR_CUDA(cudaMalloc(&gsh, sizeof(float) * (n_sh ? n_sh : 1)));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    pbr_render_opts best_o = *opts;
    int idx = 0, rc = PBR_OK;
    for (const auto &t : tiles) {
        for (const auto &sc : scheds) {
            pbr_render_opts o = *opts;
            o.tile_w = t[0];
            o.tile_h = t[1];
            o.batch_depth = sc[0];
            o.persistent = sc[1];
            o.no_pair_stats = 1; // time the kernels the captured graphs run
            float total = 0.f;
            for (int r = 0; r <= reps && rc == PBR_OK; ++r) {
                cudaEventRecord(e0, s);
                pbr_state *st = nullptr;
                rc = pbr_render_forward(c, scenes, n_scenes, scene_of_view, cams, n_cams, &o, img,
                                        mode == 1 ? &st : nullptr, stream);
                if (rc == PBR_OK && mode == 1)
                    rc = pbr_render_backward(c, st, grad, gpos, gsh, nullptr, stream);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                if (st) pbr_state_free(c, st);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) total += ms;
            }
            if (rc != PBR_OK) break;
            const double ms = total / reps;
            if (ms_out) ms_out[idx] = ms;
            if (ms < best) {
                best = ms;
                best_o = o;
            }
            ++idx;
        }
        if (rc != PBR_OK) break;
    }
    best_o.no_pair_stats = opts->no_pair_stats;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(img);
    if (grad) cudaFree(grad);
    if (gpos) cudaFree(gpos);
    if (gsh) cudaFree(gsh);
    if (rc != PBR_OK) return rc;
    *opts = best_o;
    c->tuned[key] = {best_o.tile_w, best_o.tile_h, best_o.batch_depth, best_o.persistent};
    if (n_candidates) *n_candidates = idx;
    return PBR_OK;
}

// ------------------------------------------------- autotuner cache on disk
// One JSON object: {"format": "pbr-autotune-1", "classes": [{...}, ...]},
// one object per shape class with the integer fields of kTuneFields.
namespace {

const char *const kTuneFields[9] = {"views",  "log2_pixels", "log2_point_views",
                                    "degrees", "mode",        "tile_w",
                                    "tile_h",  "batch_depth", "persistent"};

// Integer value of "name": inside [b, e); false if absent or malformed.
bool json_int_field(const char *b, const char *e, const char *name, int64_t &out)
{
    const size_t n = std::strlen(name);
    for (const char *p = b; p + n + 2 < e; ++p) {
        if (p[0] != '"' || std::strncmp(p + 1, name, n) != 0 || p[n + 1] != '"') continue;
        const char *q = p + n + 2;
        while (q < e && (*q == ' ' || *q == '\t' || *q == '\n' || *q == '\r')) ++q;
        if (q >= e || *q != ':') return false;
        ++q;
        while (q < e && (*q == ' ' || *q == '\t' || *q == '\n' || *q == '\r')) ++q;
        bool neg = false;
        if (q < e && *q == '-') {
            neg = true;
            ++q;
        }
        if (q >= e || *q < '0' || *q > '9') return false;
        int64_t v = 0;
        while (q < e && *q >= '0' && *q <= '9') {
            if (v > (INT64_MAX - 9) / 10) return false;
            v = v * 10 + (*q++ - '0');
        }
        out = neg ? -v : v;
        return true;
    }
    return false;
}

} // namespace

extern "C" int pbr_autotune_save(const pbr_ctx *c, const char *path)
{
    if (!c || !path) return set_error(PBR_ERR_INVALID_ARG, "pbr_autotune_save: NULL argument");
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return set_error(PBR_ERR_INVALID_ARG, "cannot write %s", tmp.c_str());
    std::fprintf(f, "{\"format\": \"pbr-autotune-1\", \"classes\": [");
    bool first = true;
    for (const auto &kv : c->tuned) {
        const int64_t v[9] = {std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                              std::get<3>(kv.first), std::get<4>(kv.first), kv.second[0],
                              kv.second[1],          kv.second[2],          kv.second[3]};
        std::fprintf(f, "%s\n  {", first ? "" : ",");
        for (int k = 0; k < 9; ++k)
            std::fprintf(f, "%s\"%s\": %lld", k ? ", " : "", kTuneFields[k], (long long)v[k]);
        std::fprintf(f, "}");
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    const bool ok = std::fflush(f) == 0 && !std::ferror(f);
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return set_error(PBR_ERR_INVALID_ARG, "cannot write %s", path);
    }
    return PBR_OK;
}

extern "C" int pbr_autotune_load(pbr_ctx *c, const char *path, int32_t *n_loaded)
{
    if (n_loaded) *n_loaded = 0;
    if (!c || !path) return set_error(PBR_ERR_INVALID_ARG, "pbr_autotune_load: NULL argument");
    FILE *f = std::fopen(path, "r");
    if (!f) return set_error(PBR_ERR_NOT_FOUND, "cannot read %s", path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) {
        text.append(buf, got);
        if (text.size() > (64u << 20)) {
            std::fclose(f);
            return set_error(PBR_ERR_INVALID_ARG, "%s: larger than 64 MiB", path);
        }
    }
    std::fclose(f);
    if (text.find("\"pbr-autotune-1\"") == std::string::npos)
        return set_error(PBR_ERR_INVALID_ARG, "%s: not an autotuner cache", path);
    const size_t lst = text.find("\"classes\"");
    if (lst == std::string::npos)
        return set_error(PBR_ERR_INVALID_ARG, "%s: no \"classes\" list", path);
    // parse every entry before changing the cache: a bad file changes nothing
    std::vector<std::pair<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>,
                          std::array<int, 4>>> entries;
    size_t pos = text.find('[', lst);
    if (pos == std::string::npos)
        return set_error(PBR_ERR_INVALID_ARG, "%s: no \"classes\" list", path);
    for (;;) {
        const size_t ob = text.find('{', pos), cl = text.find(']', pos);
        if (ob == std::string::npos || (cl != std::string::npos && cl < ob)) break;
        const size_t oe = text.find('}', ob);
        if (oe == std::string::npos)
            return set_error(PBR_ERR_INVALID_ARG, "%s: unterminated entry", path);
        int64_t v[9];
        for (int k = 0; k < 9; ++k)
            if (!json_int_field(text.data() + ob, text.data() + oe, kTuneFields[k], v[k]))
                return set_error(PBR_ERR_INVALID_ARG, "%s: entry %zu lacks an integer \"%s\"",
                                 path, entries.size(), kTuneFields[k]);
        pbr_render_opts o;
        pbr_default_opts(&o);
        o.tile_w = (int32_t)v[5];
        o.tile_h = (int32_t)v[6];
        o.batch_depth = (int32_t)v[7];
        o.persistent = (int32_t)v[8];
        if (v[5] != o.tile_w || v[6] != o.tile_h || v[7] != o.batch_depth ||
            (v[8] != 0 && v[8] != 1) || (v[4] != 0 && v[4] != 1) || check_opts(&o) != PBR_OK)
            return set_error(PBR_ERR_INVALID_ARG, "%s: entry %zu holds an invalid schedule", path,
                             entries.size());
        entries.push_back({std::make_tuple(v[0], v[1], v[2], v[3], v[4]),
                           {(int)v[5], (int)v[6], (int)v[7], (int)v[8]}});
        pos = oe + 1;
    }
    for (const auto &e : entries) c->tuned[e.first] = e.second;
    if (n_loaded) *n_loaded = (int32_t)entries.size();
    return PBR_OK;
}
