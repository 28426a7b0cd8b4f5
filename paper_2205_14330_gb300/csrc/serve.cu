// Serving loop of libpbr: continuous batching of render requests over
// scenes kept resident in HBM.
//
// Callers upload scenes once (pbr_upload_scene) and submit requests (scene,
// camera of any size, output buffer).  A host thread owned by the context
// admits queued requests into a batch while
//   - a CUDA stream slot is free (n_streams batches can be in flight),
//   - the batch holds at most max_batch_views views, and
//   - the estimated workspace of the batch fits in what the HBM budget has
//     left after the batches already in flight;
// it then renders the whole batch -- views of different scenes and sizes --
// with one forward chain on that slot's stream, each view writing straight
// into its request's buffer.  Requests that arrive while batches run are
// admitted as soon as a slot and memory free up, so their work overlaps the
// batches on the device.  Completion is observed with CUDA events; latency
// is completion minus arrival on the host's steady clock.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

using namespace pbr;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct SceneRes {
    pbr_points pts{}; // device pointers owned by the library
    void *mem = nullptr;
    int refs = 0; // queued or in-flight requests
    // bounds for the admission estimate: a sphere holding every point and
    // the largest radius
    double centre[3] = {0.0, 0.0, 0.0};
    double extent = 0.0, r_max = 0.0;
};

struct Request {
    uint64_t id = 0;
    int32_t scene = 0;
    pbr_camera cam{};
    float *out = nullptr;
    double t_arrival = 0, t_done = 0;
    int32_t status = PBR_OK;
    bool done = false;
    size_t bytes = 0;
};

struct InFlight {
    std::vector<uint64_t> ids;
    std::vector<int32_t> scenes;
    int slot = 0;
    cudaEvent_t ev = nullptr;       // completion (timing) event
    cudaEvent_t ev_start = nullptr; // recorded on the slot's stream before the batch
    size_t bytes = 0;
};

// Admission reservation of one view of a resident scene: the bytes its
// forward pass allocates (pbr::forward_bytes) with every point-view visible
// and every point-view listed in as many tiles as the largest splat can
// reach.  The largest splat is the largest radius at the smallest depth of
// the scene's bounding sphere along the camera's axis (no nearer than
// z_near), so the bound holds for every camera; it is loose for splats
// below the largest.  Returns 0 when the layout is invalid.
size_t admission_bytes(const SceneRes &sc, const pbr_camera &cam, const pbr_render_opts &o)
{
    HostLayout L;
    if (build_layout(&sc.pts, 1, nullptr, &cam, 1, &o, L) != PBR_OK) return 0;
    // camera centre C = -R^T t, optical axis a = R^T e_z
    double C[3], a[3];
    for (int k = 0; k < 3; ++k) {
        C[k] = -(cam.R[k] * cam.t[0] + cam.R[3 + k] * cam.t[1] + cam.R[6 + k] * cam.t[2]);
        a[k] = cam.R[6 + k];
    }
    const double along = a[0] * (sc.centre[0] - C[0]) + a[1] * (sc.centre[1] - C[1]) +
                         a[2] * (sc.centre[2] - C[2]);
    const double z_min = std::max((double)o.z_near, along - sc.extent);
    const double sigma = o.radius_mode == 0 ? cam.fx * sc.r_max / z_min
                                            : sc.r_max * std::min(cam.width, cam.height) * 0.5;
    const double side = 2.0 * o.cutoff_k * sigma + 3.0; // pixel box of the splat
    const double tx = std::ceil(side / o.tile_w) + 1.0, ty = std::ceil(side / o.tile_h) + 1.0;
    const double tiles = std::min((double)L.n_tiles, tx * ty);
    const double pairs = std::min((double)L.n_pv * tiles, 4.0e18);
    return forward_bytes(L, L.n_pv, (int64_t)pairs, &o, 0);
}

} // namespace

struct ServeState {
    pbr_ctx *ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stop = false;
    pbr_render_opts opts{};
    int max_views = 64;
    size_t budget = 0, in_use = 0;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::map<int32_t, SceneRes> scenes;
    int32_t next_scene = 0;
    uint64_t next_id = 1;
    std::vector<cudaStream_t> streams;
    std::vector<bool> busy;
    // exact workspace queries of admission (reserve_bytes)
    cudaStream_t admit_stream = nullptr;
    std::mutex admit_mu;
    std::vector<InFlight> inflight;
    // device intervals of completed batches: [start, end) in ms after t0_ev
    cudaEvent_t t0_ev = nullptr;
    std::vector<double> trace_start, trace_end;
    std::vector<int32_t> trace_views;
    // statistics
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, views = 0, max_batch = 0;
    double pixels = 0.0, t_first = -1.0, t_last = 0.0;

    void loop();
    void finish_ready();
    bool launch_one();
};

void ServeState::finish_ready()
{
    // caller holds mu
    for (size_t i = 0; i < inflight.size();) {
        InFlight &b = inflight[i];
        const cudaError_t q = cudaEventQuery(b.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = now_s();
        for (uint64_t id : b.ids) {
            auto it = reqs.find(id);
            if (it == reqs.end()) continue;
            Request &r = it->second;
            r.done = true;
            r.t_done = t;
            r.status = q == cudaSuccess ? PBR_OK : PBR_ERR_CUDA;
            lat_ms.push_back(1e3 * (t - r.t_arrival));
            pixels += (double)r.cam.width * r.cam.height;
            ++completed;
            t_last = t;
        }
        for (int32_t s : b.scenes) scenes[s].refs--;
        float ms0 = 0.f, ms1 = 0.f;
        if (t0_ev && b.ev_start && q == cudaSuccess &&
            cudaEventElapsedTime(&ms0, t0_ev, b.ev_start) == cudaSuccess &&
            cudaEventElapsedTime(&ms1, t0_ev, b.ev) == cudaSuccess) {
            trace_start.push_back(ms0);
            trace_end.push_back(ms1);
            trace_views.push_back((int32_t)b.ids.size());
        }
        cudaGetLastError();
        cudaEventDestroy(b.ev);
        if (b.ev_start) cudaEventDestroy(b.ev_start);
        busy[b.slot] = false;
        in_use -= b.bytes;
        inflight.erase(inflight.begin() + (long)i);
        done_cv.notify_all();
    }
}

bool ServeState::launch_one()
{
    // caller holds mu; returns true if a batch was launched
    int slot = -1;
    for (size_t k = 0; k < busy.size(); ++k)
        if (!busy[k]) {
            slot = (int)k;
            break;
        }
    if (slot < 0 || queue.empty()) return false;
    std::vector<uint64_t> ids;
    size_t bytes = 0;
    while (!queue.empty() && (int)ids.size() < max_views) {
        Request &r = reqs[queue.front()];
        if (in_use + bytes + r.bytes > budget) {
            if (ids.empty() && inflight.empty()) { // can never fit: reject
                r.done = true;
                r.status = PBR_ERR_OOM;
                scenes[r.scene].refs--;
                ++rejected;
                queue.pop_front();
                done_cv.notify_all();
                continue;
            }
            break; // wait for memory to free up
        }
        bytes += r.bytes;
        ids.push_back(queue.front());
        queue.pop_front();
    }
    if (ids.empty()) return false;
    // the batch: scenes referenced, one view per request
    std::vector<int32_t> scene_ids;
    std::vector<pbr_points> pts;
    std::vector<int32_t> sov;
    std::vector<pbr_camera> cams;
    std::vector<float *> outs;
    for (uint64_t id : ids) {
        const Request &r = reqs[id];
        auto f = std::find(scene_ids.begin(), scene_ids.end(), r.scene);
        int idx = (int)(f - scene_ids.begin());
        if (f == scene_ids.end()) {
            scene_ids.push_back(r.scene);
            pts.push_back(scenes[r.scene].pts);
        }
        sov.push_back(idx);
        cams.push_back(r.cam);
        outs.push_back(r.out);
    }
    cudaStream_t s = streams[slot];
    cudaEvent_t ev_start = nullptr;
    if (cudaEventCreate(&ev_start) != cudaSuccess || cudaEventRecord(ev_start, s) != cudaSuccess) {
        if (ev_start) cudaEventDestroy(ev_start);
        ev_start = nullptr;
        cudaGetLastError();
    }
    pbr_state st;
    st.stream = s;
    st.opts = opts;
    st.dopts = dev_opts(&opts);
    st.batch_depth = opts.batch_depth;
    int rc = build_layout(pts.data(), (int32_t)pts.size(), sov.data(), cams.data(),
                          (int32_t)cams.size(), &opts, st.layout);
    if (rc == PBR_OK) {
        for (size_t v = 0; v < outs.size(); ++v) st.layout.views[v].out = outs[v];
        // the per-point stage synchronises this slot's stream once; other
        // slots keep running meanwhile
        mu.unlock();
        rc = forward_eager(ctx, &st, outs[0], s);
        mu.lock();
    }
    st.release();
    cudaEvent_t ev = nullptr;
    if (rc == PBR_OK && cudaEventCreate(&ev) == cudaSuccess && cudaEventRecord(ev, s) == cudaSuccess) {
        InFlight b;
        b.ids = ids;
        for (uint64_t id : ids) b.scenes.push_back(reqs[id].scene);
        b.slot = slot;
        b.ev = ev;
        b.ev_start = ev_start;
        b.bytes = bytes;
        busy[slot] = true;
        in_use += bytes;
        inflight.push_back(b);
        ++batches;
        views += (int64_t)ids.size();
        max_batch = std::max<int64_t>(max_batch, (int64_t)ids.size());
        return true;
    }
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    if (ev_start) cudaEventDestroy(ev_start);
    for (uint64_t id : ids) {
        Request &r = reqs[id];
        r.done = true;
        r.status = rc != PBR_OK ? rc : PBR_ERR_CUDA;
        scenes[r.scene].refs--;
        ++rejected;
    }
    done_cv.notify_all();
    return true;
}

void ServeState::loop()
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        finish_ready();
        if (stop && queue.empty() && inflight.empty()) break;
        if (launch_one()) continue;
        if (inflight.empty() && queue.empty()) {
            cv.wait_for(lk, std::chrono::milliseconds(50));
        } else {
            // batches running (or waiting for memory): poll their events
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

namespace pbr {
void serve_shutdown(pbr_ctx *c)
{
    ServeState *S = c->serve;
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(c->device);
    for (auto &kv : S->scenes) cudaFree(kv.second.mem);
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    if (S->admit_stream) cudaStreamDestroy(S->admit_stream);
    if (S->t0_ev) cudaEventDestroy(S->t0_ev);
    delete S;
    c->serve = nullptr;
}
} // namespace pbr

extern "C" int pbr_serve_start(pbr_ctx *c, const pbr_render_opts *opts, int32_t max_batch_views,
                               int32_t n_streams)
{
    if (!c) return set_error(PBR_ERR_INVALID_ARG, "ctx is NULL");
    if (c->serve) return set_error(PBR_ERR_BUSY, "serving loop already running");
    if (max_batch_views < 1 || n_streams < 1 || n_streams > 16)
        return set_error(PBR_ERR_INVALID_ARG, "max_batch_views >= 1, n_streams in 1..16");
    PBR_TRY(check_opts(opts));
    PBR_CUDA(cudaSetDevice(c->device));
    ServeState *S = new ServeState();
    S->ctx = c;
    S->opts = *opts;
    S->max_views = max_batch_views;
    S->budget = c->hbm_budget;
    for (int k = 0; k < n_streams; ++k) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
            delete S;
            return set_error(PBR_ERR_CUDA, "stream creation failed");
        }
        S->streams.push_back(s);
        S->busy.push_back(false);
    }
    if (cudaStreamCreateWithFlags(&S->admit_stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
        delete S;
        return set_error(PBR_ERR_CUDA, "stream creation failed");
    }
    // reference point of the batch trace (pbr_serve_trace)
    if (cudaEventCreate(&S->t0_ev) != cudaSuccess || cudaEventRecord(S->t0_ev, S->streams[0]) != cudaSuccess) {
        cudaGetLastError();
        if (S->t0_ev) cudaEventDestroy(S->t0_ev);
        S->t0_ev = nullptr;
    }
    c->serve = S;
    S->th = std::thread([S] { S->loop(); });
    return PBR_OK;
}

extern "C" int pbr_serve_stop(pbr_ctx *c)
{
    if (!c) return set_error(PBR_ERR_INVALID_ARG, "ctx is NULL");
    serve_shutdown(c);
    return PBR_OK;
}

extern "C" int pbr_upload_scene(pbr_ctx *c, const pbr_points *p, int32_t *scene_id)
{
    if (!c || !p || !scene_id) return set_error(PBR_ERR_INVALID_ARG, "bad arguments");
    ServeState *S = c->serve;
    if (!S) return set_error(PBR_ERR_INVALID_ARG, "start the serving loop first (pbr_serve_start)");
    if (p->n < 0 || p->sh_degree < 0 || p->sh_degree > 3 ||
        (p->n > 0 && (!p->pos || !p->sh || !p->opacity || !p->radius)))
        return set_error(PBR_ERR_INVALID_ARG, "bad point set");
    PBR_CUDA(cudaSetDevice(c->device));
    const int64_t n = p->n;
    const int K = (p->sh_degree + 1) * (p->sh_degree + 1);
    const size_t b_pos = 12 * (size_t)n, b_sh = 12 * (size_t)K * n, b_s = 4 * (size_t)n;
    const size_t a = 256;
    auto up = [&](size_t x) { return (x + a - 1) / a * a; };
    const size_t total = up(b_pos) + up(b_sh) + 2 * up(b_s) + a;
    char *mem = nullptr;
    if (cudaMalloc((void **)&mem, total) != cudaSuccess) {
        cudaGetLastError();
        return set_error(PBR_ERR_OOM, "scene of %lld points does not fit", (long long)n);
    }
    pbr_points d = *p;
    d.pos = (const float *)mem;
    d.sh = (const float *)(mem + up(b_pos));
    d.opacity = (const float *)(mem + up(b_pos) + up(b_sh));
    d.radius = (const float *)(mem + up(b_pos) + up(b_sh) + up(b_s));
    // host or device sources (unified addressing decides)
    if (n > 0) {
        const cudaError_t e = [&] {
            cudaError_t r = cudaMemcpy((void *)d.pos, p->pos, b_pos, cudaMemcpyDefault);
            if (r == cudaSuccess) r = cudaMemcpy((void *)d.sh, p->sh, b_sh, cudaMemcpyDefault);
            if (r == cudaSuccess) r = cudaMemcpy((void *)d.opacity, p->opacity, b_s, cudaMemcpyDefault);
            if (r == cudaSuccess) r = cudaMemcpy((void *)d.radius, p->radius, b_s, cudaMemcpyDefault);
            return r;
        }();
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(mem);
            return set_error(PBR_ERR_CUDA, "scene upload: %s", cudaGetErrorString(e));
        }
    }
    SceneRes r;
    r.pts = d;
    r.mem = mem;
    if (n > 0) { // bounds of the admission estimate, from a host copy
        std::vector<float> hp(3 * (size_t)n), hr((size_t)n);
        if (cudaMemcpy(hp.data(), d.pos, b_pos, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(hr.data(), d.radius, b_s, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(mem);
            return set_error(PBR_ERR_CUDA, "scene upload: reading the bounds back failed");
        }
        double lo[3] = {hp[0], hp[1], hp[2]}, hi[3] = {hp[0], hp[1], hp[2]};
        for (int64_t i = 0; i < n; ++i) {
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], (double)hp[3 * i + k]);
                hi[k] = std::max(hi[k], (double)hp[3 * i + k]);
            }
            r.r_max = std::max(r.r_max, (double)hr[i]);
        }
        double e2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            r.centre[k] = 0.5 * (lo[k] + hi[k]);
            e2 += 0.25 * (hi[k] - lo[k]) * (hi[k] - lo[k]);
        }
        r.extent = std::sqrt(e2) * (1.0 + 1e-6) + 1e-6; // the box's half diagonal
    }
    std::lock_guard<std::mutex> g(S->mu);
    *scene_id = S->next_scene++;
    S->scenes[*scene_id] = r;
    return PBR_OK;
}

extern "C" int pbr_evict_scene(pbr_ctx *c, int32_t scene_id)
{
    if (!c || !c->serve) return set_error(PBR_ERR_INVALID_ARG, "no serving loop");
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->scenes.find(scene_id);
    if (it == S->scenes.end()) return set_error(PBR_ERR_NOT_FOUND, "no scene %d", scene_id);
    if (it->second.refs > 0)
        return set_error(PBR_ERR_BUSY, "scene %d has %d pending requests", scene_id,
                         it->second.refs);
    cudaFree(it->second.mem);
    S->scenes.erase(it);
    return PBR_OK;
}

// The bytes a request reserves: the host bound of admission_bytes, or, when
// that bound would take more than 1/64 of the budget (a camera close to or
// inside the scene's bounding box makes it loose), the exact workspace of
// the view from a counting pass on the device (pbr_forward_workspace_size),
// so that loose bounds do not hold back other requests.  The scene must be
// pinned (refs > 0) by the caller; mu is not held.
static int reserve_bytes(pbr_ctx *c, ServeState *S, const pbr_points &pts, size_t bound,
                         size_t budget, const pbr_camera &cam, size_t *bytes)
{
    *bytes = bound;
    if (bound <= budget / 64) return PBR_OK;
    std::lock_guard<std::mutex> ga(S->admit_mu);
    size_t exact = 0;
    PBR_TRY(pbr_forward_workspace_size(c, &pts, 1, nullptr, &cam, 1, &S->opts, 0, &exact, nullptr,
                                       (pbr_stream_t)S->admit_stream));
    *bytes = std::min(bound, exact);
    return PBR_OK;
}

extern "C" int pbr_submit_request(pbr_ctx *c, int32_t scene_id, const pbr_camera *cam,
                                  float *out_rgb_device, double arrival_time, uint64_t *req_id)
{
    if (!c || !c->serve || !cam || !out_rgb_device || !req_id)
        return set_error(PBR_ERR_INVALID_ARG, "bad arguments (is the serving loop running?)");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768)
        return set_error(PBR_ERR_INVALID_ARG, "camera size %dx%d", cam->width, cam->height);
    ServeState *S = c->serve;
    pbr_points pts{};
    size_t bound = 0, budget = 0;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->scenes.find(scene_id);
        if (it == S->scenes.end()) return set_error(PBR_ERR_NOT_FOUND, "no scene %d", scene_id);
        bound = admission_bytes(it->second, *cam, S->opts);
        if (bound == 0) return set_error(PBR_ERR_INVALID_ARG, "request camera is invalid");
        pts = it->second.pts;
        budget = S->budget;
        it->second.refs++; // pinned from here on (queued requests hold a reference)
    }
    size_t bytes = 0;
    const int rc = reserve_bytes(c, S, pts, bound, budget, *cam, &bytes);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (rc != PBR_OK) {
            S->scenes[scene_id].refs--;
            return rc;
        }
        Request r;
        r.id = S->next_id++;
        r.scene = scene_id;
        r.cam = *cam;
        r.out = out_rgb_device;
        r.t_arrival = arrival_time > 0.0 ? arrival_time : now_s();
        r.bytes = bytes;
        S->reqs[r.id] = r;
        S->queue.push_back(r.id);
        ++S->submitted;
        if (S->t_first < 0) S->t_first = r.t_arrival;
        *req_id = r.id;
    }
    S->cv.notify_all();
    return PBR_OK;
}

extern "C" int pbr_poll(pbr_ctx *c, uint64_t req_id, int32_t *done, int32_t *status)
{
    if (!c || !c->serve) return set_error(PBR_ERR_INVALID_ARG, "no serving loop");
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return set_error(PBR_ERR_NOT_FOUND, "no request %llu",
                                              (unsigned long long)req_id);
    if (done) *done = it->second.done ? 1 : 0;
    if (status) *status = it->second.status;
    if (it->second.done) S->reqs.erase(it);
    return PBR_OK;
}

extern "C" int pbr_wait(pbr_ctx *c, uint64_t req_id, int32_t timeout_ms, int32_t *status)
{
    if (!c || !c->serve) return set_error(PBR_ERR_INVALID_ARG, "no serving loop");
    ServeState *S = c->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return set_error(PBR_ERR_NOT_FOUND, "no request %llu",
                                              (unsigned long long)req_id);
    const bool ok = S->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto j = S->reqs.find(req_id);
        return j == S->reqs.end() || j->second.done;
    });
    if (!ok) return set_error(PBR_ERR_TIMEOUT, "request %llu not done after %d ms",
                              (unsigned long long)req_id, timeout_ms);
    it = S->reqs.find(req_id);
    if (status) *status = it != S->reqs.end() ? it->second.status : PBR_OK;
    if (it != S->reqs.end()) S->reqs.erase(it);
    return PBR_OK;
}

extern "C" int pbr_serve_stats(pbr_ctx *c, pbr_serve_stats_t *out, int32_t reset)
{
    if (!c || !c->serve || !out) return set_error(PBR_ERR_INVALID_ARG, "no serving loop");
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->queued = (int64_t)S->queue.size();
    out->in_flight_batches = (int64_t)S->inflight.size();
    out->batches = S->batches;
    out->max_batch_views = S->max_batch;
    out->mean_batch_views = S->batches ? (double)S->views / (double)S->batches : 0.0;
    out->megapixels = S->pixels / 1e6;
    out->span_s = S->t_first >= 0 ? S->t_last - S->t_first : 0.0;
    out->hbm_in_use = S->in_use;
    out->hbm_budget = S->budget;
    std::vector<double> l = S->lat_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double x = p * (double)(l.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - (double)i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double v : l) sum += v;
        out->mean_ms = sum / (double)l.size();
        out->max_ms = l.back();
    }
    if (reset) {
        S->lat_ms.clear();
        S->submitted = S->completed = S->rejected = S->batches = S->views = S->max_batch = 0;
        S->pixels = 0.0;
        S->t_first = -1.0;
        S->t_last = 0.0;
    }
    return PBR_OK;
}

extern "C" double pbr_now(void) { return now_s(); }

extern "C" int pbr_serve_set_budget(pbr_ctx *c, size_t hbm_budget_bytes)
{
    if (!c) return set_error(PBR_ERR_INVALID_ARG, "ctx is NULL");
    c->hbm_budget = hbm_budget_bytes;
    if (c->serve) {
        std::lock_guard<std::mutex> g(c->serve->mu);
        c->serve->budget = hbm_budget_bytes;
    }
    return PBR_OK;
}

extern "C" int pbr_serve_trace(pbr_ctx *c, double *start_ms, double *end_ms, int32_t *views,
                               int32_t cap, int32_t *n, int32_t reset)
{
    if (!c || !c->serve || !n || cap < 0) return set_error(PBR_ERR_INVALID_ARG, "bad arguments");
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    const int32_t m = (int32_t)S->trace_start.size();
    *n = m;
    for (int32_t i = 0; i < m && i < cap; ++i) {
        if (start_ms) start_ms[i] = S->trace_start[i];
        if (end_ms) end_ms[i] = S->trace_end[i];
        if (views) views[i] = S->trace_views[i];
    }
    if (reset) {
        S->trace_start.clear();
        S->trace_end.clear();
        S->trace_views.clear();
    }
    return PBR_OK;
}

extern "C" int pbr_serve_estimate(pbr_ctx *c, int32_t scene_id, const pbr_camera *cam,
                                  size_t *bytes)
{
    if (!c || !c->serve || !cam || !bytes)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_serve_estimate: bad arguments");
    ServeState *S = c->serve;
    pbr_points pts{};
    size_t bound = 0, budget = 0;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->scenes.find(scene_id);
        if (it == S->scenes.end()) return set_error(PBR_ERR_NOT_FOUND, "no scene %d", scene_id);
        bound = admission_bytes(it->second, *cam, S->opts);
        if (bound == 0) return set_error(PBR_ERR_INVALID_ARG, "camera is invalid");
        pts = it->second.pts;
        budget = S->budget;
        it->second.refs++;
    }
    const int rc = reserve_bytes(c, S, pts, bound, budget, *cam, bytes);
    std::lock_guard<std::mutex> g(S->mu);
    S->scenes[scene_id].refs--;
    return rc;
}
