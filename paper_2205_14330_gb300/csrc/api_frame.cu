// C entry points of the video frame initialisation (Sec. 3.4): the Chamfer
// distance with its gradient, and the whole initialisation (Adam descent
// of the new frame's positions on the Chamfer distance, then the transfer
// of the previous frame's parameters from the closest points).
#include <algorithm>
#include <cmath>

#include "api_internal.h"

using namespace pbr;

namespace {

// Nearest-point maps between the clouds: nn12[i] for p1[i] in p2 (index of
// p2 built here), nn21[j] for p2[j] in p1 (index S1 given).
int nearest_maps(TempBufs &tb, const float *p1, int64_t n1, const SearchIndex &S1,
                 const float *p2, int64_t n2, int32_t *nn12, int32_t *nn21, cudaStream_t s)
{
    SearchIndex S2;
    PBR_TRY(make_params(tb, p2, n2, auto_cells(n2), S2, s));
    PBR_TRY(index_points(tb, p2, n2, S2, s));
    float *d12, *d21;
    PBR_TRY(tb.alloc(&d12, sizeof(float) * n1));
    PBR_TRY(tb.alloc(&d21, sizeof(float) * n2));
    PBR_TRY(run_knn(tb, p1, n1, p2, n2, S2, 1, 1, 0, nn12, d12, s));
    PBR_TRY(run_knn(tb, p2, n2, p1, n1, S1, 1, 1, 0, nn21, d21, s));
    return PBR_OK;
}

bool finite_pos(float x) { return std::isfinite(x) && x >= 0.0f; }

// Records one descent step on stream cs (capturing): nearest-point maps,
// CD into *cur, dCD/dp2, Adam with the step number and rate of *ost.
int record_step(const float *p1, int64_t n1, const SearchIndex &S1, float *pos2, int64_t n2,
                const pbr_frame_cfg &cfg, float *grad, float *m, float *v, int32_t *nn12,
                int32_t *nn21, double *cur, OptState *ost, cudaStream_t cs)
{
    TempBufs it(cs);
    PBR_TRY(nearest_maps(it, p1, n1, S1, pos2, n2, nn12, nn21, cs));
    PBR_CUDA(cudaMemsetAsync(cur, 0, sizeof(double), cs));
    launch_chamfer(p1, n1, pos2, n2, nn12, nn21, grad, cur, cs);
    launch_step_counter(ost, cs);
    const OptParams prm{1, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, 0};
    launch_optimizer(prm, ost, 0, pos2, grad, m, v, 3 * n2, cs);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

// cfg.iters descent steps on pos2, the loss before step t in hist[t - 1]:
// the step is captured once on a private stream and replayed.
int descend(TempBufs &tb, const float *p1, int64_t n1, const SearchIndex &S1, float *pos2,
            int64_t n2, const pbr_frame_cfg &cfg, float *grad, float *m, float *v,
            int32_t *nn12, int32_t *nn21, double *hist, cudaStream_t s)
{
    OptState *ost;
    double *cur;
    PBR_TRY(tb.alloc(&ost, sizeof(OptState)));
    PBR_TRY(tb.alloc(&cur, sizeof(double)));
    const OptState init{{cfg.lr, 0.0f, 0.0f}, 0};
    PBR_CUDA(cudaMemcpyAsync(ost, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = PBR_OK;
    do {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: stream or event creation failed");
            break;
        }
        // cs starts after everything queued on s so far
        if (cudaEventRecord(ev, s) != cudaSuccess || cudaStreamWaitEvent(cs, ev, 0) != cudaSuccess) {
            rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: stream ordering failed");
            break;
        }
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: capture failed to start");
            break;
        }
        rc = record_step(p1, n1, S1, pos2, n2, cfg, grad, m, v, nn12, nn21, cur, ost, cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (rc != PBR_OK) break;
        if (ec != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: step capture failed");
            break;
        }
        for (int t = 1; t <= cfg.iters && rc == PBR_OK; ++t) {
            if (cudaGraphLaunch(exec, cs) != cudaSuccess ||
                cudaMemcpyAsync(hist + t - 1, cur, sizeof(double), cudaMemcpyDeviceToDevice,
                                cs) != cudaSuccess)
                rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: step replay failed");
        }
        // s continues after the replays
        if (cudaEventRecord(ev, cs) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess)
            rc = set_error(PBR_ERR_CUDA, "pbr_frame_init: stream ordering failed");
    } while (false);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    if (ev) cudaEventDestroy(ev);
    return rc;
}

} // namespace

extern "C" void pbr_default_frame_cfg(pbr_frame_cfg *cfg)
{
    if (!cfg) return;
    cfg->iters = 100;
    cfg->lr = 1e-3f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.999f;
    cfg->eps = 1e-8f;
    cfg->k = 4;
    cfg->reserved[0] = cfg->reserved[1] = 0;
}

extern "C" int pbr_chamfer(pbr_ctx *ctx, const float *p1, int64_t n1, const float *p2, int64_t n2,
                           double *loss_dev, float *grad2, int32_t *nn12, int32_t *nn21,
                           pbr_stream_t stream)
{
    if (!ctx || !p1 || !p2 || !loss_dev || n1 < 1 || n2 < 1 || n1 > 0x7fffffffLL ||
        n2 > 0x7fffffffLL)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_chamfer: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    TempBufs tb(s);
    if (!nn12) PBR_TRY(tb.alloc(&nn12, sizeof(int32_t) * n1));
    if (!nn21) PBR_TRY(tb.alloc(&nn21, sizeof(int32_t) * n2));
    SearchIndex S1;
    PBR_TRY(make_params(tb, p1, n1, auto_cells(n1), S1, s));
    PBR_TRY(index_points(tb, p1, n1, S1, s));
    PBR_TRY(nearest_maps(tb, p1, n1, S1, p2, n2, nn12, nn21, s));
    PBR_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(double), s));
    launch_chamfer(p1, n1, p2, n2, nn12, nn21, grad2, loss_dev, s);
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_frame_init(pbr_ctx *ctx, const pbr_points *prev, float *pos2, int64_t n2,
                              const pbr_frame_cfg *cfg, float *sh2, float *opacity2,
                              float *radius2, double *loss_history, pbr_stream_t stream)
{
    if (!ctx || !prev || !cfg || !pos2 || !sh2 || !opacity2 || !radius2)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_frame_init: null argument");
    const int64_t n1 = prev->n;
    if (n1 < 1 || n2 < 1 || n1 > 0x7fffffffLL || n2 > 0x7fffffffLL || prev->sh_degree < 0 ||
        prev->sh_degree > 3 || !prev->pos || !prev->sh || !prev->opacity || !prev->radius ||
        cfg->iters < 0 || cfg->k < 1 || cfg->k > 32 || !finite_pos(cfg->lr) ||
        !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps > 0.0f))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_frame_init: bad configuration");
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    const int nsh = 3 * (prev->sh_degree + 1) * (prev->sh_degree + 1);
    const float *p1 = prev->pos;
    TempBufs tb(s);

    // the previous frame's search index, built once
    SearchIndex S1;
    PBR_TRY(make_params(tb, p1, n1, auto_cells(n1), S1, s));
    PBR_TRY(index_points(tb, p1, n1, S1, s));

    float *m, *v, *grad;
    int32_t *nn12, *nn21;
    double *hist;
    const int iters = cfg->iters;
    PBR_TRY(tb.alloc(&m, sizeof(float) * 3 * n2));
    PBR_TRY(tb.alloc(&v, sizeof(float) * 3 * n2));
    PBR_TRY(tb.alloc(&grad, sizeof(float) * 3 * n2));
    PBR_TRY(tb.alloc(&nn12, sizeof(int32_t) * n1));
    PBR_TRY(tb.alloc(&nn21, sizeof(int32_t) * n2));
    PBR_TRY(tb.alloc(&hist, sizeof(double) * (iters + 1)));
    PBR_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * 3 * n2, s));
    PBR_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * 3 * n2, s));
    PBR_CUDA(cudaMemsetAsync(hist, 0, sizeof(double) * (iters + 1), s));

    // Adam descent of the new positions on the Chamfer distance; the loss
    // before each step, and after the last, goes to the history.  One step
    // (index of the moving cloud, both nearest-point searches, CD and its
    // gradient, Adam) has the same shape every time, so it is captured once
    // as a CUDA graph on a private stream and replayed; Adam's step number
    // and rate live in device memory.
    if (iters > 0) PBR_TRY(descend(tb, p1, n1, S1, pos2, n2, *cfg, grad, m, v, nn12, nn21, hist, s));
    {
        TempBufs it(s);
        PBR_TRY(nearest_maps(it, p1, n1, S1, pos2, n2, nn12, nn21, s));
        launch_chamfer(p1, n1, pos2, n2, nn12, nn21, nullptr, hist + iters, s);
    }

    // parameters: means over the k closest points of the previous frame
    const int k = cfg->k, keff = (int)std::min<int64_t>(k, n1);
    int32_t *idx;
    float *d2;
    PBR_TRY(tb.alloc(&idx, sizeof(int32_t) * k * n2));
    PBR_TRY(tb.alloc(&d2, sizeof(float) * k * n2));
    PBR_TRY(run_knn(tb, pos2, n2, p1, n1, S1, k, keff, 0, idx, d2, s));
    launch_generate(idx, n2, k, keff, PointArrays{p1, prev->sh, prev->opacity, prev->radius, nsh},
                    PointArraysOut{nullptr, sh2, opacity2, radius2, nsh}, 0, s, 3);
    if (loss_history)
        PBR_CUDA(cudaMemcpyAsync(loss_history, hist, sizeof(double) * (iters + 1),
                                 cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaGetLastError());
    PBR_CUDA(cudaStreamSynchronize(s));
    return PBR_OK;
}
