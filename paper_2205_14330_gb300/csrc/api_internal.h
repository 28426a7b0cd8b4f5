// Host-side objects behind the opaque handles of pbr.h.
#pragma once

#include <array>
#include <cstdarg>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "pbr.h"
#include "pbr_internal.cuh"

struct ServeState; // serving loop (serve.cu)

struct pbr_ctx {
    int device = 0;
    int sm_count = 0;
    size_t hbm_budget = 0;
    unsigned long long *host_counters = nullptr; // pinned
    ServeState *serve = nullptr;
    // optional per-stage CUDA-event timing
    std::mutex timing_mu;
    bool timing = false;
    struct StageRec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<StageRec> pending;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[pbr::STG_COUNT] = {};
    long long stage_calls[pbr::STG_COUNT] = {};
    // autotuner cache: shape class -> {tile_w, tile_h, batch_depth, persistent}
    std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>, std::array<int, 4>> tuned;
};

namespace pbr {

struct HostLayout {
    std::vector<DevView> views;
    std::vector<DevScene> scenes;
    std::vector<int32_t> view_list;
    int64_t n_pv = 0, n_pix = 0, n_point_blocks = 0;
    int64_t n_points_total = 0, n_sh_total = 0;
    uint32_t n_tiles = 0;
};

int set_error(int code, const char *fmt, ...);
int check_opts(const pbr_render_opts *o);
DevOpts dev_opts(const pbr_render_opts *o);
int build_layout(const pbr_points *scenes, int32_t n_scenes, const int32_t *scene_of_view,
                 const pbr_camera *cams, int32_t n_cams, const pbr_render_opts *o, HostLayout &L);
// Device bytes a forward pass allocates for a layout with n_vis visible
// point-views and n_pairs (tile, point-view) pairs (store_depth > 0: with
// the stored transmittance list).
size_t forward_bytes(const HostLayout &L, int64_t n_vis, int64_t n_pairs,
                     const pbr_render_opts *o, int32_t store_depth);
// Zeroes the gradient slices of the scenes that no view of the layout sees
// (the point backward runs over the points of viewed scenes only).
void zero_unviewed_grads(const HostLayout &L, float *grad_pos, float *grad_sh,
                         float *grad_opacity, cudaStream_t s);
int dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
void serve_shutdown(pbr_ctx *c);

} // namespace pbr

struct pbr_state {
    cudaStream_t stream = nullptr;
    pbr_render_opts opts{};
    pbr::DevOpts dopts{};
    int batch_depth = 256;
    pbr::HostLayout layout;
    int64_t n_vis = 0, n_pairs = 0;
    // device buffers kept for the backward pass (all freed by release())
    pbr::DevView *d_views = nullptr;
    pbr::DevScene *d_scenes = nullptr;
    int32_t *d_view_list = nullptr;
    float4 *rec = nullptr;
    uint32_t *ntiles = nullptr;
    // [0] pairs, [1] visible, [2..3] raster-fwd examined/composited pairs,
    // [4..5] raster-bwd examined/contributing pairs; byte 64: status word
    unsigned long long *counters = nullptr;
    uint32_t *tile_keys = nullptr, *tile_vals = nullptr;
    uint2 *ranges = nullptr;
    float *T_final = nullptr;
    uint32_t *n_contrib = nullptr;
    uint4 *tile_order = nullptr; // persistent raster: tile descriptors, longest list first
    uint32_t *work = nullptr;       // persistent raster: item counters + buckets
    // store mode (bwd_mode): T before the first store_depth composited points
    // of every pixel, and the points composited per pixel
    int32_t store_depth = 0;
    float *T_store = nullptr;
    uint32_t *n_comp = nullptr;

    pbr::StoreBuf store() const
    {
        pbr::StoreBuf b;
        b.T = T_store;
        b.n = n_comp;
        b.depth = store_depth;
        b.n_pix = layout.n_pix;
        return b;
    }

    pbr::Batch batch() const
    {
        pbr::Batch b;
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
    void release();
};

namespace pbr {
// Temporaries of one call, freed (stream-ordered) when the call returns.
struct TempBufs {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit TempBufs(cudaStream_t st) : s(st) {}
    ~TempBufs()
    {
        for (void *p : ptrs) dfree(p, s);
    }
    template <class T> int alloc(T **p, size_t bytes)
    {
        int rc = dalloc((void **)p, bytes, s);
        if (rc == PBR_OK) ptrs.push_back((void *)*p);
        return rc;
    }
};
} // namespace pbr

namespace pbr {
// ---- exact neighbour search over a point set (api_refine.cu)
// One search grid: device parameters, sorted (cell id, index) list, table.
struct Grid {
    GridParams *gp = nullptr;
    uint32_t *rid = nullptr, *ridx = nullptr, *cs = nullptr;
    int cells = 0;
    KnnGrid view() const { return KnnGrid{gp, rid, ridx, cs}; }
};
// The fine search grid and, for fine grids of 16 cells or more, a second
// one 8 times coarser for queries the fine search leaves open.
struct SearchIndex {
    Grid fine, coarse;
    bool has_coarse = false;
};
// Cells per axis of an automatic grid over n points (about 2 n^(1/3)).
int auto_cells(int64_t n);
// Grid parameters of both levels over the cube of the n points `pos`.
int make_params(TempBufs &tb, const float *pos, int64_t n, int cells, SearchIndex &S,
                cudaStream_t s);
// Sorted lists and tables of both levels for the n reference points.
int index_points(TempBufs &tb, const float *ref, int64_t n, SearchIndex &S, cudaStream_t s);
// Both levels restricted to kept points (indices renumbered by newpos).
int keep_points(TempBufs &tb, SearchIndex &S, int64_t m, int64_t m2, const uint32_t *keep,
                const uint32_t *newpos, void *scan_tmp, cudaStream_t s);
// Exact k nearest reference points of each query (rows of k entries).
int run_knn(TempBufs &tb, const float *q, int64_t nq, const float *ref, int64_t nr,
            const SearchIndex &S, int k, int keff, int self_mode, int32_t *out_idx, float *out_d2,
            cudaStream_t s);

int forward_eager(pbr_ctx *c, pbr_state *st, float *out_rgb, cudaStream_t s);
// Composited points per pixel whose T the forward keeps for the backward:
// 0 = recompute (bwd_mode 1, the block-staged schedule, forward-only calls,
// or auto when the list would take more than an eighth of the HBM budget).
int32_t resolve_store_depth(const pbr_ctx *c, const pbr_render_opts *o, int64_t n_pix,
                            bool keep_state);
// Bytes of the stored transmittance list for store_depth points per pixel.
size_t store_bytes(int32_t store_depth, int64_t n_pix);

// Records CUDA events around one stage on stream s when the context has
// stage timing switched on (pbr_set_stage_timing); otherwise does nothing.
class StageScope {
  public:
    StageScope(pbr_ctx *c, int stage, cudaStream_t s);
    ~StageScope();

  private:
    pbr_ctx *c_;
    int stage_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr;
};
} // namespace pbr

#define PBR_CUDA(x)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            cudaGetLastError();                                                                 \
            return pbr::set_error(PBR_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #x,         \
                                  cudaGetErrorString(e_));                                      \
        }                                                                                       \
    } while (0)

#define PBR_TRY(x)                                                                              \
    do {                                                                                        \
        int r_ = (x);                                                                           \
        if (r_ != PBR_OK) return r_;                                                            \
    } while (0)
