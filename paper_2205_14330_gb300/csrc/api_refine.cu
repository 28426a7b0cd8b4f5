// C entry points of the coarse-to-fine update (Sec. 3.3, Algorithm 1) and
// of the k-nearest-neighbour search.
#include <algorithm>
#include <cmath>

#include "api_internal.h"

using namespace pbr;

namespace {

int key_bits_of(int n_cells)
{
    const uint64_t cells = (uint64_t)n_cells * n_cells * n_cells;
    int b = 0;
    while (b < 32 && ((cells - 1) >> b)) ++b;
    return b;
}

int read_count(const unsigned long long *dev, int64_t *out, cudaStream_t s)
{
    unsigned long long v = 0;
    PBR_CUDA(cudaMemcpyAsync(&v, dev, sizeof(v), cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    *out = (int64_t)v;
    return PBR_OK;
}

// Grids up to this many cells get a dense cell-start table (4 bytes a cell).
constexpr int64_t MAX_TABLE_CELLS = 1ll << 28;

// Sorted (cell id, index) list of n points on grid gp; ends in (*keys, *vals).
// With `table` set, also the dense cell-start table of grids small enough
// for one (else *table = NULL).
int sorted_cells(TempBufs &tb, const float *pos, int64_t n, const GridParams *gp, int n_cells,
                 uint32_t **keys, uint32_t **vals, cudaStream_t s, uint32_t **table = nullptr)
{
    uint32_t *k0, *v0, *k1, *v1;
    void *tmp;
    PBR_TRY(tb.alloc(&k0, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&v0, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&k1, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&v1, sizeof(uint32_t) * n));
    PBR_TRY(tb.alloc(&tmp, radix_temp_bytes(n)));
    launch_cell_ids(pos, n, gp, k0, v0, s);
    radix_sort_pairs(k0, v0, k1, v1, nullptr, n, key_bits_of(n_cells), tmp, s);
    *keys = k0;
    *vals = v0;
    if (table) {
        *table = nullptr;
        const int64_t cells = (int64_t)n_cells * n_cells * n_cells;
        if (cells <= MAX_TABLE_CELLS) {
            void *stmp;
            PBR_TRY(tb.alloc(table, sizeof(uint32_t) * (cells + 1)));
            PBR_TRY(tb.alloc(&stmp, scan_temp_bytes(cells + 1)));
            launch_cell_start(k0, n, cells, *table, stmp, s);
        }
    }
    return PBR_OK;
}

} // namespace

int pbr::auto_cells(int64_t n)
{
    const double c = 2.0 * std::cbrt((double)std::max<int64_t>(n, 1));
    return (int)std::min(1024.0, std::max(1.0, std::ceil(c)));
}

// Parameters of both levels over the cube of the n points `pos`.
int pbr::make_params(TempBufs &tb, const float *pos, int64_t n, int cells, SearchIndex &S,
                cudaStream_t s)
{
    void *gtmp;
    PBR_TRY(tb.alloc(&S.fine.gp, sizeof(GridParams)));
    PBR_TRY(tb.alloc(&gtmp, grid_temp_bytes()));
    S.fine.cells = cells;
    S.has_coarse = cells >= 16 && n > 0;
    if (n <= 0) return PBR_OK;
    launch_grid_params(pos, n, cells, S.fine.gp, gtmp, s);
    if (S.has_coarse) {
        PBR_TRY(tb.alloc(&S.coarse.gp, sizeof(GridParams)));
        S.coarse.cells = (cells + 7) / 8;
        launch_grid_params(pos, n, S.coarse.cells, S.coarse.gp, gtmp, s);
    }
    return PBR_OK;
}

// Sorted lists and tables of both levels for the n reference points.
int pbr::index_points(TempBufs &tb, const float *ref, int64_t n, SearchIndex &S, cudaStream_t s)
{
    if (n <= 0) return PBR_OK;
    PBR_TRY(sorted_cells(tb, ref, n, S.fine.gp, S.fine.cells, &S.fine.rid, &S.fine.ridx, s,
                         &S.fine.cs));
    if (S.has_coarse)
        PBR_TRY(sorted_cells(tb, ref, n, S.coarse.gp, S.coarse.cells, &S.coarse.rid,
                             &S.coarse.ridx, s, &S.coarse.cs));
    return PBR_OK;
}

// Both levels restricted to the kept points (indices renumbered by newpos,
// the exclusive scan of keep), tables rebuilt in place.
int pbr::keep_points(TempBufs &tb, SearchIndex &S, int64_t m, int64_t m2, const uint32_t *keep,
                const uint32_t *newpos, void *scan_tmp, cudaStream_t s)
{
    uint32_t *flags;
    PBR_TRY(tb.alloc(&flags, sizeof(uint32_t) * m));
    for (int level = 0; level < (S.has_coarse ? 2 : 1); ++level) {
        Grid &G = level ? S.coarse : S.fine;
        uint32_t *sid, *sidx;
        PBR_TRY(tb.alloc(&sid, sizeof(uint32_t) * m2));
        PBR_TRY(tb.alloc(&sidx, sizeof(uint32_t) * m2));
        launch_list_keep(G.rid, G.ridx, keep, newpos, m, flags, sid, sidx, scan_tmp, s);
        G.rid = sid;
        G.ridx = sidx;
        if (G.cs) {
            void *ctmp;
            const int64_t cells = (int64_t)G.cells * G.cells * G.cells;
            PBR_TRY(tb.alloc(&ctmp, scan_temp_bytes(cells + 1)));
            launch_cell_start(sid, m2, cells, G.cs, ctmp, s);
        }
    }
    return PBR_OK;
}

int pbr::run_knn(TempBufs &tb, const float *q, int64_t nq, const float *ref, int64_t nr,
            const SearchIndex &S, int k, int keff, int self_mode, int32_t *out_idx, float *out_d2,
            cudaStream_t s)
{
    void *ktmp;
    PBR_TRY(tb.alloc(&ktmp, knn_temp_bytes(nq)));
    const KnnGrid fine = S.fine.view(), coarse = S.coarse.view();
    launch_knn(q, nq, ref, nr, fine, S.has_coarse ? &coarse : nullptr, k, keff, self_mode,
               out_idx, out_d2, ktmp, s);
    return PBR_OK;
}

extern "C" void pbr_default_refine(pbr_refine_cfg *cfg)
{
    if (!cfg) return;
    cfg->n_vox = 256;
    cfg->k = 8;
    cfg->eps = 0.01f;
    cfg->stages = 7;
}

extern "C" int pbr_knn(pbr_ctx *ctx, const float *ref_pos, int64_t n_ref, const float *query_pos,
                       int64_t n_query, int32_t k, int32_t self, int32_t grid_n, int32_t *out_idx,
                       float *out_d2, pbr_stream_t stream)
{
    if (!ctx || n_ref < 0 || n_ref > 0x7fffffffLL || k < 1 || k > 32 || grid_n < 0 ||
        grid_n > 1024 || (n_ref > 0 && !ref_pos))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_knn: bad arguments");
    if (self) {
        query_pos = ref_pos;
        n_query = n_ref;
    }
    if (n_query < 0 || (n_query > 0 && (!query_pos || !out_idx || !out_d2)))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_knn: bad query arguments");
    if (n_query == 0) return PBR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    const int64_t avail = self ? n_ref - 1 : n_ref;
    const int keff = (int)std::max<int64_t>(0, std::min<int64_t>(k, avail));
    TempBufs tb(s);
    SearchIndex S;
    PBR_TRY(make_params(tb, ref_pos, n_ref, grid_n > 0 ? grid_n : auto_cells(n_ref), S, s));
    PBR_TRY(index_points(tb, ref_pos, n_ref, S, s));
    PBR_TRY(run_knn(tb, query_pos, n_query, ref_pos, n_ref, S, k, keff, self ? 1 : 0, out_idx,
                    out_d2, s));
    PBR_CUDA(cudaGetLastError());
    return PBR_OK;
}

extern "C" int pbr_refine_points(pbr_ctx *ctx, const pbr_points *in, const pbr_refine_cfg *cfg,
                                 float *out_pos, float *out_sh, float *out_opacity,
                                 float *out_radius, int64_t out_capacity, int64_t counts[3],
                                 pbr_stream_t stream)
{
    if (!ctx || !in || !cfg || !counts)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_refine_points: null argument");
    counts[0] = counts[1] = counts[2] = 0;
    const int64_t n = in->n;
    if (n < 0 || n > 0x7fffffffLL || in->sh_degree < 0 || in->sh_degree > 3 ||
        cfg->n_vox < 1 || cfg->n_vox > 1024 || cfg->k < 1 || cfg->k > 32 ||
        !(cfg->eps >= 0.0f) || std::isinf(cfg->eps) || cfg->stages < 0 || cfg->stages > 7)
        return set_error(PBR_ERR_INVALID_ARG, "pbr_refine_points: bad configuration");
    if (n > 0 && (!in->pos || !in->sh || !in->opacity || !in->radius || !out_pos || !out_sh ||
                  !out_opacity || !out_radius))
        return set_error(PBR_ERR_INVALID_ARG, "pbr_refine_points: null array");
    if (n == 0) return PBR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PBR_CUDA(cudaSetDevice(ctx->device));
    const int nsh = 3 * (in->sh_degree + 1) * (in->sh_degree + 1);
    const int N = cfg->n_vox, k = cfg->k;
    TempBufs tb(s);

    // the voxel grid (fine search level) and a coarser search level, both
    // over the cube of the input positions
    SearchIndex S;
    void *stmp;
    unsigned long long *tot;
    PBR_TRY(tb.alloc(&stmp, scan_temp_bytes(n)));
    PBR_TRY(tb.alloc(&tot, sizeof(unsigned long long)));
    {
        StageScope sc(ctx, STG_REFINE_OTHER, s);
        PBR_TRY(make_params(tb, in->pos, n, N, S, s));
    }

    // stage 1: voxel reduction into the reduced set R
    PointArrays R{in->pos, in->sh, in->opacity, in->radius, nsh};
    int64_t m = n;
    if (cfg->stages & 1) {
        StageScope sc(ctx, STG_VOXEL_REDUCE, s);
        uint32_t *keys, *vals, *flags, *starts;
        PBR_TRY(sorted_cells(tb, in->pos, n, S.fine.gp, N, &keys, &vals, s));
        PBR_TRY(tb.alloc(&flags, sizeof(uint32_t) * n));
        PBR_TRY(tb.alloc(&starts, sizeof(uint32_t) * n));
        launch_run_starts(keys, n, flags, starts, tot, stmp, s);
        PBR_TRY(read_count(tot, &m, s));
        float *rp, *rs, *ro, *rr;
        PBR_TRY(tb.alloc(&rp, sizeof(float) * 3 * m));
        PBR_TRY(tb.alloc(&rs, sizeof(float) * nsh * m));
        PBR_TRY(tb.alloc(&ro, sizeof(float) * m));
        PBR_TRY(tb.alloc(&rr, sizeof(float) * m));
        launch_voxel_mean(vals, starts, m, n, R, PointArraysOut{rp, rs, ro, rr, nsh}, s);
        R = PointArrays{rp, rs, ro, rr, nsh};
    }
    counts[0] = m;

    // the reduced set's search index (neighbours of stages 2 and 3)
    if (cfg->stages & 6) {
        StageScope sc(ctx, STG_KNN, s);
        PBR_TRY(index_points(tb, R.pos, m, S, s));
    }

    // stage 2: outlier flags and survivor positions
    uint32_t *keep, *newpos;
    PBR_TRY(tb.alloc(&keep, sizeof(uint32_t) * m));
    PBR_TRY(tb.alloc(&newpos, sizeof(uint32_t) * m));
    int64_t m2 = m;
    if (cfg->stages & 2) {
        const int keff = (int)std::min<int64_t>(k, m - 1);
        int32_t *nidx;
        float *nd2;
        PBR_TRY(tb.alloc(&nidx, sizeof(int32_t) * k * m));
        PBR_TRY(tb.alloc(&nd2, sizeof(float) * k * m));
        {
            StageScope sc(ctx, STG_KNN, s);
            PBR_TRY(run_knn(tb, R.pos, m, R.pos, m, S, k, keff, 1, nidx, nd2, s));
        }
        StageScope sc(ctx, STG_REFINE_OTHER, s);
        launch_outlier_flags(nd2, m, k, keff, cfg->eps, keep, s);
        launch_exclusive_scan(keep, newpos, m, tot, stmp, s);
        PBR_TRY(read_count(tot, &m2, s));
    } else {
        launch_fill_u32(keep, m, 1u, s);
        launch_exclusive_scan(keep, newpos, m, nullptr, stmp, s);
    }
    const int keff3 =
        (cfg->stages & 4) ? (int)std::max<int64_t>(0, std::min<int64_t>(k, m2 - 1)) : 0;
    const int64_t total = m2 + (keff3 > 0 ? m2 : 0);
    counts[1] = m2;
    counts[2] = total;
    if (total > out_capacity)
        return set_error(PBR_ERR_CAPACITY, "pbr_refine_points: %lld output points, capacity %lld",
                         (long long)total, (long long)out_capacity);
    const PointArraysOut O{out_pos, out_sh, out_opacity, out_radius, nsh};
    {
        StageScope sc(ctx, STG_REFINE_OTHER, s);
        launch_compact_points(keep, newpos, m, R, O, s);
    }

    // stage 3: one new point per survivor from its nearest survivors
    if (keff3 > 0) {
        if ((cfg->stages & 2) && m2 < m) {
            StageScope sc(ctx, STG_REFINE_OTHER, s);
            PBR_TRY(keep_points(tb, S, m, m2, keep, newpos, stmp, s));
        }
        int32_t *nidx;
        float *nd2;
        PBR_TRY(tb.alloc(&nidx, sizeof(int32_t) * k * m2));
        PBR_TRY(tb.alloc(&nd2, sizeof(float) * k * m2));
        {
            StageScope sc(ctx, STG_KNN, s);
            PBR_TRY(run_knn(tb, out_pos, m2, out_pos, m2, S, k, keff3, 1, nidx, nd2, s));
        }
        StageScope sc(ctx, STG_REFINE_OTHER, s);
        launch_generate(nidx, m2, k, keff3,
                        PointArrays{out_pos, out_sh, out_opacity, out_radius, nsh}, O, m2, s);
    }
    PBR_CUDA(cudaGetLastError());
    PBR_CUDA(cudaStreamSynchronize(s));
    return PBR_OK;
}
