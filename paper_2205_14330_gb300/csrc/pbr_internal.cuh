// Internal declarations shared by the CUDA translation units of libpbr.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pbr {

// Status bits raised by kernels (device word, read by the host after a pass).
enum : uint32_t {
    ST_PAIR_OVERFLOW = 1u << 0,  // more (tile, point-view) pairs than capacity
    ST_COUNT_OVERFLOW = 1u << 1, // a 32-bit count or index would overflow
    ST_BAD_RANGE = 1u << 2,      // inconsistent tile range
};

// One view of the batch: camera of Sec. 3.1 Eq. 1 plus its place in the
// packed pixel, tile and point-view numbering.
struct DevView {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    uint32_t tile_base;  // first global tile id of the view
    int32_t scene;       // index into the scene table
    int64_t pix_base;    // first pixel of the view in the packed image
    int64_t pv_base;     // first point-view id: pv = pv_base + point index
    float *out;          // when set, the view's RGB goes here ([H,W,3]) instead of the
                         // packed image (serving: one output buffer per request)
};

// One scene (point set) of the batch.
struct DevScene {
    const float *pos;     // [n,3]
    const float *sh;      // [n,K,3]
    const float *opacity; // [n]
    const float *radius;  // [n]
    int64_t n;
    int32_t K, deg;
    int32_t view_begin, view_count; // slice of the scene-sorted view list
    int64_t point_base;             // offset of the scene in packed gradients
    int64_t sh_base;                // offset (floats) in the packed SH gradient
    int64_t block_begin;            // first block of the point-parallel grids
};

// Renderer constants in device form.
struct DevOpts {
    int32_t radius_mode, dir_frame;
    float cutoff_k, alpha_max, t_eps;
    int32_t max_per_pixel;
    float bg[3];
    float z_near;
    int32_t tile_w, tile_h;
};

// Everything a launch needs about the batch layout (passed by value).
struct Batch {
    const DevView *views;       // [n_views]
    const DevScene *scenes;     // [n_scenes]
    const int32_t *view_list;   // views sorted by scene
    int32_t n_views, n_scenes;
    int64_t n_pv;               // point-views
    uint32_t n_tiles;
    int64_t n_pix;
    int64_t n_point_blocks;     // blocks of the point-parallel grids
};

constexpr int PRE_THREADS = 128;

// Smallest transmittance the compositing continues below (see dev_opts).
constexpr float T_EPS_FLOOR = 1e-30f;

// Stages of a pass, for the optional per-stage CUDA-event timing.
enum Stage : int {
    STG_PREPROCESS_FWD = 0,
    STG_COMPACT,
    STG_DEPTH_SORT,
    STG_EMIT,
    STG_TILE_SORT,
    STG_RANGES,
    STG_RASTER_FWD,
    STG_RASTER_BWD,
    STG_PREPROCESS_BWD,
    STG_OTHER,
    STG_VOXEL_REDUCE, // coarse-to-fine update: voxel reduction
    STG_KNN,          // coarse-to-fine update: neighbour searches
    STG_REFINE_OTHER, // coarse-to-fine update: grid, filter, compaction, generation
    STG_COUNT
};

// Number of kernels this library has launched (process-wide).
void count_launches(int n);
unsigned long long launches_total();

// log2(e) (the kernel exponent is taken base 2: q' = -log2(e) / (2 s^2))
constexpr float LOG2E = 1.4426950408889634f;

// ---- binning rule (Sec. 3.2 cutoff), shared by the per-point stage and the
// pair emission.  A tile lists a point-view iff some pixel of the tile
// (inside the image) passes the per-pixel fp32 cutoff test; each listed
// pair carries the mask of the tile's 8 x 8 pixel blocks holding such a
// pixel (bit by * (tile_w / 8) + bx, row-major inside the tile), stored in
// the low block_bits() bits of its sort key: key = tile << block_bits | mask.

// Mask bits per key: one per 8 x 8 block when a tile holds more than one.
__host__ __device__ constexpr int block_bits(int tile_w, int tile_h)
{
    return (tile_w / 8) * (tile_h / 8) > 1 ? (tile_w / 8) * (tile_h / 8) : 0;
}

// Whether some pixel centre of the pixel rectangle [x0, x1] x [y0, y1]
// (inclusive, non-empty) passes the cutoff test d2 <= rc2 (fp32
// round-to-nearest, d2 = (ux - px)^2 + (uy - py)^2).  Rounding is monotone,
// so the centre nearest the splat centre per axis -- floor(p) + 0.5 clamped
// into the rectangle -- has the smallest fp32 d2: testing it decides for the
// whole rectangle.
__device__ __forceinline__ bool rect_reached(float px, float py, float rc2, int x0, int x1,
                                             int y0, int y1)
{
    const float cx = fminf(fmaxf(__fadd_rn(floorf(px), 0.5f), __fadd_rn((float)x0, 0.5f)),
                           __fadd_rn((float)x1, 0.5f));
    const float cy = fminf(fmaxf(__fadd_rn(floorf(py), 0.5f), __fadd_rn((float)y0, 0.5f)),
                           __fadd_rn((float)y1, 0.5f));
    const float ex = __fsub_rn(cx, px), ey = __fsub_rn(cy, py);
    return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= rc2;
}

// Mask of the 8 x 8 blocks of the TW x TH tile with top-left pixel (ox,
// oy) that hold a pixel passing the cutoff test (blocks clipped to the W x H
// image): rect_reached per block, with the squared x distance computed once
// per block column and the squared y distance once per block row (the same
// operations, so the same decisions).
template <int TW, int TH>
__device__ __forceinline__ uint32_t tile_block_mask(float px, float py, float rc2, int ox, int oy,
                                                    int W, int H)
{
    constexpr int BX = TW / 8, BY = TH / 8;
    const float fx = __fadd_rn(floorf(px), 0.5f), fy = __fadd_rn(floorf(py), 0.5f);
    float ex2[BX], ey2[BY];
#pragma unroll
    for (int bx = 0; bx < BX; ++bx) {
        const int x0 = ox + 8 * bx;
        const float c = fminf(fmaxf(fx, __fadd_rn((float)x0, 0.5f)),
                              __fadd_rn((float)min(x0 + 7, W - 1), 0.5f));
        const float e = __fsub_rn(c, px);
        ex2[bx] = x0 < W ? __fmul_rn(e, e) : __int_as_float(0x7f800000); // +inf: outside
    }
#pragma unroll
    for (int by = 0; by < BY; ++by) {
        const int y0 = oy + 8 * by;
        const float c = fminf(fmaxf(fy, __fadd_rn((float)y0, 0.5f)),
                              __fadd_rn((float)min(y0 + 7, H - 1), 0.5f));
        const float e = __fsub_rn(c, py);
        ey2[by] = y0 < H ? __fmul_rn(e, e) : __int_as_float(0x7f800000);
    }
    uint32_t m = 0;
#pragma unroll
    for (int by = 0; by < BY; ++by)
#pragma unroll
        for (int bx = 0; bx < BX; ++bx)
            if (__fadd_rn(ex2[bx], ey2[by]) <= rc2) m |= 1u << (by * BX + bx);
    return m;
}

// The clamped pixel box of a splat: [floor(px - rc) - 1, ceil(px + rc)] x
// (the same in y), clamped to the image; false when it misses the image.
// Every pixel passing the cutoff test lies inside.
__device__ __forceinline__ bool pixel_box(float px, float py, float rc, int W, int H, int &x0,
                                          int &x1, int &y0, int &y1)
{
    float xlo = __fsub_rn(floorf(__fsub_rn(px, rc)), 1.0f);
    float xhi = ceilf(__fadd_rn(px, rc));
    float ylo = __fsub_rn(floorf(__fsub_rn(py, rc)), 1.0f);
    float yhi = ceilf(__fadd_rn(py, rc));
    const float W1 = (float)(W - 1), H1 = (float)(H - 1);
    if (!(xhi >= 0.0f && xlo <= W1 && yhi >= 0.0f && ylo <= H1)) return false;
    x0 = (int)(xlo < 0.0f ? 0.0f : xlo);
    y0 = (int)(ylo < 0.0f ? 0.0f : ylo);
    x1 = (int)(xhi > W1 ? W1 : xhi);
    y1 = (int)(yhi > H1 ? H1 : yhi);
    return true;
}

// ---- preprocess (k_preprocess.cu)
// counters[0] += (tile, point-view) pairs, counters[1] += visible point-views;
// 32-bit words 12 / 13 of counters: min / max depth bits of visible
// point-views (word 12 must start at 0xffffffff, word 13 at 0).
// zbits[pv] = fp32 bits of the depth, 0xffffffff for a point-view listing no
// tile (every finite depth's bits are smaller).
// nt8[pv] = min(tile count, 255): a one-byte copy of the counts, small
// enough to stay in L2 while the emission's count gather reads it.
// rect[pv] = {px, py, rc (fp32 bits), w}: the splat centre and cutoff
// radius (the pixel box follows from them by pixel_box), w = the mask of
// the listed tiles of the box (bit (ty - ty0) * wx + (tx - tx0)) when the
// box spans at most 32 tiles, else the number of listed tiles.
// rec == nullptr: counting only (the counters; nothing else is written).
void launch_preprocess_fwd(const Batch &b, const DevOpts &o, float4 *rec, uint32_t *zbits,
                           uint32_t *ntiles, uint8_t *nt8, uint4 *rect,
                           unsigned long long *counters, cudaStream_t s);
void launch_preprocess_bwd(const Batch &b, const DevOpts &o, const float4 *g2d, float *grad_pos,
                           float *grad_sh, float *grad_opacity, cudaStream_t s);

// ---- scans, sorts and binning (k_sort.cu)
size_t scan_temp_bytes(int64_t n);
// Compacts visible point-views (ntiles > 0): keys_out = z bits, vals_out = pv.
// Writes the visible count to *n_vis (device).
void launch_compact_visible(const uint32_t *ntiles, const uint32_t *zbits, int64_t n_pv,
                            uint32_t *keys_out, uint32_t *vals_out, uint32_t *n_vis, void *temp,
                            cudaStream_t s);
// out[i] = in[0] + ... + in[i-1]; *total (device, may be NULL) = the sum.
// out may alias in.  Scratch: scan_temp_bytes(n).
void launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n,
                           unsigned long long *total, void *temp, cudaStream_t s);
// Radix sort of (key, value) pairs, stable; n read from device *n_dev,
// capacity cap.  key_bits: number of low key bits that can be non-zero.
// Sorted result ends in (keys, vals) (buffers are ping-ponged internally).
// Keys are ordered by min(key - key_lo, key_max) >> bit_lo; key_bits = bits
// of the largest such value.  Digits of up to 9 bits, ceil(key_bits / 9)
// passes.  index_vals: the input values are not read; value i is taken to
// be i.  bit_lo > 0 needs key_lo = 0 and key_max = 0xffffffff.
size_t radix_temp_bytes(int64_t cap);
int radix_passes(int key_bits);
void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *&keys_alt, uint32_t *&vals_alt,
                      const uint32_t *n_dev, int64_t cap, int key_bits, void *temp,
                      cudaStream_t s, uint32_t key_lo = 0, uint32_t key_max = 0xffffffffu,
                      bool index_vals = false, int bit_lo = 0);
// Scratch of launch_emit_pairs (depth-ordered counts, offsets, scan).
size_t emit_temp_bytes(int64_t cap_vis);
// Emits (tile, pv) pairs in depth order: gathers the tile counts in depth
// order, scans them, then writes each warp's runs cooperatively.
// Keys are tile << block_bits(tile size) | block mask.
void launch_emit_pairs(const Batch &b, const DevOpts &o, const uint32_t *sorted_pv,
                       const uint32_t *n_vis, int64_t cap_vis, const uint32_t *ntiles,
                       const uint8_t *nt8,
                       const uint4 *rect, uint32_t *keys, uint32_t *vals, int64_t cap_pairs,
                       uint32_t *status, void *temp, cudaStream_t s);
// Ranges of the tiles key >> shift of the sorted keys.
void launch_tile_ranges(const uint32_t *keys, const uint32_t *n_pairs, int64_t cap_pairs,
                        uint2 *ranges, uint32_t n_tiles, int shift, cudaStream_t s);

// ---- coarse-to-fine update and kNN (k_refine.cu)
// Cube grid over a point set: origin lo, cell side h (0 when all points
// coincide), n cells per axis, absolute slack of the kNN stop test.
struct GridParams {
    float lo[3];
    float h;
    int32_t n;
    float slack;
};
// Per-point parameter arrays: pos [n,3], sh [n,nsh], opacity [n], radius [n].
struct PointArrays {
    const float *pos, *sh, *op, *rad;
    int nsh;
};
struct PointArraysOut {
    float *pos, *sh, *op, *rad;
    int nsh;
};
size_t grid_temp_bytes();
void launch_grid_params(const float *pos, int64_t n, int n_cells, GridParams *gp, void *temp,
                        cudaStream_t s);
// keys = clamped cell ids, vals = 0..n-1
void launch_cell_ids(const float *pos, int64_t n, const GridParams *gp, uint32_t *keys,
                     uint32_t *vals, cudaStream_t s);
// Runs of equal sorted keys: starts[r] = first index of run r, *n_runs.
// flags: n words of scratch; scan_temp: scan_temp_bytes(n).
void launch_run_starts(const uint32_t *keys, int64_t n, uint32_t *flags, uint32_t *starts,
                       unsigned long long *n_runs, void *scan_temp, cudaStream_t s);
void launch_voxel_mean(const uint32_t *order, const uint32_t *starts, int64_t n_runs, int64_t n,
                       const PointArrays &in, const PointArraysOut &out, cudaStream_t s);
// One search grid over the reference points: parameters, (cell id, index)
// list sorted by id, dense cell-start table (or NULL).
struct KnnGrid {
    const GridParams *gp;
    const uint32_t *rid, *ridx, *cs;
};
// Exact K nearest reference points per query; rows of k entries, keff =
// entries filled.  Searches `fine`, then `coarse` (may be NULL) for queries
// left open, then scans every point for what is still open.
// temp: knn_temp_bytes(nq).
size_t knn_temp_bytes(int64_t nq);
void launch_knn(const float *qpos, int64_t nq, const float *rpos, int64_t nr, const KnnGrid &fine,
                const KnnGrid *coarse, int k, int keff, int self_mode, int32_t *out_idx,
                float *out_d2, void *temp, cudaStream_t s);
// cell_start[c] = first index of cell c in the sorted list (c <= cells);
// scan_temp: scan_temp_bytes(cells + 1).
void launch_cell_start(const uint32_t *rid, int64_t n, int64_t n_cells_total,
                       uint32_t *cell_start, void *scan_temp, cudaStream_t s);
void launch_outlier_flags(const float *d2, int64_t n, int k, int keff, float eps, uint32_t *keep,
                          cudaStream_t s);
void launch_compact_points(const uint32_t *keep, const uint32_t *pos, int64_t n,
                           const PointArrays &in, const PointArraysOut &out, cudaStream_t s);
// Restricts a sorted (id, index) list to kept points, renumbering indices
// with newpos (the exclusive scan of keep).  flags: n words of scratch.
void launch_list_keep(const uint32_t *rid, const uint32_t *ridx, const uint32_t *keep,
                      const uint32_t *newpos, int64_t n, uint32_t *flags, uint32_t *rid_out,
                      uint32_t *ridx_out, void *scan_temp, cudaStream_t s);
void launch_fill_u32(uint32_t *p, int64_t n, uint32_t v, cudaStream_t s);
// Row out_base + q of `out` = mean of the parameters of points nbr[q][0..keff)
// of `in`, for parameters a_begin.. (0: position first; 3: SH, opacity,
// radius only).
void launch_generate(const int32_t *nbr, int64_t n, int k, int keff, const PointArrays &in,
                     const PointArraysOut &out, int64_t out_base, cudaStream_t s,
                     int a_begin = 0);

// ---- frame initialisation (k_frame.cu)
// Chamfer distance of two clouds given the nearest-point maps (nn12[i]:
// nearest point of p2 to p1[i]; nn21[j]: nearest of p1 to p2[j]): adds CD to
// *loss (fp64, device) and, when grad2 is set, writes dCD/dp2 ([n2,3]).
void launch_chamfer(const float *p1, int64_t n1, const float *p2, int64_t n2,
                    const int32_t *nn12, const int32_t *nn21, float *grad2, double *loss,
                    cudaStream_t s);

// ---- visual hull and consistency check (k_hull.cu)
// One view of the check: camera of Eq. 1, image size, offset of its mask
// in the packed masks (uint8, [H, W] per view, > 0 = foreground).
struct HullView {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    int32_t W, H;
    int64_t pix_base;
};
// Consistency flag of every point (either output may be NULL).
void launch_consistency(const float *pos, int64_t n, const HullView *views, int nv,
                        const uint8_t *masks, float z_near, uint8_t *flags8, uint32_t *flags32,
                        cudaStream_t s);
// Candidates first .. first + count - 1 of stream `seed` in the box lo +
// [0, ext): positions and flags.
void launch_hull_candidates(uint64_t seed, uint64_t first, int64_t count, const float lo[3],
                            const float ext[3], const HullView *views, int nv,
                            const uint8_t *masks, float z_near, float *cand, uint32_t *flags,
                            cudaStream_t s);
// Accepted candidates of rank (exclusive scan of flags) below `need` to
// out[done + rank]; *last = index of the candidate of rank need - 1.
void launch_hull_take(const float *cand, const uint32_t *flags, const uint32_t *rank,
                      int64_t count, uint32_t need, float *out, int64_t done,
                      unsigned long long *last, cudaStream_t s);
// out[i] = standard normal number c0 + i of stream `seed` (Box-Muller).
void launch_sh_normals(uint64_t seed, int64_t c0, int64_t count, float *out, cudaStream_t s);

// ---- raster (k_raster.cu)
// Store mode (bwd_mode 2): T[k * n_pix + pix] = the transmittance pixel pix
// had before its k-th composited point (k < depth), n[pix] = the points it
// composited.  T == nullptr: recompute mode (the backward recovers T by
// dividing by 1 - alpha back to front).
struct StoreBuf {
    float *T = nullptr;
    uint32_t *n = nullptr;
    int32_t depth = 0;
    int64_t n_pix = 0;
};

// batch_depth 0 = warp-streamed, > 0 = block-staged.  With order/work set
// (warp-streamed only) the launch is persistent: warps pull (tile,
// sub-block) items from work[0] (forward) / work[1] (backward) over `order`.
// keys: the sorted pair keys (their block masks let a warp skip the entries
// none of its pixels can include); pv_list: the sorted point-view ids.
// sto: store mode's buffers (the warp-streamed and persistent schedules;
// the block-staged one always recomputes).
void launch_raster_fwd(const Batch &b, const DevOpts &o, int batch_depth, const uint2 *ranges,
                       const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                       float *out_rgb,
                       float *T_final, uint32_t *n_contrib, unsigned long long *stats,
                       cudaStream_t s, const uint4 *order = nullptr, uint32_t *work = nullptr,
                       const StoreBuf &sto = StoreBuf());
void launch_raster_bwd(const Batch &b, const DevOpts &o, int batch_depth, const uint2 *ranges,
                       const uint32_t *keys, const uint32_t *pv_list, const float4 *rec,
                       const float *T_final,
                       const uint32_t *n_contrib, const float *grad_rgb, float4 *g2d,
                       unsigned long long *stats, cudaStream_t s,
                       const uint4 *order = nullptr, uint32_t *work = nullptr,
                       const StoreBuf &sto = StoreBuf());
// Longest-first tile order for the persistent raster, as tile descriptors
// {view, tx | ty << 16, list start, list end}; work: 34 u32 words.
void launch_tile_order(const Batch &b, const uint2 *ranges, uint32_t n_tiles, uint4 *order,
                       uint32_t *work, cudaStream_t s);
void reset_work_counters(uint32_t *work, cudaStream_t s);

// ---- training step (k_train.cu)
struct OptParams {
    int32_t kind;  // 0 SGD, 1 Adam
    float lr, beta1, beta2, eps;
    int32_t step;  // 1-based Adam step (eager calls)
};
// Device-side rates and step number of a captured training step.
struct OptState {
    float lr[3];   // positions, SH coefficients, opacity
    int32_t step;
};
void launch_loss_tv(const DevView *views, int n_views, int64_t max_pix, int kind, float lam,
                    const float *pred, const float *target, float *grad, double *loss,
                    cudaStream_t s);
void launch_optimizer(const OptParams &prm, const OptState *dev, int group, float *p,
                      const float *g, float *m, float *v, int64_t n, cudaStream_t s);
void launch_step_counter(OptState *dev, cudaStream_t s);

// ---- misc (k_misc.cu)
void launch_image_loss(int kind, const float *pred, const float *target, int64_t n, float *grad,
                       double *loss, cudaStream_t s);
int measure_alu_peaks(int device, double *fp32_flops, double *ex2_ops);

} // namespace pbr
