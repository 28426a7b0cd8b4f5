// Hybrid coarse-to-fine update of Sec. 3.3 (Algorithm 1) and the exact grid
// k-nearest-neighbour search it rests on.
//
// Grid: the cube anchored at the per-axis minimum `lo` of a point set, side
// = the largest per-axis extent, split into n^3 cells of side h = side / n.
// Cell of p: floor((p - lo) / h) per axis in fp32 round-to-nearest, clamped
// to [0, n-1] for members of the set; id = (iz n + iy) n + ix.
//
// Voxel reduction: (id, index) pairs are radix-sorted (stable, so a voxel's
// points stay in input order); each run of equal ids becomes one point
// whose parameters are the run's means, one warp per voxel with lanes over
// the parameters, fp64 sums in ascending input index rounded to fp32.
//
// kNN: one warp per query; lane j holds the j-th best (d2, index) so far,
// d2 = (dx dx + dy dy) + dz dz in fp32 round-to-nearest, ties by lower
// index.  The search visits cubic shells of cells around the query's cell,
// r = r0, r0 + 1, ...; shell r is (2r+1)^2 rows along x (a whole row where
// |dy| or |dz| is r, else the row's two end cells).  The points of a run of
// consecutive cells are a contiguous slice of the id-sorted array, found by
// binary search.  Once shell r is done every unvisited point lies more than
// r h away along some axis, so the search stops when the K-th best d2 is
// below (r h)^2, less a relative slack for the roundings of d2 and an
// absolute one for the cell coordinates, or when every cell has been seen.
//
// Outlier removal: per point, the population standard deviation of its K
// neighbour distances, fp32 sums in neighbour order; survivors are
// compacted in order.  Generation: one warp per survivor averages its K
// nearest survivors' parameters (fp64 sums in neighbour order).
#include <cfloat>

#include "pbr_internal.cuh"

namespace pbr {

constexpr int BBOX_PARTS = 608; // partial boxes of the first reduction pass

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BBOX_THREADS = 256;

// Cell coordinate of p along one axis.  Members of the set are clamped into
// [0, n-1]; queries into [-n, 2n-1], which only moves a far query's cell
// towards the grid and so keeps every point of a cell at Chebyshev cell
// distance d > 0 more than (d - 1) h away from the query.
__device__ __forceinline__ int cell_coord(float p, float lo, float h, int n, bool member)
{
    if (h == 0.0f) return 0;
    float t = __fdiv_rn(__fsub_rn(p, lo), h);
    t = fminf(fmaxf(t, -1.0e9f), 1.0e9f); // keeps the conversion in range
    const int c = (int)floorf(t);
    return member ? min(max(c, 0), n - 1) : min(max(c, -n), 2 * n - 1);
}

__device__ __forceinline__ float sq_dist(float ax, float ay, float az, float bx, float by,
                                         float bz)
{
    const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay), dz = __fsub_rn(bz, az);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ------------------------------------------------------------------ grid
__global__ void __launch_bounds__(BBOX_THREADS)
bbox_partial_kernel(const float *__restrict__ pos, int64_t n, float *__restrict__ part)
{
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = pos[3 * i + a];
            mn[a] = fminf(mn[a], v);
            mx[a] = fmaxf(mx[a], v);
        }
    }
    __shared__ float s_v[6][BBOX_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(FULL, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(FULL, mx[a], o));
        }
        if (lane == 0) {
            s_v[a][w] = mn[a];
            s_v[3 + a][w] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        float r = s_v[a][0];
        for (int j = 1; j < BBOX_THREADS / 32; ++j)
            r = a < 3 ? fminf(r, s_v[a][j]) : fmaxf(r, s_v[a][j]);
        part[6 * blockIdx.x + a] = r;
    }
}

__global__ void grid_params_kernel(const float *__restrict__ part, int n_parts, int n_cells,
                                   GridParams *gp)
{
    if (threadIdx.x != 0) return;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int b = 0; b < n_parts; ++b)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], part[6 * b + a]);
            hi[a] = fmaxf(hi[a], part[6 * b + 3 + a]);
        }
    float side = 0.0f, amax = 0.0f;
    for (int a = 0; a < 3; ++a) {
        side = fmaxf(side, __fsub_rn(hi[a], lo[a]));
        amax = fmaxf(amax, fmaxf(fabsf(lo[a]), fabsf(hi[a])));
        gp->lo[a] = lo[a];
    }
    gp->n = n_cells;
    gp->h = __fdiv_rn(side, (float)n_cells);
    // a coordinate's cell can be off across a boundary by the rounding of
    // (p - lo) / h: a few ulps of the coordinates' magnitude
    gp->slack = 4.0e-6f * (side + amax);
}

__global__ void cell_ids_kernel(const float *__restrict__ pos, int64_t n,
                                const GridParams *__restrict__ gp, uint32_t *__restrict__ keys,
                                uint32_t *__restrict__ vals)
{
    const GridParams g = *gp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = cell_coord(pos[3 * i], g.lo[0], g.h, g.n, true);
        const int iy = cell_coord(pos[3 * i + 1], g.lo[1], g.h, g.n, true);
        const int iz = cell_coord(pos[3 * i + 2], g.lo[2], g.h, g.n, true);
        keys[i] = ((uint32_t)iz * (uint32_t)g.n + (uint32_t)iy) * (uint32_t)g.n + (uint32_t)ix;
        vals[i] = (uint32_t)i;
    }
}

// -------------------------------------------------------- voxel runs
__global__ void run_flags_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                 uint32_t *__restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// After the exclusive scan of the flags (pos), each run's first index.
__global__ void run_starts_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pos,
                                  int64_t n, uint32_t *__restrict__ starts)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || keys[i] != keys[i - 1]) starts[pos[i]] = (uint32_t)i;
}

// Parameter `a` of point i: position (a < 3), SH (a < 3 + nsh), opacity,
// radius.
struct Params {
    const float *pos, *sh, *op, *rad;
    int nsh;
    __device__ __forceinline__ float get(uint32_t i, int a) const
    {
        if (a < 3) return pos[3 * (size_t)i + a];
        if (a < 3 + nsh) return sh[(size_t)nsh * i + (a - 3)];
        return a == 3 + nsh ? op[i] : rad[i];
    }
};
struct OutParams {
    float *pos, *sh, *op, *rad;
    int nsh;
    __device__ __forceinline__ void put(int64_t i, int a, float v) const
    {
        if (a < 3) pos[3 * i + a] = v;
        else if (a < 3 + nsh) sh[(int64_t)nsh * i + (a - 3)] = v;
        else if (a == 3 + nsh) op[i] = v;
        else rad[i] = v;
    }
};

__global__ void __launch_bounds__(256)
voxel_mean_kernel(const uint32_t *__restrict__ order, const uint32_t *__restrict__ starts,
                  int64_t n_runs, int64_t n, Params in, OutParams out)
{
    const int lane = threadIdx.x & 31;
    const int nattr = 5 + in.nsh;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_runs;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t b = starts[r];
        const uint32_t e = r + 1 < n_runs ? starts[r + 1] : (uint32_t)n;
        const double cnt = (double)(e - b);
        for (int a = lane; a < nattr; a += 32) {
            double acc = 0.0;
            for (uint32_t m = b; m < e; ++m)
                acc = __dadd_rn(acc, (double)in.get(__ldg(order + m), a));
            out.put(r, a, __double2float_rn(__ddiv_rn(acc, cnt)));
        }
    }
}

// ------------------------------------------------------------------ kNN
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *__restrict__ a, uint32_t n,
                                                    uint32_t key)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Cells between coordinate c and the grid [0, n-1] along one axis, and the
// shell radius that reaches the grid's far end from c.
__device__ __forceinline__ int axis_gap(int c, int n)
{
    if (c < 0) return -c;
    return c > n - 1 ? c - (n - 1) : 0;
}
__device__ __forceinline__ int axis_span(int c, int n)
{
    return c > n - 1 - c ? c : n - 1 - c;
}

// Inserts (cd, cj) into the warp's sorted list (lane j = j-th best, j <
// keff) if it ranks among the first keff; updates the K-th best (kd, ki).
__device__ __forceinline__ void knn_insert(float &bd, uint32_t &bi, float cd, uint32_t cj,
                                           int keff, uint32_t kmask, int lane, float &kd,
                                           uint32_t &ki)
{
    const bool less = bd < cd || (bd == cd && bi < cj);
    const int p = __popc(__ballot_sync(FULL, less) & kmask);
    if (p >= keff) return;
    const float ud = __shfl_up_sync(FULL, bd, 1);
    const uint32_t ui = __shfl_up_sync(FULL, bi, 1);
    if (lane == p) {
        bd = cd;
        bi = cj;
    } else if (lane > p && lane < keff) {
        bd = ud;
        bi = ui;
    }
    kd = __shfl_sync(FULL, bd, keff - 1);
    ki = __shfl_sync(FULL, bi, keff - 1);
}

// Visits the sorted slice of cells with ids [id_lo, id_hi] starting at
// index `start`, 32 points per step.
__device__ __forceinline__ void knn_scan_run(uint32_t start, uint32_t id_hi,
                                             const uint32_t *__restrict__ rid,
                                             const uint32_t *__restrict__ ridx,
                                             const float *__restrict__ rpos, uint32_t nr,
                                             float qx, float qy, float qz, uint32_t self_idx,
                                             int keff, uint32_t kmask, int lane, float &bd,
                                             uint32_t &bi, float &kd, uint32_t &ki)
{
    for (uint32_t j0 = start;; j0 += 32) {
        const uint32_t j = j0 + lane;
        const bool in_run = j < nr && __ldg(rid + j) <= id_hi;
        uint32_t ri = 0;
        float d2 = FLT_MAX;
        bool ok = false;
        if (in_run) {
            ri = __ldg(ridx + j);
            ok = ri != self_idx;
            if (ok) d2 = sq_dist(qx, qy, qz, __ldg(rpos + 3 * (size_t)ri),
                                 __ldg(rpos + 3 * (size_t)ri + 1), __ldg(rpos + 3 * (size_t)ri + 2));
        }
        const bool better = ok && (d2 < kd || (d2 == kd && ri < ki));
        uint32_t m = __ballot_sync(FULL, better);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const float cd = __shfl_sync(FULL, d2, src);
            const uint32_t cj = __shfl_sync(FULL, ri, src);
            knn_insert(bd, bi, cd, cj, keff, kmask, lane, kd, ki);
        }
        if (!__all_sync(FULL, in_run)) break;
    }
}

// One warp per query.  self_mode: the queries are the reference points
// (query q is reference q and is skipped; its cell is clamped like theirs).
__global__ void __launch_bounds__(256)
knn_kernel(const float *__restrict__ qpos, int64_t nq, const float *__restrict__ rpos,
           const uint32_t *__restrict__ rid, const uint32_t *__restrict__ ridx, uint32_t nr,
           const GridParams *__restrict__ gp, int k, int keff, int self_mode,
           int32_t *__restrict__ out_idx, float *__restrict__ out_d2)
{
    const GridParams g = *gp;
    const int lane = threadIdx.x & 31;
    const int n = g.n;
    const uint32_t kmask = keff >= 32 ? FULL : ((1u << keff) - 1u);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const float qx = qpos[3 * q], qy = qpos[3 * q + 1], qz = qpos[3 * q + 2];
        const uint32_t self_idx = self_mode ? (uint32_t)q : 0xffffffffu;
        float bd = FLT_MAX, kd = FLT_MAX;
        uint32_t bi = 0xffffffffu, ki = 0xffffffffu;
        if (keff > 0) {
            const int cx = cell_coord(qx, g.lo[0], g.h, n, self_mode);
            const int cy = cell_coord(qy, g.lo[1], g.h, n, self_mode);
            const int cz = cell_coord(qz, g.lo[2], g.h, n, self_mode);
            // first shell that meets the grid, last shell needed to cover it
            const int r0 = max(axis_gap(cx, n), max(axis_gap(cy, n), axis_gap(cz, n)));
            const int rmax = max(axis_span(cx, n), max(axis_span(cy, n), axis_span(cz, n)));
            for (int r = r0;; ++r) {
                // rows (dy, dz) of shell r that meet the grid
                const int dy0 = max(-r, -cy), dy1 = min(r, n - 1 - cy);
                const int dz0 = max(-r, -cz), dz1 = min(r, n - 1 - cz);
                const int ny = dy1 - dy0 + 1;
                const int rows = ny * (dz1 - dz0 + 1);
                for (int base = 0; base < rows; base += 32) {
                    // this lane's row: up to two runs of cells
                    const int row = base + lane;
                    uint32_t s0 = 0xffffffffu, e0 = 0, s1 = 0xffffffffu, e1 = 0;
                    if (row < rows) {
                        const int dy = dy0 + row % ny, dz = dz0 + row / ny;
                        const int yy = cy + dy, zz = cz + dz;
                        {
                            const uint32_t rb = ((uint32_t)zz * (uint32_t)n + (uint32_t)yy) *
                                                (uint32_t)n;
                            if (abs(dy) == r || abs(dz) == r) {
                                const int x0 = max(cx - r, 0), x1 = min(cx + r, n - 1);
                                if (x0 <= x1) {
                                    e0 = rb + (uint32_t)x1;
                                    s0 = lower_bound_u32(rid, nr, rb + (uint32_t)x0);
                                }
                            } else {
                                if (cx - r >= 0 && cx - r < n) {
                                    e0 = rb + (uint32_t)(cx - r);
                                    s0 = lower_bound_u32(rid, nr, e0);
                                }
                                if (cx + r >= 0 && cx + r < n) {
                                    e1 = rb + (uint32_t)(cx + r);
                                    s1 = lower_bound_u32(rid, nr, e1);
                                }
                            }
                            // empty runs (the first id at or after the run's
                            // start is past its end) are dropped here
                            if (s0 < nr && __ldg(rid + s0) > e0) s0 = 0xffffffffu;
                            if (s1 < nr && __ldg(rid + s1) > e1) s1 = 0xffffffffu;
                        }
                    }
                    for (int part = 0; part < 2; ++part) {
                        const uint32_t st = part ? s1 : s0, en = part ? e1 : e0;
                        uint32_t m = __ballot_sync(FULL, st < nr);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1;
                            const uint32_t s_run = __shfl_sync(FULL, st, src);
                            const uint32_t e_run = __shfl_sync(FULL, en, src);
                            knn_scan_run(s_run, e_run, rid, ridx, rpos, nr, qx, qy, qz, self_idx,
                                         keff, kmask, lane, bd, bi, kd, ki);
                        }
                    }
                }
                if (r >= rmax) break;
                if (kd < FLT_MAX) {
                    const float bound = __fsub_rn(__fmul_rn((float)r * g.h, 0.99999f), g.slack);
                    if (bound > 0.0f && kd < __fmul_rn(bound, bound)) break;
                }
            }
        }
        if (lane < k) {
            const bool have = lane < keff;
            out_idx[q * k + lane] = have ? (int32_t)bi : -1;
            out_d2[q * k + lane] = have ? bd : FLT_MAX;
        }
    }
}

// ---------------------------------------------------------- outliers
__global__ void outlier_flags_kernel(const float *__restrict__ d2, int64_t n, int k, int keff,
                                     float eps, uint32_t *__restrict__ keep)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (keff == 0) {
            keep[i] = 1u;
            continue;
        }
        const float *row = d2 + i * k;
        float s = 0.0f;
        for (int j = 0; j < keff; ++j) s = __fadd_rn(s, __fsqrt_rn(row[j]));
        const float mean = __fdiv_rn(s, (float)keff);
        float t = 0.0f;
        for (int j = 0; j < keff; ++j) {
            const float e = __fsub_rn(__fsqrt_rn(row[j]), mean);
            t = __fadd_rn(t, __fmul_rn(e, e));
        }
        const float delta = __fsqrt_rn(__fdiv_rn(t, (float)keff));
        keep[i] = delta > eps ? 0u : 1u;
    }
}

// Copies kept points to their compacted slots (pos = exclusive scan of keep).
__global__ void __launch_bounds__(256)
compact_points_kernel(const uint32_t *__restrict__ keep, const uint32_t *__restrict__ pos,
                      int64_t n, Params in, OutParams out)
{
    const int lane = threadIdx.x & 31;
    const int nattr = 5 + in.nsh;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (!keep[i]) continue;
        const int64_t o = pos[i];
        for (int a = lane; a < nattr; a += 32) out.put(o, a, in.get((uint32_t)i, a));
    }
}

// The sorted (cell id, index) list restricted to kept points, indices
// renumbered: flags[j] = keep[idx[j]] first, then the scatter.
__global__ void list_keep_kernel(const uint32_t *__restrict__ ridx, const uint32_t *__restrict__ keep,
                                 int64_t n, uint32_t *__restrict__ flags)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        flags[j] = keep[ridx[j]];
}

__global__ void list_compact_kernel(const uint32_t *__restrict__ rid, const uint32_t *__restrict__ ridx,
                                    const uint32_t *__restrict__ keep,
                                    const uint32_t *__restrict__ newpos,
                                    const uint32_t *__restrict__ lpos, int64_t n,
                                    uint32_t *__restrict__ rid_out, uint32_t *__restrict__ ridx_out)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = ridx[j];
        if (keep[i]) {
            rid_out[lpos[j]] = rid[j];
            ridx_out[lpos[j]] = newpos[i];
        }
    }
}

__global__ void fill_u32_kernel(uint32_t *__restrict__ p, int64_t n, uint32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------- generation
__global__ void __launch_bounds__(256)
generate_kernel(const int32_t *__restrict__ nbr, int64_t n, int k, int keff, Params in,
                OutParams out, int64_t out_base)
{
    const int lane = threadIdx.x & 31;
    const int nattr = 5 + in.nsh;
    const double cnt = (double)keff;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t *row = nbr + q * k;
        for (int a = lane; a < nattr; a += 32) {
            double acc = 0.0;
            for (int j = 0; j < keff; ++j)
                acc = __dadd_rn(acc, (double)in.get((uint32_t)__ldg(row + j), a));
            out.put(out_base + q, a, __double2float_rn(__ddiv_rn(acc, cnt)));
        }
    }
}

unsigned grid_for(int64_t items, int per_block, int max_blocks)
{
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

constexpr int MAX_BLOCKS = 152 * 32;

} // namespace

size_t grid_temp_bytes() { return sizeof(float) * 6 * BBOX_PARTS; }

void launch_grid_params(const float *pos, int64_t n, int n_cells, GridParams *gp, void *temp,
                        cudaStream_t s)
{
    float *part = (float *)temp;
    const unsigned blocks = grid_for(n, BBOX_THREADS, BBOX_PARTS);
    bbox_partial_kernel<<<blocks, BBOX_THREADS, 0, s>>>(pos, n, part);
    grid_params_kernel<<<1, 32, 0, s>>>(part, (int)blocks, n_cells, gp);
    count_launches(2);
}

void launch_cell_ids(const float *pos, int64_t n, const GridParams *gp, uint32_t *keys,
                     uint32_t *vals, cudaStream_t s)
{
    if (n <= 0) return;
    cell_ids_kernel<<<grid_for(n, 256, MAX_BLOCKS), 256, 0, s>>>(pos, n, gp, keys, vals);
    count_launches(1);
}

void launch_run_starts(const uint32_t *keys, int64_t n, uint32_t *flags, uint32_t *starts,
                       unsigned long long *n_runs, void *scan_temp, cudaStream_t s)
{
    if (n <= 0) return;
    const unsigned g = grid_for(n, 256, MAX_BLOCKS);
    run_flags_kernel<<<g, 256, 0, s>>>(keys, n, flags);
    launch_exclusive_scan(flags, flags, n, n_runs, scan_temp, s);
    run_starts_kernel<<<g, 256, 0, s>>>(keys, flags, n, starts);
    count_launches(2);
}

void launch_voxel_mean(const uint32_t *order, const uint32_t *starts, int64_t n_runs, int64_t n,
                       const PointArrays &in, const PointArraysOut &out, cudaStream_t s)
{
    if (n_runs <= 0) return;
    voxel_mean_kernel<<<grid_for(n_runs, 8, MAX_BLOCKS), 256, 0, s>>>(
        order, starts, n_runs, n, Params{in.pos, in.sh, in.op, in.rad, in.nsh},
        OutParams{out.pos, out.sh, out.op, out.rad, out.nsh});
    count_launches(1);
}

void launch_knn(const float *qpos, int64_t nq, const float *rpos, const uint32_t *rid,
                const uint32_t *ridx, int64_t nr, const GridParams *gp, int k, int keff,
                int self_mode, int32_t *out_idx, float *out_d2, cudaStream_t s)
{
    if (nq <= 0) return;
    knn_kernel<<<grid_for(nq, 8, MAX_BLOCKS), 256, 0, s>>>(qpos, nq, rpos, rid, ridx, (uint32_t)nr,
                                                          gp, k, keff, self_mode, out_idx, out_d2);
    count_launches(1);
}

void launch_outlier_flags(const float *d2, int64_t n, int k, int keff, float eps, uint32_t *keep,
                          cudaStream_t s)
{
    if (n <= 0) return;
    outlier_flags_kernel<<<grid_for(n, 256, MAX_BLOCKS), 256, 0, s>>>(d2, n, k, keff, eps, keep);
    count_launches(1);
}

void launch_compact_points(const uint32_t *keep, const uint32_t *pos, int64_t n,
                           const PointArrays &in, const PointArraysOut &out, cudaStream_t s)
{
    if (n <= 0) return;
    compact_points_kernel<<<grid_for(n, 8, MAX_BLOCKS), 256, 0, s>>>(
        keep, pos, n, Params{in.pos, in.sh, in.op, in.rad, in.nsh},
        OutParams{out.pos, out.sh, out.op, out.rad, out.nsh});
    count_launches(1);
}

void launch_list_keep(const uint32_t *rid, const uint32_t *ridx, const uint32_t *keep,
                      const uint32_t *newpos, int64_t n, uint32_t *flags, uint32_t *rid_out,
                      uint32_t *ridx_out, void *scan_temp, cudaStream_t s)
{
    if (n <= 0) return;
    const unsigned g = grid_for(n, 256, MAX_BLOCKS);
    list_keep_kernel<<<g, 256, 0, s>>>(ridx, keep, n, flags);
    launch_exclusive_scan(flags, flags, n, nullptr, scan_temp, s);
    list_compact_kernel<<<g, 256, 0, s>>>(rid, ridx, keep, newpos, flags, n, rid_out, ridx_out);
    count_launches(2);
}

void launch_fill_u32(uint32_t *p, int64_t n, uint32_t v, cudaStream_t s)
{
    if (n <= 0) return;
    fill_u32_kernel<<<grid_for(n, 256, MAX_BLOCKS), 256, 0, s>>>(p, n, v);
    count_launches(1);
}

void launch_generate(const int32_t *nbr, int64_t n, int k, int keff, const PointArrays &in,
                     const PointArraysOut &out, int64_t out_base, cudaStream_t s)
{
    if (n <= 0 || keff <= 0) return;
    generate_kernel<<<grid_for(n, 8, MAX_BLOCKS), 256, 0, s>>>(
        nbr, n, k, keff, Params{in.pos, in.sh, in.op, in.rad, in.nsh},
        OutParams{out.pos, out.sh, out.op, out.rad, out.nsh}, out_base);
    count_launches(1);
}

} // namespace pbr
