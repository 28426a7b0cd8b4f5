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
// the parameters, compensated fp32 sums in ascending input index.
//
// kNN: one warp per query; lane j holds the j-th best (d2, index) so far,
// d2 = (dx dx + dy dy) + dz dz in fp32 round-to-nearest, ties by lower
// index.  The search visits cubic shells of cells around the query's cell,
// r = r0, r0 + 1, ...; shell r is (2r+1)^2 rows along x (a whole row where
// |dy| or |dz| is r, else the row's two end cells), one row per lane.  The
// points of a run of consecutive cells are a contiguous slice of the
// id-sorted array, read from a dense cell-start table (binary search when
// the grid is too large for one).  Runs of up to 32 points are walked by
// their lanes side by side, longer ones by the whole warp.  Once shell r is
// done every unvisited point lies beyond a face of the visited cube of
// cells, so the search stops when the K-th best d2 is below the squared
// distance to the nearest such face (less a relative slack for the
// roundings of d2 and an absolute one for the cell coordinates), or when
// every cell has been seen.  A query still open after a fixed number of
// shells (neighbours across a wide empty region) is finished by an
// exhaustive scan, one block per query.
//
// Outlier removal: per point, the population standard deviation of its K
// neighbour distances, fp32 sums in neighbour order; survivors are
// compacted in order.  Generation: one warp per survivor averages its K
// nearest survivors' parameters (compensated fp32 sums in neighbour order); the same
// kernel, from attribute 3 on, moves parameters between frames.
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

// Compensated (Kahan) fp32 sum, every operation rounded to nearest (no
// contraction): the error stays within a few ulps of the total whatever the
// number of terms, with fp32 arithmetic only.
struct KahanSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

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
        const float cnt = (float)(e - b);
        for (int a = lane; a < nattr; a += 32) {
            KahanSum acc;
            for (uint32_t m = b; m < e; ++m) acc.add(in.get(__ldg(order + m), a));
            out.put(r, a, __fdiv_rn(acc.s, cnt));
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

// Cells between coordinate c and the grid [0, n-1] along one axis.
__device__ __forceinline__ int axis_gap(int c, int n)
{
    if (c < 0) return -c;
    return c > n - 1 ? c - (n - 1) : 0;
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

// Index range [s, t) of the points in cells [a, b] (consecutive ids) of
// the sorted list: from the dense cell-start table when there is one, else
// by binary search for s and a galloping search for t.
__device__ __forceinline__ void cell_range(const uint32_t *__restrict__ cs,
                                           const uint32_t *__restrict__ rid, uint32_t nr,
                                           uint32_t a, uint32_t b, uint32_t &s, uint32_t &t)
{
    if (cs) {
        s = __ldg(cs + a);
        t = __ldg(cs + b + 1);
        return;
    }
    s = lower_bound_u32(rid, nr, a);
    if (s >= nr || __ldg(rid + s) > b) {
        t = s;
        return;
    }
    uint32_t lo = s, step = 1, hi = s + 1; // rid[lo] <= b
    while (hi < nr && __ldg(rid + hi) <= b) {
        lo = hi;
        step <<= 1;
        hi = s + step;
    }
    if (hi > nr) hi = nr;
    while (hi - lo > 1) { // rid[lo] <= b, hi == nr or rid[hi] > b
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(rid + mid) <= b) lo = mid;
        else hi = mid;
    }
    t = hi;
}

// Candidate j of the sorted list against the query: squared distance and
// whether it would enter the current list.
__device__ __forceinline__ bool knn_candidate(uint32_t j, const uint32_t *__restrict__ ridx,
                                              const float *__restrict__ rpos, float qx, float qy,
                                              float qz, uint32_t self_idx, float kd, uint32_t ki,
                                              float &d2, uint32_t &ri)
{
    ri = __ldg(ridx + j);
    if (ri == self_idx) return false;
    d2 = sq_dist(qx, qy, qz, __ldg(rpos + 3 * (size_t)ri), __ldg(rpos + 3 * (size_t)ri + 1),
                 __ldg(rpos + 3 * (size_t)ri + 2));
    return d2 < kd || (d2 == kd && ri < ki);
}

// Inserts the candidates of the lanes set in m, lowest lane first.
__device__ __forceinline__ void knn_insert_all(uint32_t m, float d2, uint32_t ri, float &bd,
                                               uint32_t &bi, int keff, uint32_t kmask, int lane,
                                               float &kd, uint32_t &ki)
{
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float cd = __shfl_sync(FULL, d2, src);
        const uint32_t cj = __shfl_sync(FULL, ri, src);
        knn_insert(bd, bi, cd, cj, keff, kmask, lane, kd, ki);
    }
}

// Lower bound on the distance from the query to any point of a cell
// outside the cube of cells [c - r, c + r] (per axis), counting only faces
// with grid cells beyond them; FLT_MAX when the cube covers the grid.  The
// slack covers the rounding of cell coordinates and face positions.
__device__ __forceinline__ float unvisited_bound(const GridParams &g, int r, int cx, int cy,
                                                 int cz, float qx, float qy, float qz)
{
    const int c[3] = {cx, cy, cz};
    const float q[3] = {qx, qy, qz};
    float bound = FLT_MAX;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] - r > 0)
            bound = fminf(bound, q[a] - (g.lo[a] + (float)(c[a] - r) * g.h));
        if (c[a] + r < g.n - 1)
            bound = fminf(bound, (g.lo[a] + (float)(c[a] + r + 1) * g.h) - q[a]);
    }
    return bound == FLT_MAX ? FLT_MAX : bound * 0.99999f - g.slack;
}

// Writes the warp's list (lane j = j-th best) as row q of the output.
__device__ __forceinline__ void knn_write(int64_t q, int k, int keff, int lane, float bd,
                                          uint32_t bi, int32_t *__restrict__ out_idx,
                                          float *__restrict__ out_d2)
{
    if (lane < k) {
        const bool have = lane < keff;
        out_idx[q * k + lane] = have ? (int32_t)bi : -1;
        out_d2[q * k + lane] = have ? bd : FLT_MAX;
    }
}

// Shells searched on one grid before a query moves on (to the coarser grid,
// then to the exhaustive kernel): a query whose neighbours lie across a wide
// empty region would otherwise walk (2r+1)^2 rows per shell alone while the
// rest of the GPU idles.
constexpr int KNN_MAX_SHELLS = 16;

// One warp per query.  Queries are 0..nq-1, or qlist[0..*nq_dev) when qlist
// is set.  self_mode: the queries are the reference points (query q is
// reference q and is skipped; its cell is clamped like theirs).  Queries
// still open after KNN_MAX_SHELLS shells are appended to `defer` (count in
// *n_defer) and their rows left unwritten.
__global__ void __launch_bounds__(256)
knn_kernel(const float *__restrict__ qpos, int64_t nq_all, const uint32_t *__restrict__ qlist,
           const uint32_t *__restrict__ nq_dev, const float *__restrict__ rpos, uint32_t nr,
           KnnGrid grid, int k, int keff, int self_mode, int32_t *__restrict__ out_idx,
           float *__restrict__ out_d2, uint32_t *__restrict__ defer, uint32_t *__restrict__ n_defer)
{
    const GridParams g = *grid.gp;
    const uint32_t *__restrict__ rid = grid.rid;
    const uint32_t *__restrict__ ridx = grid.ridx;
    const uint32_t *__restrict__ cs = grid.cs;
    const int lane = threadIdx.x & 31;
    const int n = g.n;
    const uint32_t kmask = keff >= 32 ? FULL : ((1u << keff) - 1u);
    const int64_t nq = qlist ? (int64_t)*nq_dev : nq_all;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nq;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = qlist ? (int64_t)qlist[t] : t;
        const float qx = qpos[3 * q], qy = qpos[3 * q + 1], qz = qpos[3 * q + 2];
        const uint32_t self_idx = self_mode ? (uint32_t)q : 0xffffffffu;
        float bd = FLT_MAX, kd = FLT_MAX;
        uint32_t bi = 0xffffffffu, ki = 0xffffffffu;
        bool keff_done = true;
        if (keff > 0) {
            const int cx = cell_coord(qx, g.lo[0], g.h, n, self_mode);
            const int cy = cell_coord(qy, g.lo[1], g.h, n, self_mode);
            const int cz = cell_coord(qz, g.lo[2], g.h, n, self_mode);
            // first shell that meets the grid
            const int r0 = max(axis_gap(cx, n), max(axis_gap(cy, n), axis_gap(cz, n)));
            for (int r = r0;; ++r) {
                // rows (dy, dz) of shell r that meet the grid
                const int dy0 = max(-r, -cy), dy1 = min(r, n - 1 - cy);
                const int dz0 = max(-r, -cz), dz1 = min(r, n - 1 - cz);
                const int ny = dy1 - dy0 + 1;
                const int rows = ny * (dz1 - dz0 + 1);
                for (int base = 0; base < rows; base += 32) {
                    // this lane's row: up to two index ranges of the sorted list
                    const int row = base + lane;
                    uint32_t s0 = 0, t0 = 0, s1 = 0, t1 = 0;
                    if (row < rows) {
                        const int dy = dy0 + row % ny, dz = dz0 + row / ny;
                        const uint32_t rb =
                            ((uint32_t)(cz + dz) * (uint32_t)n + (uint32_t)(cy + dy)) * (uint32_t)n;
                        if (abs(dy) == r || abs(dz) == r) {
                            const int x0 = max(cx - r, 0), x1 = min(cx + r, n - 1);
                            if (x0 <= x1)
                                cell_range(cs, rid, nr, rb + (uint32_t)x0, rb + (uint32_t)x1, s0, t0);
                        } else {
                            if (cx - r >= 0 && cx - r < n)
                                cell_range(cs, rid, nr, rb + (uint32_t)(cx - r),
                                           rb + (uint32_t)(cx - r), s0, t0);
                            if (cx + r >= 0 && cx + r < n)
                                cell_range(cs, rid, nr, rb + (uint32_t)(cx + r),
                                           rb + (uint32_t)(cx + r), s1, t1);
                        }
                    }
                    // runs longer than a warp: the whole warp, 32 points a step
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const uint32_t st = part ? s1 : s0, en = part ? t1 : t0;
                        uint32_t m = __ballot_sync(FULL, en - st > 32u);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1;
                            const uint32_t rs = __shfl_sync(FULL, st, src);
                            const uint32_t re = __shfl_sync(FULL, en, src);
                            for (uint32_t j0 = rs; j0 < re; j0 += 32) {
                                const uint32_t j = j0 + lane;
                                float d2 = FLT_MAX;
                                uint32_t ri = 0;
                                const bool better = j < re && knn_candidate(j, ridx, rpos, qx, qy, qz,
                                                                            self_idx, kd, ki, d2, ri);
                                knn_insert_all(__ballot_sync(FULL, better), d2, ri, bd, bi, keff,
                                               kmask, lane, kd, ki);
                            }
                        }
                    }
                    // short runs: every lane walks its own, one point a step
                    if (t0 - s0 > 32u) s0 = t0;
                    if (t1 - s1 > 32u) s1 = t1;
                    while (true) {
                        const bool has = s0 < t0 || s1 < t1;
                        if (!__any_sync(FULL, has)) break;
                        float d2 = FLT_MAX;
                        uint32_t ri = 0;
                        bool better = false;
                        if (has) {
                            const uint32_t j = s0 < t0 ? s0++ : s1++;
                            better = knn_candidate(j, ridx, rpos, qx, qy, qz, self_idx, kd, ki, d2, ri);
                        }
                        knn_insert_all(__ballot_sync(FULL, better), d2, ri, bd, bi, keff, kmask,
                                       lane, kd, ki);
                    }
                }
                const float bound = unvisited_bound(g, r, cx, cy, cz, qx, qy, qz);
                if (bound == FLT_MAX) break; // every cell visited
                if (kd < FLT_MAX && bound > 0.0f && kd < __fmul_rn(bound, bound)) break;
                if (r - r0 + 1 >= KNN_MAX_SHELLS) {
                    if (lane == 0) defer[atomicAdd(n_defer, 1u)] = (uint32_t)q;
                    keff_done = false;
                    break;
                }
            }
        }
        if (keff_done) knn_write(q, k, keff, lane, bd, bi, out_idx, out_d2);
    }
}

// Deferred queries, one block each: its 8 warps scan every reference point
// (warp w takes points w*32 + lane, w*32 + lane + 256, ...) into their own
// lists, which warp 0 then merges.  Exact, like the grid search.
__global__ void __launch_bounds__(256)
knn_exhaustive_kernel(const float *__restrict__ qpos, const float *__restrict__ rpos, uint32_t nr,
                      int k, int keff, int self_mode, const uint32_t *__restrict__ defer,
                      const uint32_t *__restrict__ n_defer, int32_t *__restrict__ out_idx,
                      float *__restrict__ out_d2)
{
    __shared__ float s_d[8][32];
    __shared__ uint32_t s_i[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t kmask = keff >= 32 ? FULL : ((1u << keff) - 1u);
    const uint32_t nd = *n_defer;
    for (uint32_t t = blockIdx.x; t < nd; t += gridDim.x) {
        const uint32_t q = defer[t];
        const float qx = qpos[3 * (size_t)q], qy = qpos[3 * (size_t)q + 1],
                    qz = qpos[3 * (size_t)q + 2];
        const uint32_t self_idx = self_mode ? q : 0xffffffffu;
        float bd = FLT_MAX, kd = FLT_MAX;
        uint32_t bi = 0xffffffffu, ki = 0xffffffffu;
        for (uint32_t j0 = (uint32_t)w * 32; j0 < nr; j0 += 256) {
            const uint32_t j = j0 + lane;
            float d2 = FLT_MAX;
            bool better = false;
            if (j < nr && j != self_idx) {
                d2 = sq_dist(qx, qy, qz, __ldg(rpos + 3 * (size_t)j), __ldg(rpos + 3 * (size_t)j + 1),
                             __ldg(rpos + 3 * (size_t)j + 2));
                better = d2 < kd || (d2 == kd && j < ki);
            }
            knn_insert_all(__ballot_sync(FULL, better), d2, j, bd, bi, keff, kmask, lane, kd, ki);
        }
        s_d[w][lane] = bd;
        s_i[w][lane] = bi;
        __syncthreads();
        if (w == 0) {
            for (int v = 1; v < 8; ++v) {
                const float d2 = s_d[v][lane];
                const uint32_t ri = s_i[v][lane];
                const bool better = lane < keff && (d2 < kd || (d2 == kd && ri < ki));
                knn_insert_all(__ballot_sync(FULL, better), d2, ri, bd, bi, keff, kmask, lane, kd,
                               ki);
            }
            knn_write(q, k, keff, lane, bd, bi, out_idx, out_d2);
        }
        __syncthreads();
    }
}

__global__ void cell_count_kernel(const uint32_t *__restrict__ rid, int64_t n,
                                  uint32_t *__restrict__ count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(count + rid[i], 1u);
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
                OutParams out, int64_t out_base, int a_begin)
{
    const int lane = threadIdx.x & 31;
    const int nattr = 5 + in.nsh;
    const float cnt = (float)keff;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t *row = nbr + q * k;
        for (int a = a_begin + lane; a < nattr; a += 32) {
            KahanSum acc;
            for (int j = 0; j < keff; ++j) acc.add(in.get((uint32_t)__ldg(row + j), a));
            out.put(out_base + q, a, __fdiv_rn(acc.s, cnt));
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

size_t knn_temp_bytes(int64_t nq) { return sizeof(uint32_t) * (size_t)(2 * nq + 2); }

void launch_knn(const float *qpos, int64_t nq, const float *rpos, int64_t nr, const KnnGrid &fine,
                const KnnGrid *coarse, int k, int keff, int self_mode, int32_t *out_idx,
                float *out_d2, void *temp, cudaStream_t s)
{
    if (nq <= 0) return;
    uint32_t *cnt = (uint32_t *)temp, *d1 = cnt + 2, *d2 = d1 + nq;
    cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), s);
    knn_kernel<<<grid_for(nq, 8, MAX_BLOCKS), 256, 0, s>>>(qpos, nq, nullptr, nullptr, rpos,
                                                          (uint32_t)nr, fine, k, keff, self_mode,
                                                          out_idx, out_d2, d1, cnt);
    const uint32_t *last = d1, *n_last = cnt;
    if (coarse) {
        knn_kernel<<<grid_for(nq, 8, 152 * 8), 256, 0, s>>>(qpos, 0, d1, cnt, rpos, (uint32_t)nr,
                                                          *coarse, k, keff, self_mode, out_idx,
                                                          out_d2, d2, cnt + 1);
        last = d2;
        n_last = cnt + 1;
        count_launches(1);
    }
    knn_exhaustive_kernel<<<304, 256, 0, s>>>(qpos, rpos, (uint32_t)nr, k, keff, self_mode, last,
                                              n_last, out_idx, out_d2);
    count_launches(2);
}

void launch_cell_start(const uint32_t *rid, int64_t n, int64_t n_cells_total,
                       uint32_t *cell_start, void *scan_temp, cudaStream_t s)
{
    cudaMemsetAsync(cell_start, 0, sizeof(uint32_t) * (size_t)(n_cells_total + 1), s);
    if (n > 0) {
        cell_count_kernel<<<grid_for(n, 256, MAX_BLOCKS), 256, 0, s>>>(rid, n, cell_start);
        count_launches(1);
    }
    launch_exclusive_scan(cell_start, cell_start, n_cells_total + 1, nullptr, scan_temp, s);
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
                     const PointArraysOut &out, int64_t out_base, cudaStream_t s, int a_begin)
{
    if (n <= 0 || keff <= 0) return;
    generate_kernel<<<grid_for(n, 8, MAX_BLOCKS), 256, 0, s>>>(
        nbr, n, k, keff, Params{in.pos, in.sh, in.op, in.rad, in.nsh},
        OutParams{out.pos, out.sh, out.op, out.rad, out.nsh}, out_base, a_begin);
    count_launches(1);
}

} // namespace pbr
