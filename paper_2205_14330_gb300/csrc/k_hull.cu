// Visual-hull initialisation and consistency check (Sec. 3.1 and the
// appendix): a point is consistent when its projection (Eq. 1) lands on a
// foreground pixel of every view's mask; the initial cloud is the first
// n_target consistent points of a counter-based uniform stream over the
// scene box, with SH coefficients drawn from N(0, 1).
//
// Projection in fp32 round-to-nearest with the renderer's operation order:
// X = ((R0 px + R1 py) + R2 pz) + t per row, u = fx (X.x / X.z) + cx; pixel
// (floor u, floor v); behind z_near or outside the image = background.
// Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), output i
// of stream s = finaliser of s + (i + 1) * 0x9E3779B97F4A7C15; uniforms are
// the top 24 bits times 2^-24.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform24(uint64_t z)
{
    return (float)(uint32_t)(z >> 40) * 5.9604644775390625e-8f; // 2^-24, exact
}

__device__ bool consistent(float px, float py, float pz, const HullView *__restrict__ views,
                           int nv, const uint8_t *__restrict__ masks, float z_near)
{
    for (int v = 0; v < nv; ++v) {
        const HullView &V = views[v];
        float X[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            X[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.R[3 * r], px),
                                                  __fmul_rn(V.R[3 * r + 1], py)),
                                       __fmul_rn(V.R[3 * r + 2], pz)),
                             V.t[r]);
        if (!(X[2] > z_near)) return false;
        const float u = __fadd_rn(__fmul_rn(V.fx, __fdiv_rn(X[0], X[2])), V.cx);
        const float w = __fadd_rn(__fmul_rn(V.fy, __fdiv_rn(X[1], X[2])), V.cy);
        if (!(u >= 0.0f && w >= 0.0f && u < (float)V.W && w < (float)V.H)) return false;
        const int64_t x = (int64_t)floorf(u), y = (int64_t)floorf(w);
        if (__ldg(masks + V.pix_base + y * V.W + x) == 0) return false;
    }
    return true;
}

__global__ void __launch_bounds__(256)
cc_flags_kernel(const float *__restrict__ pos, int64_t n, const HullView *__restrict__ views,
                int nv, const uint8_t *__restrict__ masks, float z_near,
                uint8_t *__restrict__ flags8, uint32_t *__restrict__ flags32)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = consistent(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], views, nv, masks,
                                   z_near);
        if (flags8) flags8[i] = ok ? 1 : 0;
        if (flags32) flags32[i] = ok ? 1u : 0u;
    }
}

// Candidates first .. first + count - 1: position and consistency flag.
__global__ void __launch_bounds__(256)
hull_candidates_kernel(uint64_t seed, uint64_t first, int64_t count, float lo0, float lo1,
                       float lo2, float ex0, float ex1, float ex2,
                       const HullView *__restrict__ views, int nv,
                       const uint8_t *__restrict__ masks, float z_near, float *__restrict__ cand,
                       uint32_t *__restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t j = first + (uint64_t)i;
        const float x = __fadd_rn(__fmul_rn(ex0, uniform24(splitmix64(seed, 3 * j))), lo0);
        const float y = __fadd_rn(__fmul_rn(ex1, uniform24(splitmix64(seed, 3 * j + 1))), lo1);
        const float z = __fadd_rn(__fmul_rn(ex2, uniform24(splitmix64(seed, 3 * j + 2))), lo2);
        cand[3 * i] = x;
        cand[3 * i + 1] = y;
        cand[3 * i + 2] = z;
        flags[i] = consistent(x, y, z, views, nv, masks, z_near) ? 1u : 0u;
    }
}

// Accepted candidates of rank < need go to out[done + rank]; the candidate
// of rank need - 1 reports its index.
__global__ void hull_take_kernel(const float *__restrict__ cand, const uint32_t *__restrict__ flags,
                                 const uint32_t *__restrict__ rank, int64_t count, uint32_t need,
                                 float *__restrict__ out, int64_t done,
                                 unsigned long long *last)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        const uint32_t k = rank[i];
        if (k >= need) continue;
        const int64_t o = done + k;
        out[3 * o] = cand[3 * i];
        out[3 * o + 1] = cand[3 * i + 1];
        out[3 * o + 2] = cand[3 * i + 2];
        if (k == need - 1) *last = (unsigned long long)i;
    }
}

// Standard normals for coefficients [c0, c0 + count) of the flattened
// [points, coefficients] array, Box-Muller on stream seed: pair p = c / 2
// uses outputs 2p and 2p + 1.  fp32 (logf, sincospif): no decision depends
// on these values, and fp64 transcendentals run at a small fraction of the
// fp32 rate on this GPU.  u1 and u2 are exact in fp32 (24-bit integers times
// 2^-24).
__global__ void sh_normals_kernel(uint64_t seed, int64_t c0, int64_t count,
                                  float *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = (uint64_t)(c0 + i), p = c >> 1;
        const float u1 = ((float)(uint32_t)(splitmix64(seed, 2 * p) >> 40) + 1.0f) * 0x1p-24f;
        const float u2 = (float)(uint32_t)(splitmix64(seed, 2 * p + 1) >> 40) * 0x1p-24f;
        const float r = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        out[i] = (c & 1) ? r * sn : r * cs;
    }
}

unsigned grid_of(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

} // namespace

void launch_consistency(const float *pos, int64_t n, const HullView *views, int nv,
                        const uint8_t *masks, float z_near, uint8_t *flags8, uint32_t *flags32,
                        cudaStream_t s)
{
    if (n <= 0) return;
    cc_flags_kernel<<<grid_of(n), 256, 0, s>>>(pos, n, views, nv, masks, z_near, flags8, flags32);
    count_launches(1);
}

void launch_hull_candidates(uint64_t seed, uint64_t first, int64_t count, const float lo[3],
                            const float ext[3], const HullView *views, int nv,
                            const uint8_t *masks, float z_near, float *cand, uint32_t *flags,
                            cudaStream_t s)
{
    if (count <= 0) return;
    hull_candidates_kernel<<<grid_of(count), 256, 0, s>>>(seed, first, count, lo[0], lo[1], lo[2],
                                                          ext[0], ext[1], ext[2], views, nv,
                                                          masks, z_near, cand, flags);
    count_launches(1);
}

void launch_hull_take(const float *cand, const uint32_t *flags, const uint32_t *rank,
                      int64_t count, uint32_t need, float *out, int64_t done,
                      unsigned long long *last, cudaStream_t s)
{
    if (count <= 0 || need == 0) return;
    hull_take_kernel<<<grid_of(count), 256, 0, s>>>(cand, flags, rank, count, need, out, done,
                                                     last);
    count_launches(1);
}

void launch_sh_normals(uint64_t seed, int64_t c0, int64_t count, float *out, cudaStream_t s)
{
    if (count <= 0) return;
    sh_normals_kernel<<<grid_of(count), 256, 0, s>>>(seed, c0, count, out);
    count_launches(1);
}

} // namespace pbr
