// Chamfer distance of Sec. 3.4 (video frame initialisation) and its
// gradient with respect to the positions of the second cloud.
//
//   CD = 1/n1 sum_i |y_nn(i) - x_i|^2 + 1/n2 sum_j |y_j - x_nn(j)|^2
//   dCD/dy_j = 2/n2 (y_j - x_nn(j)) + 2/n1 sum_{i: nn(i) = j} (y_j - x_i)
//
// with the nearest points (from the exact neighbour search) held fixed.
// The distances entering CD are taken in fp64 from the fp32 positions and
// summed per block, one fp64 atomic per block; the second gradient term is
// scattered with fp32 atomics.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ void block_add(double v, double *dst)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
        if (t != 0.0) atomicAdd(dst, t);
    }
}

// Every y_j against its nearest x: writes the first gradient term.
__global__ void __launch_bounds__(256)
chamfer_21_kernel(const float *__restrict__ p1, const float *__restrict__ p2, int64_t n2,
                  const int32_t *__restrict__ nn21, double inv_n2, float *__restrict__ grad2,
                  double *loss)
{
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n2;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = nn21[j];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = (double)p2[3 * j + a] - (double)p1[3 * i + a];
            acc += d * d;
            if (grad2) grad2[3 * j + a] = (float)(2.0 * inv_n2 * d);
        }
    }
    block_add(acc * inv_n2, loss);
}

// Every x_i against its nearest y: adds the second gradient term.
__global__ void __launch_bounds__(256)
chamfer_12_kernel(const float *__restrict__ p1, int64_t n1, const float *__restrict__ p2,
                  const int32_t *__restrict__ nn12, double inv_n1, float *__restrict__ grad2,
                  double *loss)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = nn12[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = (double)p2[3 * j + a] - (double)p1[3 * i + a];
            acc += d * d;
            if (grad2) atomicAdd(grad2 + 3 * j + a, (float)(2.0 * inv_n1 * d));
        }
    }
    block_add(acc * inv_n1, loss);
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

} // namespace

void launch_chamfer(const float *p1, int64_t n1, const float *p2, int64_t n2,
                    const int32_t *nn12, const int32_t *nn21, float *grad2, double *loss,
                    cudaStream_t s)
{
    if (n1 <= 0 || n2 <= 0) return;
    chamfer_21_kernel<<<blocks_for(n2), 256, 0, s>>>(p1, p2, n2, nn21, 1.0 / (double)n2, grad2,
                                                      loss);
    chamfer_12_kernel<<<blocks_for(n1), 256, 0, s>>>(p1, n1, p2, nn12, 1.0 / (double)n1, grad2,
                                                      loss);
    count_launches(2);
}

} // namespace pbr
