// Image loss of the training step (Sec. 3.3, Eq. 8 data term; L1 variant)
// and the ALU microbenchmarks that give the raster kernels their roofline.
#include "pbr_internal.cuh"

namespace pbr {

namespace {

// Compensated (Kahan) fp32 running sum: a thread's few hundred terms keep a
// few-ulp error without fp64 arithmetic, which runs at a small fraction of
// the fp32 rate on this GPU.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

__device__ __forceinline__ float loss_term(int kind, float d, float &g)
{
    if (kind == 0) {
        g = 2.0f * d;
        return d * d;
    }
    g = d > 0.f ? 1.0f : (d < 0.f ? -1.0f : 0.0f);
    return fabsf(d);
}

// vec4: all three arrays 16-byte aligned, n4 = n / 4 groups of four.
__global__ void image_loss_kernel(int kind, const float *__restrict__ pred,
                                  const float *__restrict__ target, int64_t n, int vec4,
                                  float *__restrict__ grad, double *loss)
{
    KahanF acc;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec4) {
        const int64_t n4 = n >> 2;
        for (int64_t i = tid; i < n4; i += stride) {
            const float4 p = reinterpret_cast<const float4 *>(pred)[i];
            const float4 t = reinterpret_cast<const float4 *>(target)[i];
            float4 g;
            acc.add(loss_term(kind, p.x - t.x, g.x));
            acc.add(loss_term(kind, p.y - t.y, g.y));
            acc.add(loss_term(kind, p.z - t.z, g.z));
            acc.add(loss_term(kind, p.w - t.w, g.w));
            reinterpret_cast<float4 *>(grad)[i] = g;
        }
        done = n4 << 2;
    }
    for (int64_t i = done + tid; i < n; i += stride) {
        float g;
        acc.add(loss_term(kind, pred[i] - target[i], g));
        grad[i] = g;
    }
    double v = (double)acc.s - (double)acc.c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double s_w[32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
        atomicAdd(loss, t);
    }
}

constexpr int MB_CHAINS = 8;

__global__ void fma_peak_kernel(float *out, int iters, float a, float b)
{
    float x[MB_CHAINS];
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < MB_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) s += x[c];
    if (s == 1234.5f) out[0] = s; // keeps the chains alive
}

__global__ void ex2_peak_kernel(float *out, int iters)
{
    float x[MB_CHAINS];
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) x[c] = -1e-3f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < MB_CHAINS; ++c) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
            x[c] = -y; // keeps the argument in (-1, 0]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < MB_CHAINS; ++c) s += x[c];
    if (s == 1234.5f) out[0] = s;
}

} // namespace

void launch_image_loss(int kind, const float *pred, const float *target, int64_t n, float *grad,
                       double *loss, cudaStream_t s)
{
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const int vec4 = (((uintptr_t)pred | (uintptr_t)target | (uintptr_t)grad) & 15u) == 0;
    image_loss_kernel<<<(unsigned)blocks, 256, 0, s>>>(kind, pred, target, n, vec4, grad, loss);
    count_launches(1);
}

int measure_alu_peaks(int device, double *fp32_flops, double *ex2_ops)
{
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    float *out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8, iters = 1 << 14;
    float best_fma = 1e30f, best_ex2 = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        fma_peak_kernel<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_fma) best_fma = ms;
        cudaEventRecord(e0);
        ex2_peak_kernel<<<blocks, threads>>>(out, iters / 4);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ex2) best_ex2 = ms;
    }
    const double n_thr = (double)blocks * threads;
    if (fp32_flops) *fp32_flops = n_thr * iters * MB_CHAINS * 2.0 / (best_fma * 1e-3);
    if (ex2_ops) *ex2_ops = n_thr * (iters / 4) * MB_CHAINS / (best_ex2 * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

} // namespace pbr
