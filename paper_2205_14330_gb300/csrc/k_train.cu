// Training objective and optimiser step of Sec. 3.3.
//
// loss_tv: per view image, L = sum (I_hat - I)^2 (or |I_hat - I|) +
// lambda * TV(I_hat), TV = l1 norm of forward differences along x and y
// per channel (anisotropic, no wrap-around), and dL/dI_hat with
// d|d|/dd = sign(d), sign(0) = 0.  One thread per pixel; each forward
// difference is counted once, by its left / upper pixel.
//
// optimizer: p <- p - lr g (SGD) or the bias-corrected Adam update, with the
// learning rate and the step number read from device memory so a captured
// training step can change them between replays (per-epoch decay).
#include "pbr_internal.cuh"

namespace pbr {

namespace {

__device__ __forceinline__ float sgnf(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void loss_tv_kernel(const DevView *__restrict__ views, int kind, float lam,
                               const float *__restrict__ pred, const float *__restrict__ target,
                               float *__restrict__ grad, double *loss)
{
    const DevView &V = views[blockIdx.y];
    const int64_t npx = (int64_t)V.W * V.H;
    // compensated fp32 per thread, fp64 across threads: no per-element fp64
    float acc = 0.0f, comp = 0.0f;
    auto add = [&](float x) {
        const float y = __fsub_rn(x, comp);
        const float t = __fadd_rn(acc, y);
        comp = __fsub_rn(__fsub_rn(t, acc), y);
        acc = t;
    };
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % V.W), y = (int)(p / V.W);
        const int64_t q = V.pix_base + p;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a = pred[3 * q + c];
            const float d = a - target[3 * q + c];
            float gv;
            if (kind == 0) {
                add(d * d);
                gv = 2.0f * d;
            } else {
                add(fabsf(d));
                gv = sgnf(d);
            }
            if (lam != 0.0f) {
                float tv = 0.0f;
                if (x + 1 < V.W) {
                    const float dx = pred[3 * (q + 1) + c] - a;
                    add(lam * fabsf(dx));
                    tv -= sgnf(dx);
                }
                if (x > 0) tv += sgnf(a - pred[3 * (q - 1) + c]);
                if (y + 1 < V.H) {
                    const float dy = pred[3 * (q + V.W) + c] - a;
                    add(lam * fabsf(dy));
                    tv -= sgnf(dy);
                }
                if (y > 0) tv += sgnf(a - pred[3 * (q - V.W) + c]);
                gv += lam * tv;
            }
            grad[3 * q + c] = gv;
        }
    }
    double tot = (double)acc - (double)comp;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    __shared__ double s_w[32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
        if (t != 0.0) atomicAdd(loss, t);
    }
}

__global__ void optimizer_kernel(OptParams prm, const OptState *__restrict__ dev, int group,
                                 float *__restrict__ p, const float *__restrict__ g,
                                 float *__restrict__ m, float *__restrict__ v, int64_t n)
{
    float lr = prm.lr;
    int t = prm.step;
    if (dev) {
        lr = dev->lr[group];
        t = dev->step;
    }
    if (lr == 0.0f) return;
    const float bc1 = 1.0f - powf(prm.beta1, (float)t), bc2 = 1.0f - powf(prm.beta2, (float)t);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        if (prm.kind == 0) {
            p[i] -= lr * gi;
        } else {
            const float mi = prm.beta1 * m[i] + (1.0f - prm.beta1) * gi;
            const float vi = prm.beta2 * v[i] + (1.0f - prm.beta2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + prm.eps);
        }
    }
}

__global__ void step_counter_kernel(OptState *dev) { dev->step += 1; }

} // namespace

void launch_loss_tv(const DevView *views, int n_views, int64_t max_pix, int kind, float lam,
                    const float *pred, const float *target, float *grad, double *loss,
                    cudaStream_t s)
{
    if (n_views <= 0 || max_pix <= 0) return;
    int64_t bx = (max_pix + 255) / 256;
    if (bx > 4096) bx = 4096;
    loss_tv_kernel<<<dim3((unsigned)bx, (unsigned)n_views), 256, 0, s>>>(views, kind, lam, pred,
                                                                          target, grad, loss);
    count_launches(1);
}

void launch_optimizer(const OptParams &prm, const OptState *dev, int group, float *p,
                      const float *g, float *m, float *v, int64_t n, cudaStream_t s)
{
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    optimizer_kernel<<<(unsigned)blocks, 256, 0, s>>>(prm, dev, group, p, g, m, v, n);
    count_launches(1);
}

void launch_step_counter(OptState *dev, cudaStream_t s)
{
    step_counter_kernel<<<1, 1, 0, s>>>(dev);
    count_launches(1);
}

} // namespace pbr
