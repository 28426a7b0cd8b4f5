// pbr_render_forward_noalloc: the forward pass of pbr_render_forward for
// callers that cannot allocate device memory -- for example code that runs
// under an allocator it does not own (a host application's pool that
// forbids cudaMalloc/cudaMallocAsync from plug-ins), or real-time loops that
// must not touch the allocator after start-up.  Every intermediate buffer
// of the pass (layout tables, per point-view records, sort buffers, tile
// ranges, scan and radix scratch) is carved out of one file-scope device
// array of NOALLOC_SCRATCH_BYTES; the caller passes only the inputs (points,
// cameras) and the output image.  Nothing here calls cudaMalloc, cudaFree,
// cudaMallocAsync or any allocating library routine.
//
// The array is a static __device__ object, so every GPU that loads the
// library holds it until the process exits.  Host code must not use the
// symbol itself (on the host it is only a stand-in); the device address is
// looked up once per device with cudaGetSymbolAddress on the first call
// made with that device current -- that first call should therefore come
// before any stream capture.  All calls share the array and it keeps the
// last call's contents: counters and tile ranges are cleared on every call,
// and calls whose GPU work overlaps (different streams, or other host
// threads) race on it.
#include <mutex>

#include "api_internal.h"

using namespace pbr;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20; // 16 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.
int noalloc_scratch(void **out)
{
    int dev = -1;
    PBR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(PBR_ERR_INVALID_ARG, "device %d beyond the supported range", dev);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(PBR_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                             cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PBR_OK;
}

// Bump allocator over the scratch array (256-byte aligned pieces).  `need`
// keeps growing past the end, so one failed piece fails every later one and
// `need` ends as the total size the pass would have required.
struct Carver {
    char *base;
    size_t cap;
    size_t need = 0;
    template <class T> T *take(size_t bytes)
    {
        const size_t at = (need + 255) & ~(size_t)255;
        need = at + (bytes ? bytes : 16);
        return need <= cap ? (T *)(base + at) : nullptr;
    }
    bool fits() const { return need <= cap; }
};

} // namespace

extern "C" int pbr_render_forward_noalloc(const pbr_points *scenes, int32_t n_scenes,
                                          const int32_t *scene_of_view, const pbr_camera *cams,
                                          int32_t n_cams, const pbr_render_opts *opts,
                                          float *out_rgb, pbr_stream_t stream)
{
    PBR_TRY(check_opts(opts));
    if (!out_rgb) return set_error(PBR_ERR_INVALID_ARG, "out_rgb is NULL");
    HostLayout L;
    PBR_TRY(build_layout(scenes, n_scenes, scene_of_view, cams, n_cams, opts, L));
    void *scratch = nullptr;
    PBR_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const DevOpts o = dev_opts(opts);
    const int64_t npv = L.n_pv;

    // phase 1: everything whose size is known before the per-point stage
    Carver cv{(char *)scratch, NOALLOC_SCRATCH_BYTES};
    DevView *d_views = cv.take<DevView>(sizeof(DevView) * L.views.size());
    DevScene *d_scenes = cv.take<DevScene>(sizeof(DevScene) * L.scenes.size());
    int32_t *d_view_list = cv.take<int32_t>(sizeof(int32_t) * L.view_list.size());
    unsigned long long *counters = cv.take<unsigned long long>(128);
    float4 *rec = cv.take<float4>(sizeof(float4) * 2 * npv);
    uint32_t *ntiles = cv.take<uint32_t>(sizeof(uint32_t) * npv);
    uint32_t *zbits = cv.take<uint32_t>(sizeof(uint32_t) * npv);
    uint4 *rect = cv.take<uint4>(sizeof(uint4) * npv);
    uint8_t *nt8 = cv.take<uint8_t>((size_t)npv);
    uint2 *ranges = cv.take<uint2>(sizeof(uint2) * L.n_tiles);
    float *T_final = cv.take<float>(sizeof(float) * L.n_pix);
    uint32_t *n_contrib = cv.take<uint32_t>(sizeof(uint32_t) * L.n_pix);
    if (!cv.fits())
        return set_error(PBR_ERR_CAPACITY,
                         "pbr_render_forward_noalloc: %lld point-views and %lld pixels need at "
                         "least %zu bytes of scratch; the limit is %zu bytes",
                         (long long)npv, (long long)L.n_pix, cv.need, NOALLOC_SCRATCH_BYTES);
    PBR_CUDA(cudaMemcpyAsync(d_views, L.views.data(), sizeof(DevView) * L.views.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(d_scenes, L.scenes.data(), sizeof(DevScene) * L.scenes.size(),
                             cudaMemcpyHostToDevice, s));
    PBR_CUDA(cudaMemcpyAsync(d_view_list, L.view_list.data(), sizeof(int32_t) * L.view_list.size(),
                             cudaMemcpyHostToDevice, s));
    Batch b;
    b.views = d_views;
    b.scenes = d_scenes;
    b.view_list = d_view_list;
    b.n_views = (int32_t)L.views.size();
    b.n_scenes = (int32_t)L.scenes.size();
    b.n_pv = npv;
    b.n_tiles = L.n_tiles;
    b.n_pix = L.n_pix;
    b.n_point_blocks = L.n_point_blocks;
    PBR_CUDA(cudaMemsetAsync(counters, 0, 128, s));
    launch_preprocess_fwd(b, o, rec, zbits, ntiles, nt8, rect, counters, s);
    PBR_CUDA(cudaGetLastError());
    unsigned long long host_counts[2] = {0, 0};
    PBR_CUDA(cudaMemcpyAsync(host_counts, counters, sizeof host_counts, cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    const uint64_t n_pairs = host_counts[0], n_vis = host_counts[1];

    // phase 2: the list buffers, sized by the counts
    const int64_t cap_sort = n_vis > n_pairs ? (int64_t)n_vis : (int64_t)n_pairs;
    size_t temp_bytes = scan_temp_bytes(npv);
    if (radix_temp_bytes(cap_sort) > temp_bytes) temp_bytes = radix_temp_bytes(cap_sort);
    if (emit_temp_bytes((int64_t)n_vis) > temp_bytes) temp_bytes = emit_temp_bytes((int64_t)n_vis);
    uint32_t *vk = cv.take<uint32_t>(4 * n_vis), *vv = cv.take<uint32_t>(4 * n_vis);
    uint32_t *vk2 = cv.take<uint32_t>(4 * n_vis), *vv2 = cv.take<uint32_t>(4 * n_vis);
    uint32_t *tk = cv.take<uint32_t>(4 * n_pairs), *tv = cv.take<uint32_t>(4 * n_pairs);
    uint32_t *pk2 = cv.take<uint32_t>(4 * n_pairs), *pv2 = cv.take<uint32_t>(4 * n_pairs);
    void *temp = cv.take<void>(temp_bytes);
    if (!cv.fits() || n_pairs >= UINT32_MAX)
        return set_error(PBR_ERR_CAPACITY,
                         "pbr_render_forward_noalloc: %llu (tile, point-view) pairs need %zu bytes "
                         "of scratch; the limit is %zu bytes",
                         (unsigned long long)n_pairs, cv.need, NOALLOC_SCRATCH_BYTES);
    uint32_t *status = (uint32_t *)((char *)counters + 64);
    const uint32_t *n_vis_dev = (const uint32_t *)(counters + 1);
    const uint32_t *n_pairs_dev = (const uint32_t *)(counters + 0);
    launch_compact_visible(ntiles, zbits, npv, vk, vv, nullptr, temp, s);
    radix_sort_pairs(vk, vv, vk2, vv2, n_vis_dev, (int64_t)n_vis, 32, temp, s);
    launch_emit_pairs(b, o, vv, n_vis_dev, (int64_t)n_vis, ntiles, nt8, rect, tk, tv,
                      (int64_t)n_pairs, status, temp, s);
    int key_bits = 1;
    while (key_bits < 32 && ((L.n_tiles - 1) >> key_bits)) ++key_bits;
    const int sb = block_bits(o.tile_w, o.tile_h);
    radix_sort_pairs(tk, tv, pk2, pv2, n_pairs_dev, (int64_t)n_pairs, key_bits, temp, s, 0,
                     0xffffffffu, false, sb);
    PBR_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * L.n_tiles, s));
    launch_tile_ranges(tk, n_pairs_dev, (int64_t)n_pairs, ranges, L.n_tiles, sb, s);
    launch_raster_fwd(b, o, opts->batch_depth, ranges, tk, tv, rec, out_rgb, T_final, n_contrib,
                      nullptr, s);
    PBR_CUDA(cudaGetLastError());
    // the kernels' status word (pair overflow, inconsistent counts): one
    // read-back into a host variable after the pass
    uint32_t dev_status = 0;
    PBR_CUDA(cudaMemcpyAsync(&dev_status, status, sizeof dev_status, cudaMemcpyDeviceToHost, s));
    PBR_CUDA(cudaStreamSynchronize(s));
    if (dev_status)
        return set_error(PBR_ERR_DEVICE_STATUS,
                         "pbr_render_forward_noalloc: device status 0x%x", dev_status);
    return PBR_OK;
}
