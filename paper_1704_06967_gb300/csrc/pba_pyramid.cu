// Image pyramid for coarse-to-fine solving (an addition beyond the paper:
// the basin of the direct method widens at coarse levels). One level down
// halves each image dimension; a pixel is the mean of the 2 x 2 block it
// covers, so pixel centres follow x_coarse = (x_fine + 0.5) / 2 - 0.5.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "pba_kernels.cuh"

namespace pba {

namespace {

__global__ void downsample_kernel(const void* __restrict__ src, int dtype, int F, int w, int h, int pitch,
                                  float* __restrict__ dst)
{
    const int w2 = w / 2, h2 = h / 2;
    const size_t total = (size_t)F * h2 * w2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % w2);
        const size_t fy = i / w2;
        const int y = (int)(fy % h2), f = (int)(fy / h2);
        const size_t r0 = ((size_t)f * h + 2 * y) * pitch + 2 * x, r1 = r0 + pitch;
        const float a = load_px(src, dtype, r0), b = load_px(src, dtype, r0 + 1);
        const float c = load_px(src, dtype, r1), d = load_px(src, dtype, r1 + 1);
        dst[i] = 0.25f * ((a + b) + (c + d));
    }
}

}  // namespace

}  // namespace pba

extern "C" pba_status pba_downsample(const void* src, pba_dtype dtype, int n_frames, int w, int h, int pitch_elems,
                                     float* dst, void* cuda_stream)
{
    if (!src || !dst || n_frames < 1 || w < 2 || h < 2 || pitch_elems < w ||
        (dtype != PBA_F32 && dtype != PBA_F16 && dtype != PBA_BF16))
        return PBA_ERR_ARG;
    if ((double)n_frames * h * pitch_elems >= 9.0e18) return PBA_ERR_ARG;
    const size_t total = (size_t)n_frames * (h / 2) * (w / 2);
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
    pba::downsample_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(src, (int)dtype, n_frames, w,
                                                                                       h, pitch_elems, dst);
    return cudaGetLastError() == cudaSuccess ? PBA_OK : PBA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Coarse-to-fine solve of one bundle (pba_pyramid_workspace_size,
// pba_solve_pyramid): host orchestration over the public entry points, one
// context per level, finest last. Level l halves the images l times
// (pba_downsample, FP32) with intrinsics f / 2^l and (c + 0.5) / 2^l - 0.5; a
// point keeps its inverse depth at every level, takes the nearest level pixel
// (u + 0.5) / 2^l - 0.5 rounded to nearest (ties to even), and sits a level
// out when its pattern and the pattern's gradient neighbours would leave
// that level's reference image. Workspace: the coarser levels' images, then
// the region every level's context uses in turn.
// ---------------------------------------------------------------------------
namespace {

struct PyrLevel {
    int w = 0, h = 0;
    size_t img_off = 0;  // coarser levels: offset of the FP32 images in the workspace
    double K[4] = {0, 0, 0, 0};
    std::vector<int32_t> uv;   // kept points' level pixels
    std::vector<int> idx;      // kept points' caller indices
    std::vector<uint8_t> vis;  // kept points' visibility rows (empty: all visible)
};

size_t pyr_align(size_t x) { return (x + 255) & ~(size_t)255; }

pba_status pyr_plan(const pba_config* cfg, int levels, int F, int w, int h, const double* K, int N,
                    const int32_t* uv, const uint8_t* vis, std::vector<PyrLevel>& L, size_t* img_bytes)
{
    if (!cfg || !K || !uv || levels < 1 || levels > 8 || F < 2 || N < 1 || cfg->pattern_size < 1 || !cfg->pattern)
        return PBA_ERR_ARG;
    if (cfg->n_bundles > 1) return PBA_ERR_ARG;
    int rad = 0;
    for (int j = 0; j < 2 * cfg->pattern_size; ++j) rad = std::max(rad, std::abs(cfg->pattern[j]));
    rad += 1;  // central differences of the template
    L.assign(levels, PyrLevel{});
    size_t off = 0;
    for (int l = 0; l < levels; ++l) {
        PyrLevel& v = L[l];
        v.w = l == 0 ? w : L[l - 1].w / 2;
        v.h = l == 0 ? h : L[l - 1].h / 2;
        if (v.w < 4 || v.h < 4) return PBA_ERR_ARG;
        if (l > 0) {
            v.img_off = off;
            off += pyr_align((size_t)F * v.w * v.h * sizeof(float));
        }
        const double s = std::ldexp(1.0, l);
        v.K[0] = K[0] / s;
        v.K[1] = K[1] / s;
        v.K[2] = (K[2] + 0.5) / s - 0.5;
        v.K[3] = (K[3] + 0.5) / s - 0.5;
        for (int n = 0; n < N; ++n) {
            const int u = (int)std::nearbyint((uv[2 * n] + 0.5) / s - 0.5);
            const int q = (int)std::nearbyint((uv[2 * n + 1] + 0.5) / s - 0.5);
            if (u < rad || u > v.w - 1 - rad || q < rad || q > v.h - 1 - rad) continue;
            v.uv.push_back(u);
            v.uv.push_back(q);
            v.idx.push_back(n);
            if (vis) v.vis.insert(v.vis.end(), vis + (size_t)n * F, vis + (size_t)(n + 1) * F);
        }
        if (v.idx.empty()) return PBA_ERR_ARG;
    }
    *img_bytes = off;
    return PBA_OK;
}

// A level's context with its frames and points set (images: device pointer
// of the level, not read before pba_set_workspace).
pba_status pyr_context(const pba_config* cfg, const PyrLevel& v, int F, const void* images, pba_dtype dtype,
                       int pitch, const double* poses, const double* inv_depth, pba_ctx** out)
{
    pba_config c = *cfg;
    c.n_bundles = 1;
    pba_ctx* ctx = nullptr;
    pba_status s = pba_create(&c, &ctx);
    if (s != PBA_OK) return s;
    std::vector<double> d(v.idx.size());
    for (size_t i = 0; i < v.idx.size(); ++i) d[i] = inv_depth[v.idx[i]];
    s = pba_set_frames(ctx, 0, F, v.w, v.h, pitch, dtype, PBA_MEM_DEVICE, images, poses, v.K);
    if (s == PBA_OK)
        s = pba_set_points(ctx, 0, (int)v.idx.size(), v.uv.data(), d.data(), v.vis.empty() ? nullptr : v.vis.data());
    if (s != PBA_OK) {
        pba_destroy(ctx);
        return s;
    }
    *out = ctx;
    return PBA_OK;
}

}  // namespace

extern "C" pba_status pba_pyramid_workspace_size(const pba_config* cfg, int levels, int n_frames, int w, int h,
                                                 const double* poses, const double* intrinsics, int n_points,
                                                 const int32_t* uv, const double* inv_depth, const uint8_t* vis,
                                                 size_t* bytes)
{
    if (!bytes || !poses || !inv_depth) return PBA_ERR_ARG;
    std::vector<PyrLevel> L;
    size_t img = 0;
    pba_status s = pyr_plan(cfg, levels, n_frames, w, h, intrinsics, n_points, uv, vis, L, &img);
    if (s != PBA_OK) return s;
    size_t most = 0;
    for (int l = 0; l < levels; ++l) {
        pba_ctx* ctx = nullptr;
        // the level's images are not read by the size query: an aligned
        // placeholder stands in for them
        s = pyr_context(cfg, L[l], n_frames, reinterpret_cast<const void*>((uintptr_t)256), PBA_F32, L[l].w, poses,
                        inv_depth, &ctx);
        if (s != PBA_OK) return s;
        size_t b = 0;
        s = pba_workspace_size(ctx, &b);
        pba_destroy(ctx);
        if (s != PBA_OK) return s;
        most = std::max(most, b);
    }
    *bytes = img + most;
    return PBA_OK;
}

extern "C" pba_status pba_solve_pyramid(const pba_config* cfg, int levels, const int* iters, int method,
                                        int reanchor_every, const void* images, pba_dtype dtype, int n_frames,
                                        int w, int h, int pitch_elems, double* poses, const double* intrinsics,
                                        int n_points, const int32_t* uv, double* inv_depth, const uint8_t* vis,
                                        void* workspace, size_t ws_bytes, pba_iter_stats* stats, double* level_ms)
{
    if (!iters || !images || !poses || !inv_depth || !workspace || (method != 0 && method != 1)) return PBA_ERR_ARG;
    if ((uintptr_t)workspace % 256) return PBA_ERR_ARG;
    std::vector<PyrLevel> L;
    size_t img = 0;
    pba_status s = pyr_plan(cfg, levels, n_frames, w, h, intrinsics, n_points, uv, vis, L, &img);
    if (s != PBA_OK) return s;
    for (int l = 0; l < levels; ++l)
        if (iters[l] < 0) return PBA_ERR_ARG;
    // every level's need first: a workspace too small solves nothing
    size_t need_all = 0;
    s = pba_pyramid_workspace_size(cfg, levels, n_frames, w, h, poses, intrinsics, n_points, uv, inv_depth, vis,
                                   &need_all);
    if (s != PBA_OK) return s;
    if (ws_bytes < need_all) return PBA_ERR_NOMEM;
    char* ws = static_cast<char*>(workspace);
    // the coarser levels' images, each from the one above
    for (int l = 1; l < levels; ++l) {
        const void* src = l == 1 ? images : static_cast<const void*>(ws + L[l - 1].img_off);
        s = pba_downsample(src, l == 1 ? dtype : PBA_F32, n_frames, L[l - 1].w, L[l - 1].h,
                           l == 1 ? pitch_elems : L[l - 1].w, reinterpret_cast<float*>(ws + L[l].img_off),
                           cfg->cuda_stream);
        if (s != PBA_OK) return s;
    }
    int stat_off = 0;
    for (int l = levels - 1; l >= 0; --l) {
        const PyrLevel& v = L[l];
        const int n = iters[levels - 1 - l];
        pba_ctx* ctx = nullptr;
        const void* lim = l == 0 ? images : static_cast<const void*>(ws + v.img_off);
        s = pyr_context(cfg, v, n_frames, lim, l == 0 ? dtype : PBA_F32, l == 0 ? pitch_elems : v.w, poses,
                        inv_depth, &ctx);
        if (s != PBA_OK) return s;
        size_t need = 0;
        s = pba_workspace_size(ctx, &need);
        if (s == PBA_OK && ws_bytes - img < need) s = PBA_ERR_NOMEM;
        if (s == PBA_OK) s = pba_set_workspace(ctx, ws + img, ws_bytes - img);
        pba_iter_stats* st = stats ? stats + stat_off : nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (s == PBA_OK && level_ms) {
            if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
                cudaEventRecord(e0, static_cast<cudaStream_t>(cfg->cuda_stream)) != cudaSuccess)
                s = PBA_ERR_CUDA;
        }
        if (s == PBA_OK) s = method == 0 ? pba_solve_ic(ctx, n, reanchor_every, st) : pba_solve_fc(ctx, n, st);
        if (s == PBA_OK && level_ms) {
            float ms = 0.0f;
            if (cudaEventRecord(e1, static_cast<cudaStream_t>(cfg->cuda_stream)) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                s = PBA_ERR_CUDA;
            level_ms[levels - 1 - l] = ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        stat_off += n + 1;
        std::vector<double> d(v.idx.size());
        if (s == PBA_OK) s = pba_get_params(ctx, 0, poses, d.data());
        pba_destroy(ctx);
        if (s != PBA_OK) return s;
        // a point the level drove to a non-positive inverse depth keeps the
        // one it entered the level with
        for (size_t i = 0; i < v.idx.size(); ++i)
            if (std::isfinite(d[i]) && d[i] > 0.0) inv_depth[v.idx[i]] = d[i];
    }
    return PBA_OK;
}
