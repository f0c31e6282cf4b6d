// Image pyramid for coarse-to-fine solving (an addition beyond the paper:
// the basin of the direct method widens at coarse levels). One level down
// halves each image dimension; a pixel is the mean of the 2 x 2 block it
// covers, so pixel centres follow x_coarse = (x_fine + 0.5) / 2 - 0.5.
#include <algorithm>

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
