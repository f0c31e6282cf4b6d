// Reduced camera system for callers that cannot allocate device memory.
//
// The context API needs a workspace that the caller allocates. Some callers
// cannot do that: code that runs inside a fixed, pre-reserved memory arena,
// a host runtime that forbids cudaMalloc after start-up (real-time loops,
// embedded or safety-certified deployments), or a framework that hands out
// only the tensors of an operation's inputs and outputs. For them this file
// provides pba_reduced_system_noalloc(): it builds the anchored reduced
// camera system S from dense Hessian blocks the caller already holds, with
// its scratch (the Schur-complement partial sums, the upper-triangle copy of
// the frame blocks and the frame flags) in one static device array.
//
// The array is a file-scope __device__ symbol: every GPU that loads the
// library holds it until the process exits, and every call on a device
// shares it. In host code its name is only a host-side stand-in, so the
// device address is looked up with cudaGetSymbolAddress and cached per
// device together with the identity of the CUDA context it belongs to; a
// call from another context on that device (after cudaDeviceReset, or with
// a context the caller made current) looks the address up again.
#include <cuda.h>

#include <mutex>

#include "pba_kernels.cuh"

namespace {

using namespace pba;

constexpr int kMaxFrames = PBA_NOALLOC_MAX_FRAMES;
constexpr int kMaxN6 = 6 * (kMaxFrames - 1);
constexpr size_t kSoffBytes = sizeof(double) * kMaxN6 * kMaxN6;
constexpr size_t kHffBytes = sizeof(double) * kMaxFrames * 21;
constexpr size_t kActiveBytes = sizeof(int) * kMaxFrames;
constexpr size_t kScratchBytes = kSoffBytes + kHffBytes + kActiveBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address belongs to

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context (0: none current). The
// two driver functions are reached through the runtime's entry-point query,
// so the library needs no link against the driver library.
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess)
            return 0;
        get_current = reinterpret_cast<CtxGetCurrentFn>(a);
        get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context of the
// current device (looked up again whenever that context changes).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current if none is
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// S_off[f][g] = sum_n Hfd(n,f) Hfd(n,g)^T / Hdd(n) from dense blocks
// (Hfd: N*F*6, zero where a point is not observed), one CTA per frame pair
// f <= g, FP64 products, fixed-order reduction. Block 0 also copies the
// frame blocks into the upper-triangle layout the assembly reads.
constexpr int kWarps = 4;

__global__ void __launch_bounds__(32 * kWarps)
schur_offdiag_dense_kernel(int F, int N, const double* Hff, const double* Hfd, const double* Hdd,
                           double* Soff, double* hff21)
{
    __shared__ double red[kWarps][36];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n6 = 6 * (F - 1);
    int idx = blockIdx.x, f = 1;
    while (idx >= F - f) {
        idx -= F - f;
        ++f;
    }
    const int g = f + idx;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < F * 21; i += blockDim.x) {
            const int fr = i / 21;
            int q = i % 21, a = 0;
            while (q >= 6 - a) {
                q -= 6 - a;
                ++a;
            }
            hff21[i] = Hff[(size_t)fr * 36 + 6 * a + a + q];
        }
    }
    double s[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) s[k] = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double h = Hdd[n];
        if (!(h > 0.0)) continue;
        const double ih = 1.0 / h;
        const double* pa = Hfd + ((size_t)n * F + f) * 6;
        const double* pb = Hfd + ((size_t)n * F + g) * 6;
        double ha[6], hb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ha[k] = pa[k];
            hb[k] = pb[k];
        }
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) s[6 * a + b] = fma(ha[a] * hb[b], ih, s[6 * a + b]);
    }
#pragma unroll
    for (int k = 0; k < 36; ++k) {
        const double v = warp_sum1d(s[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 36 && (f != g || threadIdx.x / 6 <= threadIdx.x % 6)) {
        const int k = threadIdx.x, a = k / 6, b = k % 6;
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += red[w][k];
        const int i = 6 * (f - 1) + a, j = 6 * (g - 1) + b;
        Soff[(size_t)i * n6 + j] = v;
        Soff[(size_t)j * n6 + i] = v;
    }
}

}  // namespace

extern "C" pba_status pba_reduced_system_noalloc(int n_frames, int n_points, const double* Hff,
                                                 const double* Hfd, const double* Hdd,
                                                 const double* poses, double gauge_anchor_w,
                                                 double* S, void* cuda_stream)
{
    if (n_frames > kMaxFrames) return PBA_ERR_TOO_LARGE;
    if (n_frames < 2 || n_points < 1 || !Hff || !Hfd || !Hdd || !poses || !S ||
        gauge_anchor_w < 0.0)
        return PBA_ERR_ARG;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PBA_ERR_CUDA;
    double* soff = reinterpret_cast<double*>(base);
    double* hff21 = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kSoffBytes);
    int* active = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kSoffBytes + kHffBytes);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int F = n_frames, n_pairs = (F - 1) * F / 2;
    // every S_off entry, frame-block copy and flag the assembly reads is
    // rewritten by this call, so the previous call's contents never leak in
    schur_offdiag_dense_kernel<<<n_pairs, 32 * kWarps, 0, st>>>(F, n_points, Hff, Hfd, Hdd, soff,
                                                                hff21);
    if (cudaGetLastError() != cudaSuccess) return PBA_ERR_CUDA;
    BundleSet one{};
    one.B = 1;
    one.one.F = F;
    one.n6max = 6 * (F - 1);
    if (launch_assemble_S(one, hff21, 21, soff, poses, gauge_anchor_w == 0.0 ? 1.0 : gauge_anchor_w, 0.0,
                          S, active, st) != cudaSuccess)
        return PBA_ERR_CUDA;
    return PBA_OK;
}
