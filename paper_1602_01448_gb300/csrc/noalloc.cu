// Data projection P_a of explicit frames that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a host
// application that hands this library a fixed memory budget and owns every
// allocation itself, or a real-time loop that must never stall on the
// allocator (cudaMalloc and cudaFree can synchronise the device).  Such a
// caller provides the frames, amplitudes and outputs and calls this entry
// point, which keeps its only scratch -- one partial residual per frame -- in
// a fixed array in device global memory that belongs to the library.
//
// The array holds SHARP_NOALLOC_MAX_FRAMES doubles (512 KiB) and every GPU
// that loads the library keeps it until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up once (cudaGetSymbolAddress, with that device current)
// and caches it; make that first call before any stream capture begins.  All
// calls share the array, so calls whose work overlaps on the GPU (different
// streams, or several host threads) race and must be serialised by the
// caller.  Every call overwrites the entries it uses before reading them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "frame_kernel.cuh"
#include "sharp_common.cuh"

namespace {

constexpr int kMaxDevices = 64;

// One partial residual per frame; nothing else is stored between calls.
static __device__ __align__(256) double g_frame_resid[SHARP_NOALLOC_MAX_FRAMES];

std::mutex g_lookup_mutex;
double* g_resid_addr[kMaxDevices] = {nullptr};

int noalloc_fail(int code, const char* msg) {
    sharp::set_last_error(msg);
    return code;
}

// Sum of the per-frame residuals in frame order (one block, fixed order, so
// the result does not depend on how the frames were scheduled).
__global__ void sum_frames_kernel(const double* __restrict__ per_frame, int K, double* __restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) acc += per_frame[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <int M>
cudaError_t launch_pf(const float2* z, const float* amp, float2* out, double* scratch, int K, cudaStream_t s) {
    sharp::FrameArgs a;
    memset(&a, 0, sizeof(a));
    a.K = K;
    a.m = M;
    a.zin = z;
    a.zout = out;
    a.amp = amp;
    a.sums = scratch;
    return sharp::launch_one<M, sharp::MODE_PROJECT_PF, 0>(a, s);
}

}  // namespace

extern "C" int sharp_fourier_project_noalloc(const float2* z, const float* amp, float2* out, double* resid_sq,
                                             int K, int m, cudaStream_t stream) {
    if (!z || !amp || !out) return noalloc_fail(SHARP_ERR_INVALID_ARG, "z, amp and out must not be NULL");
    if (K < 1) return noalloc_fail(SHARP_ERR_INVALID_ARG, "K must be at least 1");
    if (K > SHARP_NOALLOC_MAX_FRAMES)
        return noalloc_fail(SHARP_ERR_INVALID_ARG,
                            "K exceeds SHARP_NOALLOC_MAX_FRAMES; use sharp_fourier_project with a plan");
    if (m != 64 && m != 128) return noalloc_fail(SHARP_ERR_UNSUPPORTED_SIZE, "frame size m must be 64 or 128");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SHARP_ERR_CUDA, "cannot determine the current device");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_lookup_mutex);
        if (!g_resid_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_frame_resid);
            if (e != cudaSuccess) return noalloc_fail(SHARP_ERR_CUDA, cudaGetErrorString(e));
            g_resid_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_resid_addr[dev];
    }
    cudaError_t e = (m == 64) ? launch_pf<64>(z, amp, out, scratch, K, stream)
                              : launch_pf<128>(z, amp, out, scratch, K, stream);
    if (e == cudaSuccess && resid_sq) {
        sum_frames_kernel<<<1, 256, 0, stream>>>(scratch, K, resid_sq);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return noalloc_fail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    return SHARP_OK;
}
