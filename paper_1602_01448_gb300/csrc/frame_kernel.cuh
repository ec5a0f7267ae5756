// Per-frame kernels for the standalone operators: one thread block transforms
// one m x m frame in registers and shared memory (fft_frame.cuh), one block
// per frame.  Modes:
//   MODE_PROJECT    P_a z = F* (a Fz/|Fz|) of explicit frames (Eq. 7) and the
//                   residual sum ||P_a z - z||^2
//   MODE_PROJECT_PF the same with one residual per frame (allocation-free entry)
//   MODE_AMPS       forward model a = |F (w . obj(r + x_i))| (Eq. 1)
//   MODE_LOSS       sum (|F z| - a)^2 with z = w . obj(r + x_i)
//   MODE_GRAD       adjoint of the loss: r = z - P_a z scattered as conj(w) r
//                   (object) and conj(obj) r (probe)
//   MODE_MASK       F^-1{(F z) mask} (the illumination Fourier-mask constraint,
//                   Sec. 2.2 step 7)
// The fused RAAR step lives in raar_kernel.cuh (64^2, 128^2) and frame256.cuh
// (256^2, which also serves these modes for 256^2 frames).
#pragma once
#include <cuda_runtime.h>

#include "fft_frame.cuh"
#include "sharp_common.cuh"

namespace sharp {

// Compiler barrier between chunks of the gather/scatter loops: keeps ptxas
// from hoisting all 32 rows of loads at once (which overflows the 128
// registers of a 512-thread block); the other warps of the block hide the
// latency of each chunk.
__device__ __forceinline__ void chunk_fence() { asm volatile("" ::: "memory"); }
// Returns v unchanged but opaque to the optimiser, so address arithmetic that
// depends on it stays below this point instead of being hoisted above the
// FFT (where its registers would stay live).
__device__ __forceinline__ int pin(int v) {
    asm volatile("" : "+r"(v));
    return v;
}
constexpr int CHUNK = 4;
// Ordinary (coherent) load: unlike ld.global.nc it stays behind chunk_fence().
template <class T>
__device__ __forceinline__ T ld_plain(const T* p) { return *p; }

template <int M, int MODE, int FLAGS>
__global__ void __launch_bounds__(Fft3<M>::NT, 1) frame_kernel(const FrameArgs a) {
    using G = Fft3<M>;
    constexpr int NT = G::NT;
    constexpr int TX = G::TX;
    constexpr int MM = M * M;
    extern __shared__ float2 S[];             // exchange buffer, then twiddles
    float2* tw = S + G::SMEM_ELEMS;
    __shared__ float red[32 * 5];

    const int tid = threadIdx.x;
    G::load_twiddles(tw);
    __syncthreads();
    const int q = tid / M;        // pass-1 layout: rows y = q + TX k, column x
    const int x = tid % M;
    const float inv_m = 1.0f / M;

    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};

    for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
        // explicit frames carry no position (the plan-free projection has none)
        const int py = (MODE == MODE_PROJECT_PF) ? 0 : a.pos[2 * i];
        const int px = (MODE == MODE_PROJECT_PF) ? 0 : a.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;
        float2 v[32];

        // ------------------------------------------------ form the frame
        if constexpr (MODE == MODE_PROJECT || MODE == MODE_PROJECT_PF || MODE == MODE_MASK) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int y = q + TX * k;
                v[k] = ld_plain(a.zin + fo + y * M + x);
                if ((k % CHUNK) == CHUNK - 1) chunk_fence();
            }
        } else {  // AMPS, LOSS, GRAD: z = w . obj(r + x_i)
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int y = q + TX * k;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                v[k] = cmul(ld_plain(a.probe + y * M + x), ld_plain(a.obj + o));
                if ((k % CHUNK) == CHUNK - 1) chunk_fence();
            }
        }

        G::forward(v, S, tw);

        // ------------------------------------------------ Fourier domain
        const float* ai = (MODE == MODE_AMPS) ? nullptr : a.amp + fo;
#pragma unroll
        for (int c = 0; c < G::C3; ++c) {
            const int ky = G::p3_ky(c);
#pragma unroll
            for (int s = 0; s < G::X0; ++s) {
                const int kx = G::p3_kx(s);
                float2& X = v[c * G::X0 + s];
                const float m2 = cabs2(X);
                const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                const float mag = m2 * rs * inv_m;     // |F z| on the unitary scale
                if constexpr (MODE == MODE_AMPS) {
                    a.amp_out[fo + ky * M + kx] = mag;
                } else if constexpr (MODE == MODE_MASK) {
                    X = cscale(X, __ldg(ai + ky * M + kx) * inv_m * inv_m);
                } else {
                    const float av = __ldg(ai + ky * M + kx);
                    const float d = av - mag;
                    acc[0] += d * d;
                    if constexpr (MODE == MODE_PROJECT || MODE == MODE_PROJECT_PF) {
                        // Z'' = (a Z/|Z|) / m so that the raw inverse gives P_a z
                        X = m2 > 0.f ? cscale(X, av * inv_m * rs) : make_float2(av * inv_m, 0.f);
                    } else if constexpr (MODE == MODE_GRAD) {
                        // (Z - a Z/|Z|) / m  ->  r = z - P_a z after the raw inverse
                        X = m2 > 0.f ? cscale(X, (inv_m - av * rs) * inv_m) : make_float2(-av * inv_m, 0.f);
                    }
                }
            }
        }
        if constexpr (MODE == MODE_AMPS || MODE == MODE_LOSS) continue;

        G::inverse(v, S, tw);

        // ------------------------------------------------ epilogue
        if constexpr (MODE == MODE_PROJECT || MODE == MODE_PROJECT_PF || MODE == MODE_MASK) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int y = q + TX * k;
                a.zout[fo + y * M + x] = v[k];
                if ((k % CHUNK) == CHUNK - 1) chunk_fence();
            }
        } else if constexpr (MODE == MODE_GRAD) {
            const float gs = a.gscale;
            const int epy = pin(py), epx = pin(px), enx = pin(a.nx);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int y = q + TX * k;
                const int o = obj_index(epy, epx, y, x, a.ny, enx, a.wrap);
                const float2 r = cscale(v[k], gs);
                red_add_f2(a.g_obj + o, cmulc(ld_plain(a.probe + y * M + x), r));
                if (a.g_probe) red_add_f2(a.g_probe + y * M + x, cmulc(ld_plain(a.obj + o), r));
                if ((k % CHUNK) == CHUNK - 1) chunk_fence();
            }
        }
        if constexpr (MODE == MODE_PROJECT_PF) {
            // one residual per frame, each written by its own block
            block_sum<NT, 5>(acc, red);
            if (tid == 0) a.sums[i] = (double)acc[0];
#pragma unroll
            for (int j = 0; j < 5; ++j) acc[j] = 0.f;
        }
    }

    if constexpr (MODE != MODE_PROJECT_PF && MODE != MODE_MASK) {
        block_sum<NT, 5>(acc, red);
        if (tid == 0) {
            if constexpr (MODE != MODE_AMPS) atomicAdd(a.sums, (double)acc[0]);
        }
    }
}

template <int M, int MODE, int FLAGS>
static cudaError_t launch_one(const FrameArgs& a, cudaStream_t s) {
    using G = Fft3<M>;
    const size_t smem = sizeof(float2) * (G::SMEM_ELEMS + G::TW1 + G::TW2);
    auto kern = frame_kernel<M, MODE, FLAGS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.K, G::NT, smem, s>>>(a);
    return cudaGetLastError();
}

// All kernels of one frame size (instantiated once per translation unit).
template <int M>
cudaError_t launch_frames_m(int mode, int flags, const FrameArgs& a, cudaStream_t s) {
    switch (mode) {
        case MODE_PROJECT: return launch_one<M, MODE_PROJECT, 0>(a, s);
        case MODE_AMPS: return launch_one<M, MODE_AMPS, 0>(a, s);
        case MODE_LOSS: return launch_one<M, MODE_LOSS, 0>(a, s);
        case MODE_GRAD: return launch_one<M, MODE_GRAD, 0>(a, s);
        case MODE_MASK: return launch_one<M, MODE_MASK, 0>(a, s);
        case MODE_RAAR: return launch_raar_m<M>(flags, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sharp
