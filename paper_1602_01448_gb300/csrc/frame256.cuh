// 256 x 256 frames: the standalone frame operators (forward model Eq. 1, P_a
// Eq. 7, amplitude loss and its adjoint, the Fourier mask of the illumination
// constraint) for frames too large for one SM.  (The RAAR frame pass of
// 256^2 frames runs in raar_split256.cuh.)
//
// A 256^2 frame is 512 KB of complex values, more than an SM's registers and
// shared memory together, so the 2D transform F (Eq. 2) runs as 1D passes
// over lines with the frame parked between passes in a per-block slab of
// global memory (512 KB per block, one block per SM: 78 MB on 152 SMs, held
// in L2 with an evict_last policy while the streamed state and amplitudes go
// evict_first):
//   pass 1  rows:    form z (frames in, or probe x object), 256-point DFT of
//                    each row, park in the slab
//   pass 2  columns: 256-point DFT of each column, the Fourier-domain step
//                    (P_a / amplitudes / loss / residual / mask), inverse DFT
//                    of each column, park
//   pass 3  rows:    inverse DFT of each row, epilogue (frames out, gradient
//                    scatter)
// Each pass walks the frame in chunks of 32 lines.  A 256-point line
// transform is 16 x 16 Cooley-Tukey: 16 threads (rows) or 16 thread groups
// (columns) each hold 16 samples n = 16 n1 + j, take a 16-point DFT over
// n1, multiply by W_256^(j k1), exchange through shared memory, and take a
// 16-point DFT over the other index:
//   X[k1 + 16 k2] = sum_n2 W_16^(n2 k2) W_256^(n2 k1) sum_n1 W_16^(n1 k1) x[16 n1 + n2]
// Input and output then share one layout (thread j holds indices j + 16 q),
// forward and inverse alike, so the passes chain without reordering.
//
// Row layout:    thread tid = 16 line + j, row y = 32 chunk + line,
//                holds x = 16 n + j (two rows of 16 x 8 bytes per warp access)
// Column layout: thread tid = 32 j + cx, column x = 32 chunk + cx,
//                holds y = 16 n + j (one 256-byte row segment per warp access)
// Exchange slots (conflict-free for 8-byte accesses):
//   rows    (line, a, b) at line*272 + a*17 + b
//   columns (a, b, cx)   at (a*16 + b)*32 + cx
// Two exchange buffers alternate between successive line transforms, so a
// transform needs a single barrier.
//
// Frames are handed out by an atomic counter (dynamic scheduling).  No wait
// in this kernel spins on memory.
#pragma once

#include <cstring>

#include "fft_frame.cuh"
#include "sharp_common.cuh"
#include "tma.cuh"
#include "twiddle_tables.cuh"

namespace sharp {
namespace big {

constexpr int M = 256;
constexpr int MM = M * M;
constexpr int NT = 512;
constexpr int LINES = 32;             // lines per chunk
constexpr int NCHUNK = M / LINES;
constexpr int RP = 17;                // row exchange: pitch of one a-row
constexpr int LP = 16 * RP;           // row exchange: pitch of one line
constexpr int E_ELEMS = LINES * LP;   // 8704 float2 per exchange buffer
constexpr int TW = 256;
constexpr size_t SMEM = (size_t)(2 * E_ELEMS + TW) * sizeof(float2);
static_assert(E_ELEMS >= 16 * 16 * LINES, "the column exchange fits the buffer");
static_assert(NT == 16 * LINES && NT == 32 * 16, "thread layouts");

__device__ __forceinline__ void fence_c() { asm volatile("" ::: "memory"); }

// ---------------------------------------------------------------- line DFTs
// Rows: v[n] = x[16 n + j] -> v[q] = X[j + 16 q] (raw, e^{-2 pi i}).
__device__ __forceinline__ void row_fwd(float2 (&v)[16], float2* E, const float2* tw, int line, int j) {
    dft_reg<16, -1>(v, 0, 1);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], tw[k * 16 + j]);
    float2* e = E + line * LP;
#pragma unroll
    for (int k = 0; k < 16; ++k) e[k * RP + j] = v[k];
    __syncthreads();
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = e[j * RP + n];
    dft_reg<16, -1>(v, 0, 1);
}

// Rows: v[q] = X[j + 16 q] -> v[n] = sum_k X[k] e^{+2 pi i k (16 n + j)/256} (raw).
__device__ __forceinline__ void row_inv(float2 (&v)[16], float2* E, const float2* tw, int line, int j) {
    dft_reg<16, 1>(v, 0, 1);
#pragma unroll
    for (int n = 1; n < 16; ++n) v[n] = cmulc(tw[n * 16 + j], v[n]);
    float2* e = E + line * LP;
#pragma unroll
    for (int n = 0; n < 16; ++n) e[n * RP + j] = v[n];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = e[j * RP + k];
    dft_reg<16, 1>(v, 0, 1);
}

// Columns: the same transforms with the column exchange layout.
__device__ __forceinline__ void col_fwd(float2 (&v)[16], float2* E, const float2* tw, int cx, int j) {
    dft_reg<16, -1>(v, 0, 1);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], tw[k * 16 + j]);
#pragma unroll
    for (int k = 0; k < 16; ++k) E[(k * 16 + j) * 32 + cx] = v[k];
    __syncthreads();
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = E[(j * 16 + n) * 32 + cx];
    dft_reg<16, -1>(v, 0, 1);
}

__device__ __forceinline__ void col_inv(float2 (&v)[16], float2* E, const float2* tw, int cx, int j) {
    dft_reg<16, 1>(v, 0, 1);
#pragma unroll
    for (int n = 1; n < 16; ++n) v[n] = cmulc(tw[n * 16 + j], v[n]);
#pragma unroll
    for (int n = 0; n < 16; ++n) E[(n * 16 + j) * 32 + cx] = v[n];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = E[(j * 16 + k) * 32 + cx];
    dft_reg<16, 1>(v, 0, 1);
}

// ---------------------------------------------------------------- phases
// Pass 1: form the frame samples of row y at x = 16 n + j.
template <int MODE>
__device__ __forceinline__ void form_row(const FrameArgs& a, int py, int px, size_t fo, int y, int j,
                                         float2 (&v)[16], uint64_t pol_stream, uint64_t pol_keep) {
    constexpr int CH = 4;
#pragma unroll
    for (int n0 = 0; n0 < 16; n0 += CH) {
        if constexpr (MODE == MODE_PROJECT || MODE == MODE_MASK) {
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) v[n] = ld_hint(a.zin + fo + y * M + 16 * n + j, pol_stream);
        } else {   // AMPS, LOSS, GRAD: z = w . obj(r + x_i)
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const int x = 16 * n + j;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                v[n] = cmul(ld_hint(a.probe + y * M + x, pol_keep), a.obj[o]);
            }
        }
        fence_c();
    }
}

// Pass 2: the Fourier-domain step on column x, v[q] = X[16 q + j][x] (raw
// DFT, m times the unitary transform).  AMPS and LOSS need no inverse.
// `bad` collects measured amplitudes that are not finite and non-negative.
template <int MODE>
__device__ __forceinline__ void fourier_col(const FrameArgs& a, size_t fo, int x, int j, float2 (&v)[16],
                                            float (&acc)[5], int& bad) {
    const float inv_m = 1.0f / M;
    if constexpr (MODE == MODE_AMPS) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float m2 = cabs2(v[q]);
            const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
            a.amp_out[fo + (16 * q + j) * M + x] = m2 * rs * inv_m;
        }
        return;
    } else if constexpr (MODE == MODE_MASK) {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = cscale(v[q], a.amp[fo + (16 * q + j) * M + x] * inv_m * inv_m);
        return;
    } else {
        float av[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) av[q] = __ldcs(a.amp + fo + (16 * q + j) * M + x);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float2& X = v[q];
            const float m2 = cabs2(X);
            const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
            const float d = av[q] - m2 * rs * inv_m;
            acc[0] += d * d;
            bad |= (int)bad_amplitude(av[q]);
            if constexpr (MODE == MODE_PROJECT) {
                X = m2 > 0.f ? cscale(X, av[q] * inv_m * rs) : make_float2(av[q] * inv_m, 0.f);
            } else if constexpr (MODE == MODE_GRAD) {
                X = m2 > 0.f ? cscale(X, (inv_m - av[q] * rs) * inv_m) : make_float2(-av[q] * inv_m, 0.f);
            }
        }
    }
}

// Pass 3: epilogue of row y, v[n] = result at x = 16 n + j.
template <int MODE>
__device__ __forceinline__ void finish_row(const FrameArgs& a, int py, int px, size_t fo, int y, int j,
                                           const float2 (&v)[16], uint64_t pol_stream, uint64_t pol_keep) {
    constexpr int CH = 4;
#pragma unroll
    for (int n0 = 0; n0 < 16; n0 += CH) {
        if constexpr (MODE == MODE_PROJECT || MODE == MODE_MASK) {
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) st_hint(a.zout + fo + y * M + 16 * n + j, v[n], pol_stream);
        } else if constexpr (MODE == MODE_GRAD) {
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const int x = 16 * n + j;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                const float2 r = cscale(v[n], a.gscale);
                red_add_f2(a.g_obj + o, cmulc(ld_hint(a.probe + y * M + x, pol_keep), r));
                if (a.g_probe) red_add_f2(a.g_probe + y * M + x, cmulc(a.obj[o], r));
            }
        }
        fence_c();
    }
}

// ---------------------------------------------------------------- kernel
// One scan's frames; `slab` holds gridDim.x frames of scratch.
template <int MODE>
__global__ void __launch_bounds__(NT, 1) big_kernel(const FrameArgs ap, float2* slab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* Ebuf = reinterpret_cast<float2*>(smem_raw);
    float2* tw = Ebuf + 2 * E_ELEMS;
    __shared__ float red[32 * 5];
    __shared__ FrameArgs a;
    __shared__ int s_frame;
    const int tid = threadIdx.x;
    float2* scr = slab + (size_t)blockIdx.x * MM;
    for (int i = tid; i < TW; i += NT) tw[i] = c_tw256x16[i];
    if (tid == 0) {
        a = ap;
        __nanosleep(2000u * (blockIdx.x & 3u));
    }
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    // row layout
    const int line = tid >> 4, jr = tid & 15;
    // column layout
    const int cx = tid & 31, jc = tid >> 5;

    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    double accd = 0.0;
    int eb = 0;
    int bad = 0;

    for (;;) {
        if (tid == 0) s_frame = atomicAdd(a.counter, 1);
        __syncthreads();
        const int i = s_frame;
        if (i >= a.K) break;
        const int py = a.pos[2 * i];
        const int px = a.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;

        // ---------------------------------------------- pass 1: rows
        for (int r0 = 0; r0 < M; r0 += LINES) {
            const int y = r0 + line;
            float2 v[16];
            form_row<MODE>(a, py, px, fo, y, jr, v, pol_stream, pol_keep);
            row_fwd(v, Ebuf + eb * E_ELEMS, tw, line, jr);
            eb ^= 1;
#pragma unroll
            for (int q = 0; q < 16; ++q) st_hint(scr + y * M + jr + 16 * q, v[q], pol_keep);
        }
        __syncthreads();
        // ---------------------------------------------- pass 2: columns
        for (int c0 = 0; c0 < M; c0 += LINES) {
            const int x = c0 + cx;
            float2 v[16];
#pragma unroll
            for (int n = 0; n < 16; ++n) v[n] = ld_hint(scr + (16 * n + jc) * M + x, pol_keep);
            col_fwd(v, Ebuf + eb * E_ELEMS, tw, cx, jc);
            eb ^= 1;
            fourier_col<MODE>(a, fo, x, jc, v, acc, bad);
            if constexpr (MODE != MODE_AMPS && MODE != MODE_LOSS) {
                col_inv(v, Ebuf + eb * E_ELEMS, tw, cx, jc);
                eb ^= 1;
#pragma unroll
                for (int n = 0; n < 16; ++n) st_hint(scr + (16 * n + jc) * M + x, v[n], pol_keep);
            }
        }
        if constexpr (MODE != MODE_AMPS && MODE != MODE_LOSS) {
            __syncthreads();
            // ------------------------------------------ pass 3: rows
            for (int r0 = 0; r0 < M; r0 += LINES) {
                const int y = r0 + line;
                float2 v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = ld_hint(scr + y * M + jr + 16 * q, pol_keep);
                row_inv(v, Ebuf + eb * E_ELEMS, tw, line, jr);
                eb ^= 1;
                finish_row<MODE>(a, py, px, fo, y, jr, v, pol_stream, pol_keep);
            }
        }
        accd += (double)acc[0];
        acc[0] = 0.f;
    }
    if (__syncthreads_or(bad) && tid == 0) raise_error(a.err, SHARP_ERR_INVALID_ARG);
    float s[1] = {(float)accd};
    block_sum<NT, 1>(s, red);
    if constexpr (MODE != MODE_AMPS && MODE != MODE_MASK)
        if (tid == 0) atomicAdd(a.sums, (double)s[0]);
}

}  // namespace big

// ---------------------------------------------------------------- launchers
// Resident blocks of the 256^2 kernels: one per SM (each owns a slab).
inline cudaError_t big_max_grid(int* grid) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *grid = sms;
    return e;
}

template <int MODE>
cudaError_t big_launch(const FrameArgs& a, float2* slab, cudaStream_t s) {
    auto kern = big::big_kernel<MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big::SMEM);
    if (e != cudaSuccess) return e;
    int grid = 0;
    if ((e = big_max_grid(&grid)) != cudaSuccess) return e;   // never more blocks than slabs
    if (grid > a.K) grid = a.K;
    if (grid <= 0) return cudaSuccess;
    if (!slab || !a.counter) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(a.counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    kern<<<grid, big::NT, big::SMEM, s>>>(a, slab);
    return cudaGetLastError();
}

}  // namespace sharp
