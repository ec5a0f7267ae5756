// 256 x 256 frames: the RAAR frame pass (Sec. 2.2, Eqs. 5, 7-9) and the
// standalone frame operators (forward model Eq. 1, P_a Eq. 7, amplitude loss
// and its adjoint) for frames too large for one SM.
//
// A 256^2 frame is 512 KB of complex values, more than an SM's registers and
// shared memory together, so the 2D transform F (Eq. 2) runs as 1D passes
// over lines with the frame parked between passes in a per-block slab of
// global memory (512 KB per block, one block per SM: 78 MB on 152 SMs, held
// in L2 with an evict_last policy while the streamed state and amplitudes go
// evict_first):
//   pass 1  rows:    form z (gather, state, metrics), 256-point DFT of each
//                    row, park in the slab
//   pass 2  columns: 256-point DFT of each column, the Fourier-domain step
//                    (P_a / RAAR combination / amplitudes / loss / residual),
//                    inverse DFT of each column, park
//   pass 3  rows:    inverse DFT of each row, epilogue (state store, overlap
//                    scatter, frames out, gradient scatter)
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
// Frames are handed out by an atomic counter (dynamic scheduling).  The same
// kernel serves one scan (arguments as a kernel parameter) or a batch of
// scans (a device table of arguments, BatchTable), as the 64/128 RAAR kernels
// do.  No wait in this kernel spins on memory.
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
// Pass 1: form the frame samples of row y at x = 16 n + j, loading RCH
// samples per round trip in the RAAR mode without metrics (a tile parameter
// of the batch tuner), 4 otherwise.
template <int MODE, int FLAGS, int RCH = 8>
__device__ __forceinline__ void form_row(const FrameArgs& a, int py, int px, size_t fo, int y, int j,
                                         float2 (&v)[16], float (&acc)[5], uint64_t pol_stream,
                                         uint64_t pol_keep) {
    constexpr int CH = (MODE == MODE_RAAR && !(FLAGS & RF_METRIC)) ? RCH : 4;
#pragma unroll
    for (int n0 = 0; n0 < 16; n0 += CH) {
        if constexpr (MODE == MODE_RAAR) {
            float2 wf[CH], yv[CH], cv[CH], pv[CH], ev[CH];
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const int x = 16 * n + j;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                wf[n - n0] = ld_hint(a.w_form + y * M + x, pol_keep);
                yv[n - n0] = a.psiy[o];
                cv[n - n0] = ld_hint(a.c + fo + y * M + x, pol_stream);
                if constexpr (FLAGS & (RF_METRIC | RF_FORM_B)) pv[n - n0] = a.psi[o];
                if constexpr (FLAGS & RF_METRIC)
                    ev[n - n0] = a.read_e ? ld_hint(a.ebuf + fo + y * M + x, pol_stream) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const float2 wy = cmul(wf[n - n0], yv[n - n0]);
                const float2 z = cadd(wy, cv[n - n0]);
                v[n] = z;
                acc[2] += cabs2(z);
                if constexpr (FLAGS & RF_METRIC) {
                    acc[3] += cabs2(csub(cmul(wf[n - n0], pv[n - n0]), z));
                    acc[4] += cabs2(cadd(wy, ev[n - n0]));
                }
            }
            if constexpr (FLAGS & RF_FORM_B) {
#pragma unroll
                for (int n = n0; n < n0 + CH; ++n) {
                    const int x = 16 * n + j;
                    const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                    // B' = Q*(z - w psi), relative to the object (image pass)
                    const float2 wp = ld_hint(a.w_proj + y * M + x, pol_keep);
                    red_add_f2(a.accB + o, cmulc(wp, csub(v[n], cmul(wp, pv[n - n0]))));
                }
            }
            if (a.write_e) {
#pragma unroll
                for (int n = n0; n < n0 + CH; ++n)
                    st_hint(a.ebuf + fo + y * M + 16 * n + j, make_float2(-v[n].x, -v[n].y), pol_stream);
            }
        } else if constexpr (MODE == MODE_PROJECT || MODE == MODE_MASK) {
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
        const float b = a.beta;
        const float cp = 1.f - 2.f * b;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float2& X = v[q];
            const float m2 = cabs2(X);
            const float rs = m2 > 0.f ? (MODE == MODE_RAAR ? rsqrt_refined(m2) : rsqrtf(m2)) : 0.f;
            const float d = av[q] - m2 * rs * inv_m;
            acc[0] += d * d;
            bad |= (int)bad_amplitude(av[q]);
            if constexpr (MODE == MODE_RAAR) {
                // ((1-2b) a Z/|Z| + b Z)/m on the unitary scale: the raw
                // inverse returns c_new = (1-2b) P_a z + b z
                acc[1] += av[q] * av[q];
                X = m2 > 0.f ? cscale(X, fmaf(cp * av[q], rs, b * inv_m) * inv_m)
                             : make_float2(cp * av[q] * inv_m, 0.f);
            } else if constexpr (MODE == MODE_PROJECT) {
                X = m2 > 0.f ? cscale(X, av[q] * inv_m * rs) : make_float2(av[q] * inv_m, 0.f);
            } else if constexpr (MODE == MODE_GRAD) {
                X = m2 > 0.f ? cscale(X, (inv_m - av[q] * rs) * inv_m) : make_float2(-av[q] * inv_m, 0.f);
            }
        }
    }
}

// Pass 3: epilogue of row y, v[n] = result at x = 16 n + j (RCH samples per
// round trip in the RAAR mode).
template <int MODE, int RCH = 8>
__device__ __forceinline__ void finish_row(const FrameArgs& a, int py, int px, size_t fo, int y, int j,
                                           const float2 (&v)[16], uint64_t pol_stream, uint64_t pol_keep) {
    constexpr int CH = MODE == MODE_RAAR ? RCH : 4;
#pragma unroll
    for (int n0 = 0; n0 < 16; n0 += CH) {
        if constexpr (MODE == MODE_RAAR) {
            // C' += conj(w) (c_new - (1-b) w psi): overlap sum relative to the
            // object (image pass)
            const float rho = 1.f - a.beta;
            float2 wp[CH], pv[CH];
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const int x = 16 * n + j;
                wp[n - n0] = ld_hint(a.w_proj + y * M + x, pol_keep);
                pv[n - n0] = a.psi[obj_index(py, px, y, x, a.ny, a.nx, a.wrap)];
            }
#pragma unroll
            for (int n = n0; n < n0 + CH; ++n) {
                const int x = 16 * n + j;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, a.wrap);
                st_hint(a.c + fo + y * M + x, v[n], pol_stream);
                red_add_f2(a.accA + o, cmulc(wp[n - n0], csub(v[n], cscale(cmul(wp[n - n0], pv[n - n0]), rho))));
                if (a.write_e) red_hint(a.ebuf + fo + y * M + x, v[n], pol_stream);
            }
        } else if constexpr (MODE == MODE_PROJECT || MODE == MODE_MASK) {
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
// `ap` serves a single scan when bt.scans is null; otherwise frames come
// from the scans of `bt`.  `slab` holds gridDim.x frames of scratch.
template <int MODE, int FLAGS, int RCH = 8>
__global__ void __launch_bounds__(NT, 1) big_kernel(const FrameArgs ap, const BatchTable bt, float2* slab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* Ebuf = reinterpret_cast<float2*>(smem_raw);
    float2* tw = Ebuf + 2 * E_ELEMS;
    __shared__ float red[32 * 5];
    __shared__ FrameArgs a;
    __shared__ int s_frame, s_scan;
    const int tid = threadIdx.x;
    const bool batch = bt.scans != nullptr;
    const int total = batch ? bt.total : ap.K;
    int* counter = batch ? bt.counter : ap.counter;
    float2* scr = slab + (size_t)blockIdx.x * MM;
    for (int i = tid; i < TW; i += NT) tw[i] = c_tw256x16[i];
    if (tid == 0) {
        if (!batch) a = ap;
        __nanosleep((batch ? (unsigned)bt.stagger_ns : 2000u) * (blockIdx.x & 3u));
    }
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    // row layout
    const int line = tid >> 4, jr = tid & 15;
    // column layout
    const int cx = tid & 31, jc = tid >> 5;

    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    double accd[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int loaded = batch ? -1 : 0;
    int eb = 0;
    int bad = 0;

    auto flush = [&]() {   // block-wide
        if (__syncthreads_or(bad) && tid == 0) {
            raise_error(a.err, SHARP_ERR_INVALID_ARG);   // the scan's plan status
            if (batch) raise_error(bt.err, SHARP_ERR_INVALID_ARG);
        }
        bad = 0;
        float s[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            s[k] = (float)accd[k];
            accd[k] = 0.0;
        }
        block_sum<NT, 5>(s, red);
        if (tid == 0) {
            if constexpr (MODE == MODE_RAAR) {
#pragma unroll
                for (int k = 0; k < 5; ++k) atomicAdd(a.sums + k, (double)s[k]);
            } else if constexpr (MODE != MODE_AMPS && MODE != MODE_MASK) {
                atomicAdd(a.sums, (double)s[0]);
            }
        }
    };

    for (;;) {
        if (tid == 0) {
            const int g = atomicAdd(counter, 1);
            s_frame = g;
            if (batch && g < total) {
                int s = 0;
                while (s + 1 < bt.nscans && bt.base[s + 1] <= g) ++s;
                s_scan = s;
            }
        }
        __syncthreads();
        const int g = s_frame;
        if (g >= total) break;
        int i = g;
        if (batch) {
            const int s = s_scan;
            if (s != loaded) {
                if (loaded >= 0) flush();
                __syncthreads();
                if (tid == 0) a = bt.scans[s];
                __syncthreads();
                loaded = s;
            }
            i = g - bt.base[s];
        }
        const int py = a.pos[2 * i];
        const int px = a.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;

        // ---------------------------------------------- pass 1: rows
        for (int r0 = 0; r0 < M; r0 += LINES) {
            const int y = r0 + line;
            float2 v[16];
            form_row<MODE, FLAGS, RCH>(a, py, px, fo, y, jr, v, acc, pol_stream, pol_keep);
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
                finish_row<MODE, RCH>(a, py, px, fo, y, jr, v, pol_stream, pol_keep);
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            accd[k] += (double)acc[k];
            acc[k] = 0.f;
        }
    }
    if (loaded >= 0) flush();
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

template <int MODE, int FLAGS, int RCH = 8>
cudaError_t big_launch(const FrameArgs& a, const BatchTable* bt, int grid, float2* slab, cudaStream_t s) {
    auto kern = big::big_kernel<MODE, FLAGS, RCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big::SMEM);
    if (e != cudaSuccess) return e;
    int maxg = 0;
    if ((e = big_max_grid(&maxg)) != cudaSuccess) return e;
    BatchTable t;
    memset(&t, 0, sizeof(t));
    if (bt) t = *bt;
    const int total = bt ? bt->total : a.K;
    int* counter = bt ? bt->counter : a.counter;
    if (grid <= 0 || grid > maxg) grid = maxg;   // never more blocks than slabs
    if (grid > total) grid = total;
    if (grid <= 0) return cudaSuccess;
    if (!slab || !counter) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    kern<<<grid, big::NT, big::SMEM, s>>>(a, t, slab);
    return cudaGetLastError();
}

}  // namespace sharp
