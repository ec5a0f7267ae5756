// Two-dimensional DFT of one m x m frame held by one thread block, in three
// register passes joined by two shared-memory exchanges.
//
// The frame transform F of Eq. 2 (unitary, e^{-2 pi i} reading) is computed
// unnormalised here; callers apply the 1/m factors.  With M = 32 * TX,
// TT = 32 / TX and X0 = M / TT, the 2D index space is split as
//   y = q + TX k        (q < TX, k < 32)      pass 1: 32-point DFT over k
//   x = x0 + X0 t       (x0 < X0, t < TT)     pass 2: TX x TT 2D DFT over (q, t)
//   ky = k' + 32 j,  kx = t' + TT s            pass 3: X0-point DFT over x0
// with the twiddles W_M^{q k'} after pass 1 and W_M^{x0 t'} after pass 2:
//   X[k'+32j][t'+TT s] = sum_x0 W_X0^{x0 s} W_M^{x0 t'} sum_t W_TT^{t t'}
//                        sum_q W_TX^{q j} W_M^{q k'} sum_k W_32^{k k'} z[q+TX k][x0+X0 t]
// Every pass works on 32 complex values per thread, so a block of
// NT = M^2/32 threads holds the whole frame in registers.  Both twiddles are
// uniform across a warp (q = tid / M in pass 1, x0 = tid / 32 in pass 2), so
// a shared-memory copy of the tables serves them as broadcasts; loads from
// shared memory cannot be hoisted across the pass barriers, which keeps the
// register footprint of forward + inverse under the 128-register cap of a
// 512-thread block.
//
// Layouts (all conflict-free for 8-byte accesses; verified by enumeration):
//   pass 1 : thread tid = q*M + x holds v[k]        = z[q + TX k][x]
//   pass 2 : thread tid = x0*32 + k' holds v[t*TX+q]
//   pass 3 : thread tid holds v[c*X0 + s] = X[ky][kx] with t' = tid % TT,
//            ky = tid / TT + (NT/TT) c, kx = t' + TT s,  c < C3 = 32 / X0
//   exchange 1 slot (rho = q*M + x, k') at rho*33 + k'   (pitch 33: every
//     address is a per-thread base plus an immediate)
//   exchange 2 slot (x0, t', ky)        at (x0*TT + t')*M + (ky ^ (t'*16/TT))
#pragma once

#include "sharp_common.cuh"
#include "twiddle_tables.cuh"

namespace sharp {

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// b * exp(DIR * 2 pi i e / 32); DIR = -1 forward, +1 inverse.
template <int DIR>
__device__ __forceinline__ float2 rot32(float2 b, int e) {
    e &= 31;
    if (e == 0) return b;
    if (e == 16) return make_float2(-b.x, -b.y);
    if (e == 8) return DIR < 0 ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x);
    if (e == 24) return DIR < 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
    const float c = cos32(e);
    const float s = DIR < 0 ? -sin32(e) : sin32(e);
    return make_float2(fmaf(b.x, c, -b.y * s), fmaf(b.x, s, b.y * c));
}

// In-register radix-2 DIT DFT of N <= 32 points v[off + i*str], natural
// order in and out, unnormalised.  All indices are compile-time after
// unrolling, so the values stay in registers.
template <int N, int DIR, int L>
__device__ __forceinline__ void dft_reg(float2 (&v)[L], int off, int str) {
    float2 t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[bitrev(i, N)] = v[off + i * str];
#pragma unroll
    for (int half = 1; half < N; half <<= 1) {
#pragma unroll
        for (int base = 0; base < N; base += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float2 a = t[base + k];
                const float2 b = rot32<DIR>(t[base + k + half], k * (32 / (2 * half)));
                t[base + k] = cadd(a, b);
                t[base + k + half] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[off + i * str] = t[i];
}

template <int M>
struct Fft3 {
    static constexpr int TX = M / 32;
    static constexpr int NT = M * M / 32;
    static constexpr int TT = 32 / TX;
    static constexpr int X0 = M / TT;
    static constexpr int C3 = 32 / X0;
    static constexpr int SW2 = 16 / TT;
    static constexpr int SMEM_ELEMS = NT * 33;   // exchange buffer, float2 (>= M*M)
    static_assert(M == 64 || M == 128, "frame size without a single-block FFT");

    static constexpr int TW1 = TX * 32;       // entries of the pass-1 twiddle table
    static constexpr int TW2 = X0 * TT;       // entries of the pass-2 twiddle table
    __device__ static __forceinline__ const float2* tw1_const() {
        if constexpr (M == 64) return c_tw1_64; else return c_tw1_128;
    }
    __device__ static __forceinline__ const float2* tw2_const() {
        if constexpr (M == 64) return c_tw2_64; else return c_tw2_128;
    }
    // Copy both twiddle tables into shared memory (tw: TW1 + TW2 float2).
    // Callers synchronise before the first transform.
    __device__ static __forceinline__ void load_twiddles(float2* tw) {
        for (int i = threadIdx.x; i < TW1; i += NT) tw[i] = tw1_const()[i];
        for (int i = threadIdx.x; i < TW2; i += NT) tw[TW1 + i] = tw2_const()[i];
    }
    __device__ static __forceinline__ int s1(int rho, int k) { return rho * 33 + k; }
    __device__ static __forceinline__ int s2(int x0, int tp, int ky) {
        return (x0 * TT + tp) * M + (ky ^ ((tp * SW2) & 15));
    }
    // pass-3 coordinates of register c*X0 + s
    __device__ static __forceinline__ int p3_ky(int c) { return threadIdx.x / TT + (NT / TT) * c; }
    __device__ static __forceinline__ int p3_kx(int s) { return threadIdx.x % TT + TT * s; }

    // pass-1 layout in, pass-3 layout out (raw DFT).
    __device__ static __forceinline__ void forward(float2 (&v)[32], float2* S, const float2* tw) {
        const int tid = threadIdx.x;
        const float2* t1 = tw;
        const float2* t2 = tw + TW1;
        // pass 1
        {
            const int q = tid / M;
            dft_reg<32, -1>(v, 0, 1);
#pragma unroll
            for (int k = 1; k < 32; ++k) v[k] = cmul(v[k], t1[q * 32 + k]);
            __syncthreads();  // previous users of S are done
#pragma unroll
            for (int k = 0; k < 32; ++k) S[s1(tid, k)] = v[k];
        }
        __syncthreads();
        // pass 2
        {
            const int x0 = tid >> 5, kp = tid & 31;
#pragma unroll
            for (int t = 0; t < TT; ++t)
#pragma unroll
                for (int q = 0; q < TX; ++q) v[t * TX + q] = S[s1(q * M + x0 + X0 * t, kp)];
            __syncthreads();
#pragma unroll
            for (int t = 0; t < TT; ++t) dft_reg<TX, -1>(v, t * TX, 1);
#pragma unroll
            for (int j = 0; j < TX; ++j) dft_reg<TT, -1>(v, j, TX);
#pragma unroll
            for (int tp = 1; tp < TT; ++tp) {
                const float2 w = t2[x0 * TT + tp];
#pragma unroll
                for (int j = 0; j < TX; ++j) v[tp * TX + j] = cmul(v[tp * TX + j], w);
            }
#pragma unroll
            for (int tp = 0; tp < TT; ++tp)
#pragma unroll
                for (int j = 0; j < TX; ++j) S[s2(x0, tp, kp + 32 * j)] = v[tp * TX + j];
        }
        __syncthreads();
        // pass 3
        {
            const int tp = tid % TT;
#pragma unroll
            for (int c = 0; c < C3; ++c)
#pragma unroll
                for (int x0 = 0; x0 < X0; ++x0) v[c * X0 + x0] = S[s2(x0, tp, p3_ky(c))];
#pragma unroll
            for (int c = 0; c < C3; ++c) dft_reg<X0, -1>(v, c * X0, 1);
        }
    }

    // pass-3 layout in, pass-1 layout out; unnormalised inverse (adjoint of
    // forward), so inverse(forward(z)) = M^2 z.
    __device__ static __forceinline__ void inverse(float2 (&v)[32], float2* S, const float2* tw) {
        const int tid = threadIdx.x;
        const float2* t1 = tw;
        const float2* t2 = tw + TW1;
        {
            const int tp = tid % TT;
#pragma unroll
            for (int c = 0; c < C3; ++c) dft_reg<X0, +1>(v, c * X0, 1);
            __syncthreads();  // all pass-3 reads of S are done
#pragma unroll
            for (int c = 0; c < C3; ++c)
#pragma unroll
                for (int x0 = 0; x0 < X0; ++x0) S[s2(x0, tp, p3_ky(c))] = v[c * X0 + x0];
        }
        __syncthreads();
        {
            const int x0 = tid >> 5, kp = tid & 31;
#pragma unroll
            for (int tp = 0; tp < TT; ++tp) {
                const float2 w = t2[x0 * TT + tp];
#pragma unroll
                for (int j = 0; j < TX; ++j) {
                    const float2 s = S[s2(x0, tp, kp + 32 * j)];
                    v[tp * TX + j] = tp == 0 ? s : cmulc(w, s);
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < TX; ++j) dft_reg<TT, +1>(v, j, TX);
#pragma unroll
            for (int t = 0; t < TT; ++t) dft_reg<TX, +1>(v, t * TX, 1);
#pragma unroll
            for (int t = 0; t < TT; ++t)
#pragma unroll
                for (int q = 0; q < TX; ++q) S[s1(q * M + x0 + X0 * t, kp)] = v[t * TX + q];
        }
        __syncthreads();
        {
            const int q = tid / M;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float2 s = S[s1(tid, k)];
                v[k] = k == 0 ? s : cmulc(t1[q * 32 + k], s);
            }
            dft_reg<32, +1>(v, 0, 1);
        }
    }
};

}  // namespace sharp
