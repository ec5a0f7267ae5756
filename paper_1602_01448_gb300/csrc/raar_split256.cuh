// FP32 RAAR frame pass for 256 x 256 frames through four 128 x 128
// register-resident transforms (Sec. 2.2 RAAR update; Eqs. 2, 5, 7-9;
// metrics of Eqs. 11-13).
//
// The unitary 256^2 transform of Eq. 2 is split once, radix 2 in frequency
// along each axis (n = nu + 128 p, k = 2 kappa + a, omega = e^{-2 pi i/256}):
//   Z[2 kappa1 + a][2 kappa2 + b] = X_ab[kappa1][kappa2] / 256,
//   X_ab = raw (unnormalised) 128^2 DFT of
//   y_ab[nu1][nu2] = omega^(a nu1 + b nu2) sum_pq (-1)^(a p + b q) z[nu1 + 128 p][nu2 + 128 q].
// Each sub-problem (a, b) is one 128^2 frame for the register FFT of
// fft_frame.cuh (Fft3<128>: a 512-thread block holds it as 32 complex values
// per thread): forward transform, the Fourier-domain step on the frequencies
// (2 kappa1 + a, 2 kappa2 + b), whose input to the raw inverse is
// U_ab / 256 with U = (1-2b) a Z/|Z| + b Z, and the raw inverse, which then
// returns y'_ab = F128^-1(U_ab) / 2; the split is undone by
//   c[nu1 + 128 p][nu2 + 128 q] = sum_ab (-1)^(a p + b q) omega^-(a nu1 + b nu2) y'_ab[nu1][nu2].
// The load phase forms the four y_ab from the four quadrants of z at once and
// parks them in slots of 128 KB (FP32): y_00 and y_01 in the block's global
// slab, y_10 and y_11 in tensor memory (TMEM, 256 KB per SM, which this
// kernel does not need otherwise).  Entries are thread-private: the thread
// that writes an entry is the one that reads it, so no synchronisation is
// needed.  Each sub-problem takes its y_ab from its slot into registers and
// leaves y'_ab there; the final combination reads the four y'_ab and runs the
// epilogue (state store, overlap scatter relative to the object, as the other
// frame passes).  Keeping the transforms' registers free during the memory
// phases (the 32 complex values of a thread are not live there) avoids
// spills.  With half the slots in TMEM the global slab holds 256 KB per SM
// (39 MB on 152 SMs), so more of it stays in L2.
//
// TMEM layout: thread (q, nu2) of warp w reaches lane 32 (w % 4) + (lane id)
// = nu2 (t = 128 q + nu2); the four threads of a lane (q = 0..3) use column
// ranges of their own: value k of slot s in {2, 3} at column
// 256 (s - 2) + 64 q + 2 k (real part) and + 1 (imaginary part).
//
// Thread layout (Fft3<128> pass 1): thread t holds nu2 = t % 128 and the 32
// rows nu1 = t / 128 + 4 k, k < 32.  One persistent block per SM (each owns
// a 512 KB slab) takes frames from an atomic counter; the same kernel serves
// one scan (arguments as a kernel parameter) or a batch of scans (a device
// table, BatchTable; WRAP = -1 reads the wrap flag of each scan at run time),
// with LCH rows per round trip of the load phase and the epilogue (a tile
// parameter of the batch tuner).
#pragma once

#include <cstring>

#include "fft_frame.cuh"
#include "sharp_common.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace sharp {
namespace split {

constexpr int M = 256;        // frame size
constexpr int H = 128;        // sub-problem size
constexpr int MM = M * M;
constexpr int HH = H * H;
using G = Fft3<H>;
constexpr int NT = G::NT;     // 512
constexpr int TX = G::TX;     // 4 rows per row group of the thread layout
constexpr size_t S_BYTES = sizeof(float2) * G::SMEM_ELEMS;
constexpr size_t TW_BYTES = sizeof(float2) * (G::TW1 + G::TW2);
constexpr size_t SMEM = S_BYTES + TW_BYTES;

__device__ __forceinline__ void fence_s() { asm volatile("" ::: "memory"); }

}  // namespace split

template <int FLAGS, int WRAP, int LCH>
__global__ void __launch_bounds__(split::NT, 1)
raar_split256_kernel(const FrameArgs ap, const BatchTable bt, float2* slab) {
    using namespace split;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tw = reinterpret_cast<float2*>(smem_raw + S_BYTES);
    __shared__ float red[32 * 5];
    __shared__ FrameArgs a;
    __shared__ float2 s_om[M];           // omega^k, k < 256
    __shared__ int s_next, s_scan;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const bool batch = bt.scans != nullptr;
    const int total = batch ? bt.total : ap.K;
    int* const counter = batch ? bt.counter : ap.counter;
    auto scan_of = [&](int g) {          // thread 0 only
        int s = 0;
        while (s + 1 < bt.nscans && bt.base[s + 1] <= g) ++s;
        return s;
    };

    G::load_twiddles(tw);
    for (int k = tid; k < M; k += NT) {
        double sn, cs;
        sincospi(-2.0 * k / M, &sn, &cs);
        s_om[k] = make_float2((float)cs, (float)sn);
    }
    if (warp == 0) {                     // all 512 TMEM columns: slots 2 and 3
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        if (!batch) a = ap;
        __nanosleep((batch ? (unsigned)bt.stagger_ns : 2000u) * (blockIdx.x & 3u));
        const int g = atomicAdd(counter, 1);
        s_next = g;
        s_scan = (batch && g < total) ? scan_of(g) : 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int q = tid / H;               // row group
    const int nu2 = tid % H;             // quadrant column
    float2* const slot = slab + (size_t)blockIdx.x * MM;   // slots 0 and 1 (H x H each)
    auto slab_at = [&](int s, int nu1) { return slot + (size_t)s * HH + nu1 * H + nu2; };
    // TMEM column of value k of slot s (2, 3) for this thread's lane quarter
    const uint32_t tl = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)q;
    auto tcol = [&](int s, int k) { return tl + 256u * (uint32_t)(s - 2) + 2u * (uint32_t)k; };
    constexpr float inv_m = 1.0f / M;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    int cur = s_next, cur_scan = s_scan, loaded = batch ? -1 : 0;
    __syncthreads();   // everyone has read s_next before thread 0 rewrites it

    auto flush = [&]() {   // block-wide: metric sums and invalid-data flag to the current scan
        if (__syncthreads_or(bad) && tid == 0) {
            raise_error(a.err, SHARP_ERR_INVALID_ARG);
            if (batch) raise_error(bt.err, SHARP_ERR_INVALID_ARG);
        }
        bad = 0;
        block_sum<NT, 5>(acc, red);
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 5; ++j) atomicAdd(a.sums + j, (double)acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] = 0.f;
    };

    while (cur < total) {
        if (batch && cur_scan != loaded) {
            if (loaded >= 0) flush();
            __syncthreads();
            if (tid == 0) a = bt.scans[cur_scan];
            __syncthreads();
            loaded = cur_scan;
        }
        const int i = batch ? cur - bt.base[cur_scan] : cur;
        const size_t fo = (size_t)i * MM;
        if (tid == 0) {
            const int g = atomicAdd(counter, 1);
            s_next = g;
            s_scan = (batch && g < total) ? scan_of(g) : 0;
            for (int k = 0; k < 2; ++k) bulk_prefetch_l2(a.amp + fo + k * (MM / 2), (unsigned)(MM / 2 * sizeof(float)));
        }
        const int py = a.pos[2 * i];
        const int px = a.pos[2 * i + 1];
        const int wrap = WRAP >= 0 ? WRAP : a.wrap;
        const float b = a.beta;
        const float cp = 1.f - 2.f * b;
        const float rho = 1.f - b;

        // ---------------------------------------------- load: the four y_ab
        {
            constexpr int CH = (FLAGS & (RF_METRIC | RF_FORM_B)) ? 2 : LCH;   // rows per round trip
#pragma unroll 1
            for (int k0 = 0; k0 < 32; k0 += CH) {
                float2 cv[CH][4], wf[CH][4], yv[CH][4], wp[CH][4], pv[CH][4], ev[CH][4];
                float t2[2 * CH], t3[2 * CH];   // y_10, y_11 of the chunk (re, im) for TMEM
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int nu1 = q + TX * (k0 + kk);
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        const int y = nu1 + H * (pq >> 1), x = nu2 + H * (pq & 1);
                        const int o = obj_index(py, px, y, x, a.ny, a.nx, wrap);
                        cv[kk][pq] = ld_hint(a.c + fo + y * M + x, pol_stream);
                        wf[kk][pq] = ld_hint(a.w_form + y * M + x, pol_keep);
                        yv[kk][pq] = ld_hint(a.psiy + o, pol_keep);
                        if constexpr (FLAGS & RF_FORM_B) wp[kk][pq] = ld_hint(a.w_proj + y * M + x, pol_keep);
                        if constexpr (FLAGS & (RF_METRIC | RF_FORM_B)) pv[kk][pq] = ld_hint(a.psi + o, pol_keep);
                        if constexpr (FLAGS & RF_METRIC)
                            ev[kk][pq] = a.read_e ? ld_hint(a.ebuf + fo + y * M + x, pol_stream) : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    const int nu1 = q + TX * k;
                    float2 z[4];   // quadrant (p, q) at index 2 p + q
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        const int y = nu1 + H * (pq >> 1), x = nu2 + H * (pq & 1);
                        const float2 wy = cmul(wf[kk][pq], yv[kk][pq]);
                        z[pq] = cadd(wy, cv[kk][pq]);
                        acc[2] += cabs2(z[pq]);
                        if constexpr (FLAGS & RF_METRIC) {
                            acc[3] += cabs2(csub(cmul(wf[kk][pq], pv[kk][pq]), z[pq]));
                            acc[4] += cabs2(cadd(wy, ev[kk][pq]));
                        }
                        if constexpr (FLAGS & RF_FORM_B) {
                            // B' = Q*(z - w psi), relative to the object (image pass)
                            const int o = obj_index(py, px, y, x, a.ny, a.nx, wrap);
                            if (!a.no_scatter)
                                red_hint(a.accB + o, cmulc(wp[kk][pq], csub(z[pq], cmul(wp[kk][pq], pv[kk][pq]))),
                                         pol_keep);
                        }
                        if (a.write_e) st_hint(a.ebuf + fo + y * M + x, make_float2(-z[pq].x, -z[pq].y), pol_stream);
                    }
                    // quadrant butterflies, then the twiddles
                    const float2 s0 = cadd(z[0], z[1]), d0 = csub(z[0], z[1]);   // row quadrant p = 0
                    const float2 s1 = cadd(z[2], z[3]), d1 = csub(z[2], z[3]);   // p = 1
                    st_hint(slab_at(0, nu1), cadd(s0, s1), pol_keep);
                    st_hint(slab_at(1, nu1), cmul(s_om[nu2], cadd(d0, d1)), pol_keep);
                    const float2 y10 = cmul(s_om[nu1], csub(s0, s1));
                    const float2 y11 = cmul(s_om[nu1 + nu2], csub(d0, d1));
                    t2[2 * kk] = y10.x;
                    t2[2 * kk + 1] = y10.y;
                    t3[2 * kk] = y11.x;
                    t3[2 * kk + 1] = y11.y;
                }
                tmem_st_cols<2 * CH>(tcol(2, k0), t2);
                tmem_st_cols<2 * CH>(tcol(3, k0), t3);
                fence_s();
            }
            tmem_wait_st();
        }

        // ---------------------------------------------- four sub-problems
#pragma unroll 1
        for (int sub = 0; sub < 4; ++sub) {
            const int sa = sub >> 1, sb = sub & 1;
            float2 v[32];
            if (sub < 2) {
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = ld_hint(slab_at(sub, q + TX * k), pol_keep);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float ra[16], rb[16];
                    tmem_ld16x2(tcol(sub, 16 * h), tcol(sub, 16 * h + 8), ra, rb);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v[16 * h + j] = make_float2(ra[2 * j], ra[2 * j + 1]);
                        v[16 * h + 8 + j] = make_float2(rb[2 * j], rb[2 * j + 1]);
                    }
                }
            }
            G::forward(v, S, tw);
            {   // Fourier step (pass-3 layout): frequency (2 ky + a, 2 kx + b);
                // ky, kx of register j are this thread's first plus constants
                constexpr int DKY = G::NT / (32 / G::TX);   // ky step between register groups
                constexpr int TT = 32 / G::TX;               // kx step within a group
                const float* ai = a.amp + fo + (size_t)(2 * G::p3_ky(0) + sa) * M + 2 * G::p3_kx(0) + sb;
                float av[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) av[j] = __ldcs(ai + 2 * DKY * M * (j / G::X0) + 2 * TT * (j % G::X0));
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float2& X = v[j];
                    const float m2 = cabs2(X);
                    const float rs = m2 > 0.f ? rsqrt_refined(m2) : 0.f;
                    const float d = av[j] - m2 * rs * inv_m;
                    acc[0] += d * d;
                    acc[1] += av[j] * av[j];
                    bad |= (int)bad_amplitude(av[j]);
                    X = m2 > 0.f ? cscale(X, fmaf(cp * av[j], rs, b * inv_m) * inv_m)
                                 : make_float2(cp * av[j] * inv_m, 0.f);
                }
            }
            G::inverse(v, S, tw);
            if (sub < 2) {
#pragma unroll
                for (int k = 0; k < 32; ++k) st_hint(slab_at(sub, q + TX * k), v[k], pol_keep);
            } else {
#pragma unroll
                for (int k0 = 0; k0 < 32; k0 += 4) {
                    float t[8];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        t[2 * j] = v[k0 + j].x;
                        t[2 * j + 1] = v[k0 + j].y;
                    }
                    tmem_st_cols<8>(tcol(sub, k0), t);
                }
                tmem_wait_st();
            }
        }

        // ---------------------------------------------- combination + epilogue
        {
            constexpr int CH = LCH;
#pragma unroll 1
            for (int k0 = 0; k0 < 32; k0 += CH) {
                float2 u0[CH], u1[CH], u2[CH], u3[CH], wp[CH][4], pv[CH][4];
                {
                    float t2[2 * CH], t3[2 * CH];
                    tmem_ld_cols2<2 * CH>(tcol(2, k0), tcol(3, k0), t2, t3);
#pragma unroll
                    for (int kk = 0; kk < CH; ++kk) {
                        u2[kk] = make_float2(t2[2 * kk], t2[2 * kk + 1]);
                        u3[kk] = make_float2(t3[2 * kk], t3[2 * kk + 1]);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int nu1 = q + TX * (k0 + kk);
                    u0[kk] = ld_hint(slab_at(0, nu1), pol_keep);
                    u1[kk] = ld_hint(slab_at(1, nu1), pol_keep);
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        const int y = nu1 + H * (pq >> 1), x = nu2 + H * (pq & 1);
                        wp[kk][pq] = ld_hint(a.w_proj + y * M + x, pol_keep);
                        pv[kk][pq] = ld_hint(a.psi + obj_index(py, px, y, x, a.ny, a.nx, wrap), pol_keep);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int k = k0 + kk;
                    const int nu1 = q + TX * k;
                    const float2 u01 = cmulc(s_om[nu2], u1[kk]);
                    const float2 u10 = cmulc(s_om[nu1], u2[kk]);
                    const float2 u11 = cmulc(s_om[nu1 + nu2], u3[kk]);
                    const float2 e0 = cadd(u0[kk], u10), e1 = csub(u0[kk], u10);   // row quadrant p = 0, 1
                    const float2 f0 = cadd(u01, u11), f1 = csub(u01, u11);
                    float2 cn[4];
                    cn[0] = cadd(e0, f0);   // (p, q) = (0, 0)
                    cn[1] = csub(e0, f0);   // (0, 1)
                    cn[2] = cadd(e1, f1);   // (1, 0)
                    cn[3] = csub(e1, f1);   // (1, 1)
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        const int y = nu1 + H * (pq >> 1), x = nu2 + H * (pq & 1);
                        const int o = obj_index(py, px, y, x, a.ny, a.nx, wrap);
                        st_hint(a.c + fo + y * M + x, cn[pq], pol_stream);
                        // C' += conj(w) (c_new - (1-b) w psi), relative to the object
                        if (!a.no_scatter)
                            red_hint(a.accA + o,
                                     cmulc(wp[kk][pq], csub(cn[pq], cscale(cmul(wp[kk][pq], pv[kk][pq]), rho))),
                                     pol_keep);
                        if (a.write_e) red_hint(a.ebuf + fo + y * M + x, cn[pq], pol_stream);
                    }
                }
                fence_s();
            }
        }
        __syncthreads();   // s_next is read below and rewritten by thread 0 next frame
        cur = s_next;
        cur_scan = s_scan;
        __syncthreads();
    }
    if (loaded >= 0) flush();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(s_tmem, 512);
    }
}

// One launch: a single scan (bt null: grid = min(K, SMs)) or a batch (grid
// given, at most one block per SM: each block owns a slab).
template <int FLAGS, int WRAP, int LCH>
static cudaError_t launch_split256_one(const FrameArgs& a, const BatchTable* bt, int grid, float2* slab,
                                       cudaStream_t s) {
    auto kern = raar_split256_kernel<FLAGS, WRAP, LCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    BatchTable t;
    memset(&t, 0, sizeof(t));
    if (bt) t = *bt;
    const int total = bt ? bt->total : a.K;
    int* counter = bt ? bt->counter : a.counter;
    if (grid <= 0 || grid > sms) grid = sms;
    if (grid > total) grid = total;
    if (grid <= 0) return cudaSuccess;
    if (!slab || !counter) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    kern<<<grid, split::NT, split::SMEM, s>>>(a, t, slab);
    return cudaGetLastError();
}

}  // namespace sharp
