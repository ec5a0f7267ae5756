// Persistent fused RAAR frame pass (Sec. 2.2 RAAR update, Eqs. 5, 7-9).
//
// For frame i with state c_i and measured amplitudes a_i:
//   z   = w_f . psi_y(r + x_i) + c_i                      split Q (Eq. 5)
//   Z   = F z                                             Eq. 2
//   Z'  = a Z/|Z|                                         P_a (Eq. 7); eps_a partials
//   c_i <- F* [(1-2b) Z' + b Z] = (1-2b) P_a z + b z       RAAR state
//   C'(r + x_i) += conj(w) (c_i - (1-b) w psi(r + x_i))    Q* of the new state,
//                                                          relative to the object
// Because c_new = (1-2b) P_a z + b z, Q* c_new = (1-2b) A + b B with
// A = Q* P_a z and B = Q* z, so the image pass recovers
// A/D = psi + (C' - b B')/((1-2b) D) and psi_y = (2b A - b B)/D, where
// B' = Q*(z - w psi) is zero unless the probe changed (then it is scattered
// here from z).  The sums are taken relative to w psi so that near
// convergence they hold small corrections: FP32 rounding of the overlap sums
// then stays far below the step-to-step change instead of being amplified
// by 1/|1-2b| from the full-size sums.  Transforming the combination instead
// of Z' alone means the epilogue needs neither the old state nor the old
// iterate: each frame is read once and written once.
//
// One persistent block per SM walks frames i = blockIdx.x + k * gridDim.x.
// Frame i+1's state is copied by TMA (one cp.async.bulk of m^2 complex values)
// into the FFT exchange buffer while frame i finishes its epilogue; its
// completion is tracked by an mbarrier with a bounded wait.  Each frame's
// amplitudes are prefetched into L2 by a bulk prefetch when the frame starts
// and read by the Fourier phase.  L2 policies keep the object, probe and
// overlap images resident (evict_last) while the streamed state and
// amplitudes go first (evict_first).
#pragma once

#include "fft_frame.cuh"
#include "sharp_common.cuh"
#include "tma.cuh"

namespace sharp {

template <int M>
struct RaarGeo {
    using G = Fft3<M>;
    static constexpr size_t S_BYTES = sizeof(float2) * G::SMEM_ELEMS;
    static constexpr size_t TW_BYTES = sizeof(float2) * (G::TW1 + G::TW2);
    static constexpr size_t SMEM = S_BYTES + TW_BYTES + 2 * sizeof(uint64_t);
    static_assert(S_BYTES >= sizeof(float2) * M * M, "state staging must fit the exchange buffer");
    static_assert((S_BYTES + TW_BYTES) % 8 == 0, "mbarrier alignment");
};

__device__ __forceinline__ void chunk_fence_r() { asm volatile("" ::: "memory"); }

template <class T>
__device__ __forceinline__ T ldg_plain(const T* p) { return *p; }

// ------------------------------------------------------------------ phases
// The three per-frame phases, shared by the single-scan and the batch kernel.
// `a` is the scan's arguments (kernel parameter or a shared-memory copy).

// z = w_f . psi_y(r + x_i) + c_i into v (pass-1 layout); c_i is in S.
// CH rows are loaded per round trip (a tile parameter of the batch tuner).
template <int M, int FLAGS, int WRAP, int CH = 8>
__device__ __forceinline__ void raar_load_phase(const FrameArgs& a, int py, int px, size_t fo, const float2* S,
                                                float2 (&v)[32], float (&acc)[5], uint64_t pol_stream,
                                                uint64_t pol_keep) {
    constexpr int TX = Fft3<M>::TX;
    static_assert(32 % CH == 0, "row chunks divide the 32 rows of a thread");
    const int q = threadIdx.x / M;
    const int x = threadIdx.x % M;
    // Per chunk of CH rows: issue every load first, then compute, then store
    // (a store ahead of the next row's loads would serialise them).
#pragma unroll
    for (int k0 = 0; k0 < 32; k0 += CH) {
        float2 wf[CH], yv[CH], pv[CH], ev[CH], wp[CH];
#pragma unroll
        for (int k = k0; k < k0 + CH; ++k) {
            const int y = q + TX * k;
            const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
            wf[k - k0] = ld_hint(a.w_form + y * M + x, pol_keep);
            yv[k - k0] = ld_hint(a.psiy + o, pol_keep);
            if constexpr (FLAGS & RF_FORM_B) wp[k - k0] = ld_hint(a.w_proj + y * M + x, pol_keep);
            if constexpr (FLAGS & (RF_METRIC | RF_FORM_B)) pv[k - k0] = ld_hint(a.psi + o, pol_keep);
            if constexpr (FLAGS & RF_METRIC)
                ev[k - k0] = a.read_e ? ld_hint(a.ebuf + fo + y * M + x, pol_stream) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = k0; k < k0 + CH; ++k) {
            const int y = q + TX * k;
            const float2 wy = cmul(wf[k - k0], yv[k - k0]);
            const float2 z = cadd(wy, S[y * M + x]);
            v[k] = z;
            acc[2] += cabs2(z);
            if constexpr (FLAGS & RF_METRIC) {
                acc[3] += cabs2(csub(cmul(wf[k - k0], pv[k - k0]), z));
                acc[4] += cabs2(cadd(wy, ev[k - k0]));
            }
        }
        if constexpr (FLAGS & RF_FORM_B) {
            if (!a.no_scatter) {
#pragma unroll
                for (int k = k0; k < k0 + CH; ++k) {
                    const int y = q + TX * k;
                    const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
                    red_hint(a.accB + o, cmulc(wp[k - k0], csub(v[k], cmul(wp[k - k0], pv[k - k0]))), pol_keep);
                }
            }
        }
        if (a.write_e) {
#pragma unroll
            for (int k = k0; k < k0 + CH; ++k) {
                const int y = q + TX * k;
                st_hint(a.ebuf + fo + y * M + x, make_float2(-v[k].x, -v[k].y), pol_stream);
            }
        }
        chunk_fence_r();
    }
}

// Y = ((1-2b) a Z/|Z| + b Z) / m on the unitary scale (pass-3 layout), so the
// raw inverse returns c_new directly; phase 1 where Z = 0.  `bad` collects
// amplitudes that are not finite and non-negative.
template <int M>
__device__ __forceinline__ void raar_fourier_phase(const FrameArgs& a, size_t fo, float2 (&v)[32],
                                                   float (&acc)[5], int& bad) {
    using G = Fft3<M>;
    const float inv_m = 1.0f / M;
    const float b = a.beta;
    const float cp = 1.f - 2.f * b;
    const float* ai = a.amp + fo;
    // all 32 amplitude loads in flight at once, then the arithmetic
    float av[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) av[j] = __ldcs(ai + G::p3_ky(j / G::X0) * M + G::p3_kx(j % G::X0));
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

// Store c_new and scatter C' += conj(w_p) (c_new - (1-b) w_p psi) (pass-1
// layout), CH rows per round trip.
template <int M, int WRAP, int CH = 8>
__device__ __forceinline__ void raar_epilogue(const FrameArgs& a, int py, int px, size_t fo, const float2 (&v)[32],
                                              uint64_t pol_stream, uint64_t pol_keep) {
    constexpr int TX = Fft3<M>::TX;
    const int q = threadIdx.x / M;
    const int x = threadIdx.x % M;
    const float rho = 1.f - a.beta;
#pragma unroll
    for (int k0 = 0; k0 < 32; k0 += CH) {
        float2 wp[CH], pv[CH];
#pragma unroll
        for (int k = k0; k < k0 + CH; ++k) {
            const int y = q + TX * k;
            wp[k - k0] = ld_hint(a.w_proj + y * M + x, pol_keep);
            pv[k - k0] = ld_hint(a.psi + obj_index(py, px, y, x, a.ny, a.nx, WRAP), pol_keep);
        }
#pragma unroll
        for (int k = k0; k < k0 + CH; ++k) {
            const int y = q + TX * k;
            const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
            const float2 cn = v[k];
            st_hint(a.c + fo + y * M + x, cn, pol_stream);
            const float2 dn = csub(cn, cscale(cmul(wp[k - k0], pv[k - k0]), rho));
            if (!a.no_scatter) red_hint(a.accA + o, cmulc(wp[k - k0], dn), pol_keep);
            if (a.write_e) red_hint(a.ebuf + fo + y * M + x, cn, pol_stream);
        }
        chunk_fence_r();
    }
}

// ------------------------------------------------------------------ single scan
template <int M, int FLAGS, int WRAP>
__global__ void __launch_bounds__(Fft3<M>::NT, M == 64 ? 3 : 1) raar_kernel(const FrameArgs ap) {
    using G = Fft3<M>;
    using R = RaarGeo<M>;
    constexpr int NT = G::NT;
    constexpr int MM = M * M;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tw = reinterpret_cast<float2*>(smem_raw + R::S_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + R::S_BYTES + R::TW_BYTES);
    __shared__ float red[32 * 5];
    // Arguments served from shared memory: the compiler re-reads them where
    // needed instead of holding pointers in registers (it spills much less).
    __shared__ FrameArgs a;
    const int tid = threadIdx.x;

    G::load_twiddles(tw);
    if (tid == 0) {
        a = ap;
        mbar_init(&bars[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    auto issue_c = [&](int f) {
        mbar_expect_tx(&bars[0], (unsigned)(MM * sizeof(float2)));
        bulk_g2s_hint(S, a.c + (size_t)f * MM, (unsigned)(MM * sizeof(float2)), &bars[0], pol_stream);
        // the eps_Delta buffer the load phase will read (a frame ahead, so the
        // chunked loads hit L2 instead of making four round trips to HBM)
        if (FLAGS & RF_METRIC)
            if (a.read_e) bulk_prefetch_l2(a.ebuf + (size_t)f * MM, (unsigned)(MM * sizeof(float2)));
    };
    // Frames are handed out by an atomic counter.  Blocks start staggered by
    // a fraction of a frame time so that the SMs' memory phases (gathers,
    // scatter, state stores) interleave instead of all hitting the memory
    // system at once.
    __shared__ int s_next;
    if (tid == 0) {
        __nanosleep(2000u * (blockIdx.x & 3u));
        const int f = atomicAdd(a.counter, 1);
        s_next = f;
        if (f < a.K) issue_c(f);
    }
    __syncthreads();
    int cur = s_next;

    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    unsigned par_c = 0;
    bool c_pending = cur < a.K;   // uniform across the block
    bool ok = true;
    const unsigned polls = wait_polls(a.spin);

    while (cur < a.K) {
        const int i = cur;
        if (tid == 0) s_next = atomicAdd(a.counter, 1);
        const int py = a.pos[2 * i];
        const int px = a.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;
        float2 v[32];

        if (tid == 0) bulk_prefetch_l2(a.amp + fo, (unsigned)(MM * sizeof(float)));

        // ---------------------------------------------- state arrives (TMA)
        ok = __syncthreads_and(mbar_wait(&bars[0], par_c, polls));
        if (!ok) break;
        par_c ^= 1u;
        c_pending = false;
        const int nxt = s_next;   // published before the barrier above

        raar_load_phase<M, FLAGS, WRAP>(a, py, px, fo, S, v, acc, pol_stream, pol_keep);
        G::forward(v, S, tw);
        raar_fourier_phase<M>(a, fo, v, acc, bad);
        G::inverse(v, S, tw);

        fence_proxy_async_smem();
        __syncthreads();                       // exchange buffer free
        if (nxt < a.K) {
            if (tid == 0) issue_c(nxt);
            c_pending = true;
        }
        raar_epilogue<M, WRAP>(a, py, px, fo, v, pol_stream, pol_keep);
        cur = nxt;
    }

    if (!ok) {
        // A wait gave up: drain (bounded, full limit) whatever copies this
        // block may still have in flight, flag the failure, and leave the
        // sums alone.
        if (c_pending) mbar_wait(&bars[0], par_c);
        if (tid == 0) atomicExch(a.err, SHARP_ERR_TIMEOUT);
        return;
    }
    if (__syncthreads_or(bad) && tid == 0) raise_error(a.err, SHARP_ERR_INVALID_ARG);
    block_sum<NT, 5>(acc, red);
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < 5; ++j) atomicAdd(a.sums + j, (double)acc[j]);
    }
}

// ------------------------------------------------------------------ batch
// Frames of several independent scans of the same frame size in one
// persistent launch.  Global frame g belongs to the scan s with
// base[s] <= g < base[s+1]; the scan's arguments are copied to shared memory
// when a block moves to a frame of another scan, and the block's metric sums
// are flushed to the scan it leaves.  Scans may differ in everything but the
// frame size and the step's flags (FORM_B / METRIC are compile-time).

template <int M, int FLAGS, int CH>
__global__ void __launch_bounds__(Fft3<M>::NT, M == 64 ? 3 : 1) raar_batch_kernel(const BatchTable bt) {
    using G = Fft3<M>;
    using R = RaarGeo<M>;
    constexpr int NT = G::NT;
    constexpr int MM = M * M;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tw = reinterpret_cast<float2*>(smem_raw + R::S_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + R::S_BYTES + R::TW_BYTES);
    __shared__ float red[32 * 5];
    __shared__ FrameArgs sa;                  // arguments of the current scan
    __shared__ int s_next, s_next_scan;
    const int tid = threadIdx.x;

    G::load_twiddles(tw);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    auto scan_of = [&](int g) {               // thread 0 only
        int s = 0;
        while (s + 1 < bt.nscans && __ldg(bt.base + s + 1) <= g) ++s;
        return s;
    };
    auto issue_c = [&](int g, int s) {        // thread 0 only
        const FrameArgs& t = bt.scans[s];
        const int f = g - __ldg(bt.base + s);
        mbar_expect_tx(&bars[0], (unsigned)(MM * sizeof(float2)));
        bulk_g2s_hint(S, t.c + (size_t)f * MM, (unsigned)(MM * sizeof(float2)), &bars[0], pol_stream);
        if (FLAGS & RF_METRIC)
            if (t.read_e) bulk_prefetch_l2(t.ebuf + (size_t)f * MM, (unsigned)(MM * sizeof(float2)));
    };
    if (tid == 0) {
        __nanosleep((unsigned)bt.stagger_ns * (blockIdx.x & 3u));
        const int g = atomicAdd(bt.counter, 1);
        s_next = g;
        s_next_scan = g < bt.total ? scan_of(g) : 0;
        if (g < bt.total) issue_c(g, s_next_scan);
    }
    __syncthreads();
    int cur = s_next, cur_scan = s_next_scan, loaded_scan = -1;

    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    unsigned par_c = 0;
    bool c_pending = cur < bt.total;
    bool ok = true;

    auto flush = [&](int s) {                 // block-wide: metric sums to scan s
        if (__syncthreads_or(bad) && tid == 0) {
            raise_error(bt.scans[s].err, SHARP_ERR_INVALID_ARG);   // the scan's plan status
            raise_error(bt.err, SHARP_ERR_INVALID_ARG);
        }
        bad = 0;
        block_sum<NT, 5>(acc, red);
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 5; ++j) atomicAdd(bt.scans[s].sums + j, (double)acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] = 0.f;
    };

    while (cur < bt.total) {
        if (cur_scan != loaded_scan) {
            if (loaded_scan >= 0) flush(loaded_scan);
            __syncthreads();
            if (tid == 0) sa = bt.scans[cur_scan];
            __syncthreads();
            loaded_scan = cur_scan;
        }
        const int i = cur - __ldg(bt.base + cur_scan);
        if (tid == 0) {
            const int g = atomicAdd(bt.counter, 1);
            s_next = g;
            s_next_scan = g < bt.total ? scan_of(g) : 0;
        }
        const int py = sa.pos[2 * i];
        const int px = sa.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;
        float2 v[32];
        if (tid == 0) bulk_prefetch_l2(sa.amp + fo, (unsigned)(MM * sizeof(float)));

        ok = __syncthreads_and(mbar_wait(&bars[0], par_c, wait_polls(sa.spin)));
        if (!ok) break;
        par_c ^= 1u;
        c_pending = false;
        const int nxt = s_next, nxt_scan = s_next_scan;

        if (sa.wrap) raar_load_phase<M, FLAGS, 1, CH>(sa, py, px, fo, S, v, acc, pol_stream, pol_keep);
        else raar_load_phase<M, FLAGS, 0, CH>(sa, py, px, fo, S, v, acc, pol_stream, pol_keep);
        G::forward(v, S, tw);
        raar_fourier_phase<M>(sa, fo, v, acc, bad);
        G::inverse(v, S, tw);

        fence_proxy_async_smem();
        __syncthreads();
        if (nxt < bt.total) {
            if (tid == 0) issue_c(nxt, nxt_scan);
            c_pending = true;
        }
        if (sa.wrap) raar_epilogue<M, 1, CH>(sa, py, px, fo, v, pol_stream, pol_keep);
        else raar_epilogue<M, 0, CH>(sa, py, px, fo, v, pol_stream, pol_keep);
        cur = nxt;
        cur_scan = nxt_scan;
    }

    if (!ok) {
        if (c_pending) mbar_wait(&bars[0], par_c);
        if (tid == 0) {
            atomicExch(bt.err, SHARP_ERR_TIMEOUT);
            atomicExch(bt.scans[cur_scan].err, SHARP_ERR_TIMEOUT);   // the scan's plan status
        }
        return;
    }
    if (loaded_scan >= 0) flush(loaded_scan);
}

template <int M, int FLAGS, int CH>
static cudaError_t launch_raar_batch_one(const BatchTable& bt, int grid, cudaStream_t s) {
    using R = RaarGeo<M>;
    auto kern = raar_batch_kernel<M, FLAGS, CH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bt.counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    kern<<<grid, Fft3<M>::NT, R::SMEM, s>>>(bt);
    return cudaGetLastError();
}

// Largest useful grid of the batch kernel (resident blocks on the device).
template <int M>
cudaError_t raar_batch_max_grid(int* grid) {
    using R = RaarGeo<M>;
    auto kern = raar_batch_kernel<M, 0, 8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Fft3<M>::NT, R::SMEM)) != cudaSuccess)
        return e;
    *grid = sms * (per_sm < 1 ? 1 : per_sm);
    return cudaSuccess;
}

// All flag variants of one (frame size, row chunk) pair.
template <int M, int CH>
cudaError_t launch_raar_batch_mc(int flags, const BatchTable& bt, int grid, cudaStream_t s) {
    switch (flags & (RF_FORM_B | RF_METRIC)) {
        case 0: return launch_raar_batch_one<M, 0, CH>(bt, grid, s);
        case RF_FORM_B: return launch_raar_batch_one<M, RF_FORM_B, CH>(bt, grid, s);
        case RF_METRIC: return launch_raar_batch_one<M, RF_METRIC, CH>(bt, grid, s);
        default: return launch_raar_batch_one<M, RF_FORM_B | RF_METRIC, CH>(bt, grid, s);
    }
}

template <int M, int FLAGS, int WRAP>
static cudaError_t launch_raar_one(const FrameArgs& a, cudaStream_t s) {
    using R = RaarGeo<M>;
    auto kern = raar_kernel<M, FLAGS, WRAP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Fft3<M>::NT, R::SMEM)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (grid > a.K) grid = a.K;
    if ((e = cudaMemsetAsync(a.counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    kern<<<grid, Fft3<M>::NT, R::SMEM, s>>>(a);
    return cudaGetLastError();
}

// All flag variants of one (frame size, wrap) pair; one translation unit each.
template <int M, int WRAP>
cudaError_t launch_raar_w(int flags, const FrameArgs& a, cudaStream_t s) {
    switch (flags & (RF_FORM_B | RF_METRIC)) {
        case 0: return launch_raar_one<M, 0, WRAP>(a, s);
        case RF_FORM_B: return launch_raar_one<M, RF_FORM_B, WRAP>(a, s);
        case RF_METRIC: return launch_raar_one<M, RF_METRIC, WRAP>(a, s);
        default: return launch_raar_one<M, RF_FORM_B | RF_METRIC, WRAP>(a, s);
    }
}

}  // namespace sharp
