// Persistent fused RAAR frame pass (Sec. 2.2 RAAR update, Eqs. 5, 7-9).
//
// For frame i with state c_i and measured amplitudes a_i:
//   z   = w_f . psi_y(r + x_i) + c_i                      split Q (Eq. 5)
//   Z   = F z                                             Eq. 2
//   Z'  = a Z/|Z|                                         P_a (Eq. 7); eps_a partials
//   c_i <- F* [(1-2b) Z' + b Z] = (1-2b) P_a z + b z       RAAR state
//   C(r + x_i) += conj(w) c_i                             Q* of the new state
// Because c_new = (1-2b) P_a z + b z, Q* c_new = (1-2b) A + b B with
// A = Q* P_a z and B = Q* z, so the image pass recovers A = (C - b B)/(1-2b)
// and forms psi = A/D, psi_y = (2b A - b B)/D; B/D is the previous object
// unless the probe changed (then B is scattered here from z).  Transforming
// the combination instead of Z' alone means the epilogue needs neither the old
// state nor a second gather: each frame is read once and written once.
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

template <int M, int FLAGS, int WRAP>
__global__ void __launch_bounds__(Fft3<M>::NT, M == 64 ? 3 : 1) raar_kernel(const FrameArgs a) {
    using G = Fft3<M>;
    using R = RaarGeo<M>;
    constexpr int NT = G::NT;
    constexpr int TX = G::TX;
    constexpr int MM = M * M;
    constexpr int CH = 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* tw = reinterpret_cast<float2*>(smem_raw + R::S_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + R::S_BYTES + R::TW_BYTES);
    __shared__ float red[32 * 5];

    const int tid = threadIdx.x;
    const int q = tid / M;
    const int x = tid % M;
    const float inv_m = 1.0f / M;
    const float b = a.beta;
    const float cp = 1.f - 2.f * b;

    G::load_twiddles(tw);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    auto issue_c = [&](int f) {
        mbar_expect_tx(&bars[0], (unsigned)(MM * sizeof(float2)));
        bulk_g2s_hint(S, a.c + (size_t)f * MM, (unsigned)(MM * sizeof(float2)), &bars[0], pol_stream);
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
    unsigned par_c = 0;
    bool c_pending = cur < a.K;   // uniform across the block
    bool ok = true;

    while (cur < a.K) {
        const int i = cur;
        if (tid == 0) s_next = atomicAdd(a.counter, 1);
        const int py = a.pos[2 * i];
        const int px = a.pos[2 * i + 1];
        const size_t fo = (size_t)i * MM;
        float2 v[32];

        if (tid == 0) bulk_prefetch_l2(a.amp + fo, (unsigned)(MM * sizeof(float)));

        // ---------------------------------------------- state arrives (TMA)
        ok = __syncthreads_and(mbar_wait(&bars[0], par_c));
        if (!ok) break;
        par_c ^= 1u;
        c_pending = false;
        const int nxt = s_next;   // published before the barrier above

        // ---------------------------------------------- z = w_f . psi_y + c
        // Per chunk of CH rows: issue every load first, then compute, then
        // store (a store ahead of the next row's loads would serialise them).
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += CH) {
            float2 wf[CH], yv[CH], pv[CH], ev[CH];
#pragma unroll
            for (int k = k0; k < k0 + CH; ++k) {
                const int y = q + TX * k;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
                wf[k - k0] = ld_hint(a.w_form + y * M + x, pol_keep);
                yv[k - k0] = ld_hint(a.psiy + o, pol_keep);
                if constexpr (FLAGS & RF_METRIC) {
                    pv[k - k0] = ld_hint(a.psi + o, pol_keep);
                    ev[k - k0] = a.read_e ? ld_hint(a.ebuf + fo + y * M + x, pol_stream) : make_float2(0.f, 0.f);
                }
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
#pragma unroll
                for (int k = k0; k < k0 + CH; ++k) {
                    const int y = q + TX * k;
                    const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
                    red_hint(a.accB + o, cmulc(ld_hint(a.w_proj + y * M + x, pol_keep), v[k]), pol_keep);
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

        G::forward(v, S, tw);

        // ---------------------------------------------- Fourier domain
        // Y = ((1-2b) a Z/|Z| + b Z) / m on the unitary scale, so the raw
        // inverse returns c_new directly; phase 1 where Z = 0.
        const float* ai = a.amp + fo;
        {
            // all 32 amplitude loads in flight at once, then the arithmetic
            float av[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) av[j] = __ldcs(ai + G::p3_ky(j / G::X0) * M + G::p3_kx(j % G::X0));
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float2& X = v[j];
                const float m2 = cabs2(X);
                const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                const float d = av[j] - m2 * rs * inv_m;
                acc[0] += d * d;
                acc[1] += av[j] * av[j];
                X = m2 > 0.f ? cscale(X, fmaf(cp * av[j], rs, b * inv_m) * inv_m)
                             : make_float2(cp * av[j] * inv_m, 0.f);
            }
        }

        G::inverse(v, S, tw);

        fence_proxy_async_smem();
        __syncthreads();                       // exchange buffer free
        if (nxt < a.K) {
            if (tid == 0) issue_c(nxt);
            c_pending = true;
        }

        // ---------------------------------------------- epilogue: store, scatter
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += CH) {
            float2 wp[CH];
#pragma unroll
            for (int k = k0; k < k0 + CH; ++k) wp[k - k0] = ld_hint(a.w_proj + (q + TX * k) * M + x, pol_keep);
#pragma unroll
            for (int k = k0; k < k0 + CH; ++k) {
                const int y = q + TX * k;
                const int o = obj_index(py, px, y, x, a.ny, a.nx, WRAP);
                const float2 cn = v[k];
                st_hint(a.c + fo + y * M + x, cn, pol_stream);
                red_hint(a.accA + o, cmulc(wp[k - k0], cn), pol_keep);
                if (a.write_e) red_hint(a.ebuf + fo + y * M + x, cn, pol_stream);
            }
            chunk_fence_r();
        }
        cur = nxt;
    }

    if (!ok) {
        // A wait gave up: drain (bounded) whatever copies this block may still
        // have in flight, flag the failure, and leave the sums alone.
        if (c_pending) mbar_wait(&bars[0], par_c);
        if (tid == 0) atomicExch(a.err, SHARP_ERR_TIMEOUT);
        return;
    }
    block_sum<NT, 5>(acc, red);
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < 5; ++j) atomicAdd(a.sums + j, (double)acc[j]);
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
