// RAAR frame pass with the frame transforms as DFT-matrix contractions on the
// fifth-generation tensor cores (tcgen05, TMEM accumulators), 128 x 128
// frames, in two mixed-precision modes:
//   SHARP_PREC_FP16S  : FP16 operands scaled per frame by powers of two, one
//                       product per real matrix product: the input of each
//                       transform so that its largest component maps into
//                       [2^14, 2^15), the input of the transform's second
//                       contraction by 2^-4 (a component of a unitary
//                       128-point transform is at most sqrt(2 * 128) = 16
//                       times the largest input component, so the operand
//                       stays below 2^15 with no pass over the intermediate;
//                       FP16 rounding is relative, so the smaller range costs
//                       no precision);
//   SHARP_PREC_BF16X3 : BF16 operands split x = hi + lo, three products
//                       hi.hi + hi.lo + lo.hi per real matrix product;
// both accumulated in FP32 in tensor memory.
//
// The step computes the same quantities as the FP32 frame pass (Sec. 2.2 RAAR
// update; Eqs. 2, 5, 7-9; metrics of Eqs. 11-13):
//   z   = w_f . psi_y(r + x_i) + c_i
//   Z   = F z F^T                 (F the unitary m x m DFT matrix of Eq. 2, F^T = F)
//   U   = (1-2b) a Z/|Z| + b Z    (phase 1 where Z = 0)
//   c_i <- F* U F*^T
//   C(r + x_i) += conj(w) c_i
// and, as the standalone data projection P_a of Eq. 7, out = F* (a Z/|Z|) F*^T.
//
// A 2D transform is two contractions with the roles of the frame's indices
// swapped, so every intermediate leaves tensor memory already in the layout
// the next contraction reads:
//   stage 1: D1[k1][n2] = sum_n1 F[k1][n1]  z[n1][n2]      (B rows = n2)
//   stage 2: D2[k2][k1] = sum_n2 F[k2][n2]  D1[k1][n2]     = Z[k1][k2]
//   stage 3: D3[n1][k2] = sum_k1 F*[n1][k1] U[k1][k2]      (B rows = k2)
//   stage 4: D4[n2][n1] = sum_k2 F*[n2][k2] D3[n1][k2]     = c_new[n1][n2]
// A (the DFT matrix) is M x K with K-major rows and sits in shared memory for
// the whole launch; B of each stage is written by the threads from tensor
// memory (TMEM lane = B row, TMEM column = K) into shared memory in the
// canonical no-swizzle K-major layout, converted to FP16 / BF16 on the way.
// A complex product is four real ones, D_r = A_r B_r -+ A_i B_i and
// D_i = A_r B_i +- A_i B_r (the sign of the A_i terms through the
// instruction's negate-A bit: forward F, inverse F*).
//
// Thread layout.  A block of 512 threads (16 warps, one block per SM) walks
// its frames one at a time.  Thread t owns TMEM lane r = 32 (w % 4) + lane
// and, in each of the two K-chunks j of 64 columns, the CW = 16 columns
// 64 j + 16 (w / 4) + [0, 16); in frame coordinates that is one column index
// n2 = r (coalesced global accesses across a warp) and 32 row indices.  (Two
// independent 256-thread frame groups per block, each transforming in place
// in 256 TMEM columns, were measured no faster than one block-wide pipeline:
// the memory phases of the two groups share the SM's outstanding requests.)
// Stages alternate between two 256-column TMEM regions P and Q (z in P ->
// D1 in Q -> D2 in P -> D3 in Q -> D4 in P; real part in columns 0-127 of a
// region, imaginary part in 128-255).
//  - FP16S: B holds both K-chunks of a stage (64 KB), so the second chunk is
//    converted while the MMAs of the first run.  The frame's input (state,
//    or the frames of P_a) is copied into shared memory by two bulk copies
//    (rows 0-63 into a staging buffer, rows 64-127 into the B buffer, idle
//    from the last MMA of one frame to the first conversion of the next),
//    issued when the previous frame's epilogue starts.
//  - BF16X3: its operands are twice as large (hi and lo parts), so B holds
//    one K-chunk at a time; the input frame is read by the threads after an
//    L2 prefetch issued at the previous epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sharp_common.cuh"
#include "tcgen05.cuh"

namespace sharp {

template <int PREC>
struct MixGeo {
    static constexpr int M = 128;
    static constexpr int NT = 512;
    static constexpr bool F16 = PREC == SHARP_PREC_FP16S;
    static constexpr int NW = NT / 32;                  // warps
    static constexpr int CW = 64 / (NW / 4);            // columns per thread per K-chunk (16)
    static constexpr int NPART = F16 ? 2 : 4;           // operand parts: {re, im} or {re_hi, re_lo, im_hi, im_lo}
    static constexpr int NBUF = F16 ? 2 : 1;            // K-chunks of 64 held in B at once
    static constexpr int A_PART = M * M * 2;            // 32 KB: one 128 x 128 16-bit matrix
    static constexpr int B_PART = M * 64 * 2;           // 16 KB: 128 rows x one K-chunk of 64
    static constexpr int A_BYTES = NPART * A_PART;
    static constexpr int B_SLOT = NPART * B_PART;
    static constexpr int B_BYTES = NBUF * B_SLOT;
    // FP16S stages each frame's input (state or frames, complex64) in shared
    // memory by TMA: rows 0-63 in CBUF, rows 64-127 in the B buffer, which is
    // idle between the last contraction of one frame and the first of the next
    static constexpr bool STAGE = F16;
    static constexpr int CBUF = STAGE ? 64 * M * 8 : 0;
    static_assert(!STAGE || B_BYTES == 64 * M * 8, "the B buffer holds the second half of a staged frame");
    static constexpr int SMEM = A_BYTES + B_BYTES + CBUF + 128;
    static constexpr uint32_t LBO = 16 * 128;           // K-adjacent core matrices (16 row groups of 128 B)
    static constexpr uint32_t SBO = 128;                // row-group-adjacent core matrices
    static_assert(SMEM <= 232448, "shared memory of one block");
    static_assert(SMEM > 232448 / 2, "one block per SM: the kernel allocates all 512 TMEM columns");
    static_assert(CW % 16 == 0, "TMEM accesses of 16 columns");
};


// FP16S scale of the second contraction of a transform: its operand is the
// first contraction's output, whose components are at most 16 times the
// largest (scaled, < 2^15) input component.
constexpr float kMixStage2Scale = 0.0625f;

// Power of two 2^e with mx 2^e in [2^14, 2^15) (1 for 0, Inf or NaN).
__device__ __forceinline__ float mix_pow2_scale(float mx) {
    if (!(mx > 0.f) || !(mx < 3.0e38f)) return 1.f;
    const int ex = ((__float_as_int(mx) >> 23) & 0xff) - 127;
    int e = 14 - ex;
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_h2(float x, float y) {
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_b2(__nv_bfloat16 x, __nv_bfloat16 y) {
    __nv_bfloat162 h;
    h.x = x;
    h.y = y;
    return *reinterpret_cast<const uint32_t*>(&h);
}
// hi and lo BF16 parts of (x, y), packed
__device__ __forceinline__ void split_b2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 hx = __float2bfloat16_rn(x), hy = __float2bfloat16_rn(y);
    hi = pack_b2(hx, hy);
    lo = pack_b2(__float2bfloat16_rn(x - __bfloat162float(hx)), __float2bfloat16_rn(y - __bfloat162float(hy)));
}

// Per-thread state of the pipeline.
struct MixCtx {
    uint32_t sA;           // shared address of the DFT matrix parts
    uint32_t sB;           // shared address of the B buffer
    uint32_t tbase;        // TMEM base (lane 0, column 0)
    uint32_t tl;           // TMEM address of this warp's lane quarter
    int r, h;              // TMEM lane (frame index owned) and column group
    bool leader;           // issues the MMAs and the bulk copies (thread 0)
    uint64_t* bar;         // MMA completion
    float* s_max;          // one float per warp
    unsigned phase;
    unsigned polls;        // poll limit of the first wait on each completion
    bool mma_pending;      // a commit has not been waited for (uniform)
};

// Largest value over the block (all threads receive it).
template <int PREC>
__device__ __forceinline__ float mix_block_max(const MixCtx& x, float v) {
    using G = MixGeo<PREC>;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) x.s_max[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = x.s_max[0];
#pragma unroll
    for (int k = 1; k < G::NW; ++k) m = fmaxf(m, x.s_max[k]);
    return m;
}

// Columns of this thread in K-chunk j.
template <int PREC>
__device__ __forceinline__ int mix_col(int j, int h) { return 64 * j + MixGeo<PREC>::CW * h; }

// Write 16 K-values of this thread (row r of B, K-groups kg and kg + 1 of a
// K-chunk) of the real and imaginary planes, times g, into B buffer sb.
template <int PREC>
__device__ __forceinline__ void mix_put16(uint32_t sb, int r, int kg, const float (&re)[16], const float (&im)[16],
                                          float g) {
    using G = MixGeo<PREC>;
    const uint32_t base = (uint32_t)((kg * 16 + (r >> 3)) * 128 + (r & 7) * 16);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const uint32_t off = base + u * G::LBO;
        const float* pr = re + 8 * u;
        const float* pi = im + 8 * u;
        if constexpr (G::F16) {
            sts128(sb + off, pack_h2(pr[0] * g, pr[1] * g), pack_h2(pr[2] * g, pr[3] * g),
                   pack_h2(pr[4] * g, pr[5] * g), pack_h2(pr[6] * g, pr[7] * g));
            sts128(sb + G::B_PART + off, pack_h2(pi[0] * g, pi[1] * g), pack_h2(pi[2] * g, pi[3] * g),
                   pack_h2(pi[4] * g, pi[5] * g), pack_h2(pi[6] * g, pi[7] * g));
        } else {
            uint32_t h4[4], l4[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) split_b2(pr[2 * t] * g, pr[2 * t + 1] * g, h4[t], l4[t]);
            sts128(sb + off, h4[0], h4[1], h4[2], h4[3]);
            sts128(sb + G::B_PART + off, l4[0], l4[1], l4[2], l4[3]);
#pragma unroll
            for (int t = 0; t < 4; ++t) split_b2(pi[2 * t] * g, pi[2 * t + 1] * g, h4[t], l4[t]);
            sts128(sb + 2 * G::B_PART + off, h4[0], h4[1], h4[2], h4[3]);
            sts128(sb + 3 * G::B_PART + off, l4[0], l4[1], l4[2], l4[3]);
        }
    }
}

// MMAs of K-chunk j of one stage (thread 0): D (columns d, d + 128)
// (+)= F(or F*)[:, 64 j .. 64 j + 63] . B(chunk in sb)^T.
template <int PREC>
__device__ __forceinline__ void mix_issue(uint32_t sA, uint32_t sb, uint32_t d, int j, bool inverse) {
    using G = MixGeo<PREC>;
    constexpr int BF = G::F16 ? 0 : 1;
    constexpr uint32_t ID_POS = idesc_f16(BF, 0, 128, 128);
    constexpr uint32_t ID_NEG = idesc_f16(BF, 1, 128, 128);
    const uint32_t id_ai_r = inverse ? ID_POS : ID_NEG;   // sign of A_i B_i in D_r
    const uint32_t id_ai_i = inverse ? ID_NEG : ID_POS;   // sign of A_i B_r in D_i
    const uint32_t dr = d, di = d + 128;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int kk = 4 * j + s;
        const uint32_t acc0 = (j > 0 || s > 0) ? 1u : 0u;
        auto ad = [&](int part) { return smem_desc(sA + part * G::A_PART + kk * 2 * G::LBO, G::LBO, G::SBO); };
        auto bd = [&](int part) { return smem_desc(sb + part * G::B_PART + s * 2 * G::LBO, G::LBO, G::SBO); };
        if constexpr (G::F16) {   // A: 0 F_r, 1 F_i;  B: 0 re, 1 im
            mma_f16_ss(dr, ad(0), bd(0), ID_POS, acc0);
            mma_f16_ss(dr, ad(1), bd(1), id_ai_r, 1u);
            mma_f16_ss(di, ad(0), bd(1), ID_POS, acc0);
            mma_f16_ss(di, ad(1), bd(0), id_ai_i, 1u);
        } else {                  // A: 0 F_r hi, 1 F_r lo, 2 F_i hi, 3 F_i lo;  B: 0 re hi, 1 re lo, 2 im hi, 3 im lo
            auto prod = [&](uint32_t dd, int a0, int b0, uint32_t id, uint32_t acc) {
                mma_f16_ss(dd, ad(a0), bd(b0), id, acc);
                mma_f16_ss(dd, ad(a0), bd(b0 + 1), id, 1u);
                mma_f16_ss(dd, ad(a0 + 1), bd(b0), id, 1u);
            };
            prod(dr, 0, 0, ID_POS, acc0);
            prod(dr, 2, 2, id_ai_r, 1u);
            prod(di, 0, 2, ID_POS, acc0);
            prod(di, 2, 0, id_ai_i, 1u);
        }
    }
}

// Convert this thread's CW columns of K-chunk j of region `src`, times g,
// into B buffer sb (16 columns at a time).
template <int PREC>
__device__ __forceinline__ void mix_convert(const MixCtx& x, uint32_t src, int j, uint32_t sb, float g) {
    using G = MixGeo<PREC>;
    const int c = mix_col<PREC>(j, x.h);
#pragma unroll
    for (int s = 0; s < G::CW / 16; ++s) {
        float re[16], im[16];
        tmem_ld16x2(x.tl + src + c + 16 * s, x.tl + src + 128 + c + 16 * s, re, im);
        mix_put16<PREC>(sb, x.r, (G::CW / 8) * x.h + 2 * s, re, im, g);
    }
}

// Wait (bounded) for the issued MMAs; false if the wait gave up.  The leader
// polls the mbarrier; the other threads wait at the block barrier and order
// their later TMEM accesses after it.
template <int PREC>
__device__ __forceinline__ bool mix_wait(MixCtx& x) {
    const bool ok = __syncthreads_and(x.leader ? mbar_wait(x.bar, x.phase, x.polls) : true);
    if (!ok) return false;
    x.mma_pending = false;
    x.phase ^= 1u;
    tc_fence_after();
    return true;
}

// One contraction stage: region dst = F(or F*) . (g * region src)^T in the
// stage layout above.  False if an MMA completion wait gave up.
template <int PREC>
__device__ __forceinline__ bool mix_stage(MixCtx& x, uint32_t src, uint32_t dst, bool inverse, float g) {
    using G = MixGeo<PREC>;
    if constexpr (G::NBUF == 2) {
        // both K-chunks in their own buffers: chunk 1 is converted while the
        // MMAs of chunk 0 run (src != dst)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            mix_convert<PREC>(x, src, j, x.sB + j * G::B_SLOT, g);
            fence_proxy_async_smem();   // generic-proxy writes -> tensor-core (async proxy) reads
            tc_fence_before();
            __syncthreads();
            if (x.leader) {
                tc_fence_after();
                mix_issue<PREC>(x.sA, x.sB + j * G::B_SLOT, x.tbase + dst, j, inverse);
                if (j == 1) mma_commit(x.bar);
            }
        }
        x.mma_pending = true;
        return mix_wait<PREC>(x);
    } else {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            mix_convert<PREC>(x, src, j, x.sB, g);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (x.leader) {
                tc_fence_after();
                mix_issue<PREC>(x.sA, x.sB, x.tbase + dst, j, inverse);
                mma_commit(x.bar);
            }
            x.mma_pending = true;
            if (!mix_wait<PREC>(x)) return false;
        }
        return true;
    }
}

// FP16S contraction stage in place: region r = F(or F*) . (g * region r)^T.
// Both K-chunks of the source are converted into the B buffer before any MMA
// writes the region.  False if the MMA completion wait gave up.
template <int PREC>
__device__ __forceinline__ bool mix_stage_ip(MixCtx& x, uint32_t r, bool inverse, float g) {
    using G = MixGeo<PREC>;
    static_assert(G::NBUF == 2, "in-place stages need both K-chunks in shared memory");
#pragma unroll
    for (int j = 0; j < 2; ++j) mix_convert<PREC>(x, r, j, x.sB + j * G::B_SLOT, g);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (x.leader) {
        tc_fence_after();
#pragma unroll
        for (int j = 0; j < 2; ++j) mix_issue<PREC>(x.sA, x.sB + j * G::B_SLOT, x.tbase + r, j, inverse);
        mma_commit(x.bar);
    }
    x.mma_pending = true;
    return mix_wait<PREC>(x);
}

template <int PREC, int MODE, int FLAGS, int WRAP>
__global__ void __launch_bounds__(512, 1) raar_mixed_kernel(const FrameArgs ap) {
    using G = MixGeo<PREC>;
    constexpr int M = 128;
    constexpr int MM = M * M;
    constexpr int CW = G::CW;
    constexpr bool RAAR = MODE == MODE_RAAR;
    extern __shared__ __align__(128) unsigned char mix_smem[];
    __shared__ FrameArgs a;
    __shared__ __align__(8) uint64_t bar;    // MMAs completed
    __shared__ __align__(8) uint64_t cbar;   // staged frame input arrived
    __shared__ __align__(8) uint64_t abar;   // staged amplitudes arrived
    __shared__ uint32_t s_tmem;
    __shared__ float s_max[16];
    __shared__ float red[32 * 5];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    MixCtx x;
    x.sA = (smem_addr(mix_smem) + 127u) & ~127u;
    x.sB = x.sA + G::A_BYTES;
    x.r = 32 * (warp & 3) + lane;
    x.h = warp >> 2;
    x.leader = tid == 0;
    x.bar = &bar;
    x.s_max = s_max;
    x.phase = 0;
    x.polls = wait_polls(ap.spin);
    x.mma_pending = false;

    {   // DFT matrix parts, already in the operand layout, into shared memory
        const uint4* src = reinterpret_cast<const uint4*>(ap.dft_tab);
        uint4* dst = reinterpret_cast<uint4*>(mix_smem + (x.sA - smem_addr(mix_smem)));
        for (int k = tid; k < G::A_BYTES / 16; k += G::NT) dst[k] = __ldg(src + k);
    }
    if (tid == 0) {
        a = ap;
        mbar_init(&bar, 1);
        mbar_init(&cbar, 1);
        mbar_init(&abar, 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    x.tbase = s_tmem;
    x.tl = x.tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    // TMEM regions: stages alternate between P = 0 and Q = 256
    const uint32_t RA = 0u;
    const uint32_t RB = 256u;
    unsigned char* const sbase = mix_smem + (x.sA - smem_addr(mix_smem));
    const float2* const stage_lo = reinterpret_cast<const float2*>(sbase + G::A_BYTES + G::B_BYTES);
    const float2* const stage_hi = reinterpret_cast<const float2*>(sbase + G::A_BYTES);

    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const float b = RAAR ? a.beta : 0.f;
    const float cp = 1.f - 2.f * b;
    const int xcol = x.r;   // frame column n2 owned by this thread
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;   // an amplitude that is not finite and non-negative
    bool ok = true;

    // The frame inputs streamed from HBM (state or input frames, eps_Delta
    // buffer) of the block's next frame are prefetched into L2 when the block
    // starts the epilogue of its current frame (a whole frame ahead they were
    // evicted again before use), so that the load phase's per-thread loads
    // mostly wait on L2 rather than on HBM.
    // FP16S instead copies the whole input frame into shared memory (two bulk
    // copies of 64 rows) at the same point, and the load phase reads it there.
    unsigned cpar = 0;
    bool st_pending = false;                  // uniform across the block
    // FP16S also stages the frame's amplitudes (64 KB) in the first staging
    // buffer, free from the end of the load phase to the next frame's input
    // copy, by one bulk copy issued before the forward contractions, so the
    // Fourier step reads them from shared memory.
    float* const stage_amp = reinterpret_cast<float*>(const_cast<float2*>(stage_lo));
    unsigned apar = 0;
    bool am_pending = false;                  // uniform across the block
    auto stage_frame = [&](int f) {           // leader only
        const float2* src = (RAAR ? a.c : a.zin) + (size_t)f * MM;
        mbar_expect_tx(&cbar, (unsigned)(MM * sizeof(float2)));
        bulk_g2s_hint(const_cast<float2*>(stage_lo), src, (unsigned)(64 * M * sizeof(float2)), &cbar, pol_stream);
        bulk_g2s_hint(const_cast<float2*>(stage_hi), src + 64 * M, (unsigned)(64 * M * sizeof(float2)), &cbar,
                      pol_stream);
    };
    auto prefetch_frame = [&](int f) {
        if (f >= a.K) return;
        if constexpr (G::STAGE) {
            if constexpr (RAAR && (FLAGS & RF_METRIC))
                if (a.read_e) bulk_prefetch_l2(a.ebuf + (size_t)f * MM, (unsigned)(MM * sizeof(float2)));
            stage_frame(f);
            return;
        }
        const size_t o = (size_t)f * MM;
        if constexpr (RAAR) {
            bulk_prefetch_l2(a.c + o, (unsigned)(MM * sizeof(float2)));
            if constexpr (FLAGS & RF_METRIC)
                if (a.read_e) bulk_prefetch_l2(a.ebuf + o, (unsigned)(MM * sizeof(float2)));
        } else {
            bulk_prefetch_l2(a.zin + o, (unsigned)(MM * sizeof(float2)));
        }
    };
    if (x.leader) prefetch_frame(blockIdx.x);
    if constexpr (G::STAGE) st_pending = (int)blockIdx.x < a.K;

    for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
        const size_t fo = (size_t)i * MM;
        if (x.leader) bulk_prefetch_l2(a.amp + fo, (unsigned)(MM * sizeof(float)));
        const int py = RAAR ? a.pos[2 * i] : 0;
        const int px = RAAR ? a.pos[2 * i + 1] : 0;

        // ------------------------------------------------ load: z into RA
        if constexpr (G::STAGE) {
            ok = __syncthreads_and(mbar_wait(&cbar, cpar, x.polls));
            if (!ok) break;
            cpar ^= 1u;
            st_pending = false;
        }
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll 1
            for (int hh = 0; hh < CW / 8; ++hh) {
                const int y0 = mix_col<PREC>(j, x.h) + 8 * hh;
                float zr[8], zi[8];
                if constexpr (RAAR) {
                    float2 cv[8], wf[8], yv[8], wp[8], pv[8], ev[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int y = y0 + k;
                        const int o = obj_index(py, px, y, xcol, a.ny, a.nx, WRAP);
                        if constexpr (G::STAGE) cv[k] = (j == 0 ? stage_lo : stage_hi)[(y - 64 * j) * M + xcol];
                        else cv[k] = ld_hint(a.c + fo + y * M + xcol, pol_stream);
                        wf[k] = ld_hint(a.w_form + y * M + xcol, pol_keep);
                        yv[k] = ld_hint(a.psiy + o, pol_keep);
                        if constexpr (FLAGS & RF_FORM_B) wp[k] = ld_hint(a.w_proj + y * M + xcol, pol_keep);
                        if constexpr (FLAGS & (RF_METRIC | RF_FORM_B)) pv[k] = ld_hint(a.psi + o, pol_keep);
                        if constexpr (FLAGS & RF_METRIC)
                            ev[k] = a.read_e ? ld_hint(a.ebuf + fo + y * M + xcol, pol_stream)
                                             : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int y = y0 + k;
                        const float2 wy = cmul(wf[k], yv[k]);
                        const float2 z = cadd(wy, cv[k]);
                        zr[k] = z.x;
                        zi[k] = z.y;
                        acc[2] += cabs2(z);
                        if constexpr (FLAGS & RF_METRIC) {
                            acc[3] += cabs2(csub(cmul(wf[k], pv[k]), z));
                            acc[4] += cabs2(cadd(wy, ev[k]));
                        }
                        if constexpr (FLAGS & RF_FORM_B) {
                            const int o = obj_index(py, px, y, xcol, a.ny, a.nx, WRAP);
                            if (!a.no_scatter)
                                red_hint(a.accB + o, cmulc(wp[k], csub(z, cmul(wp[k], pv[k]))), pol_keep);
                        }
                        if (a.write_e) st_hint(a.ebuf + fo + y * M + xcol, make_float2(-z.x, -z.y), pol_stream);
                    }
                } else {
                    float2 zv[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if constexpr (G::STAGE) zv[k] = (j == 0 ? stage_lo : stage_hi)[(y0 + k - 64 * j) * M + xcol];
                        else zv[k] = ld_hint(a.zin + fo + (y0 + k) * M + xcol, pol_stream);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        zr[k] = zv[k].x;
                        zi[k] = zv[k].y;
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) mx = fmaxf(mx, fmaxf(fabsf(zr[k]), fabsf(zi[k])));
                tmem_st8x2(x.tl + RA + y0, x.tl + RA + 128 + y0, zr, zi);
            }
        }
        tmem_wait_st();
        float g0 = 1.f, g1 = 1.f, g2 = 1.f, g3 = 1.f;
        if constexpr (G::F16) g0 = mix_pow2_scale(mix_block_max<PREC>(x, mx));
        if constexpr (G::STAGE) {   // every thread has read its staged input (block max above)
            if (x.leader) {
                mbar_expect_tx(&abar, (unsigned)(MM * sizeof(float)));
                bulk_g2s_hint(stage_amp, a.amp + fo, (unsigned)(MM * sizeof(float)), &abar, pol_stream);
            }
            am_pending = true;
        }

        // ------------------------------------------------ forward transform
        ok = mix_stage<PREC>(x, RA, RB, false, g0);
        if (!ok) break;
        if constexpr (G::F16) g1 = kMixStage2Scale;
        ok = mix_stage<PREC>(x, RB, RA, false, g1);
        if (!ok) break;

        // ------------------------------------------------ Fourier step on RA
        {
            const float inv = 1.f / (g0 * g1);   // exact: powers of two
            float um = 0.f;
            if constexpr (G::STAGE) {
                ok = __syncthreads_and(mbar_wait(&abar, apar, x.polls));
                if (!ok) break;
                apar ^= 1u;
                am_pending = false;
            }
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int s = 0; s < CW / 16; ++s) {
                    const int k0 = mix_col<PREC>(j, x.h) + 16 * s;
                    float re[16], im[16];
                    tmem_ld16x2(x.tl + RA + k0, x.tl + RA + 128 + k0, re, im);
                    float av[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        av[t] = G::STAGE ? stage_amp[(k0 + t) * M + xcol] : __ldcs(a.amp + fo + (size_t)(k0 + t) * M + xcol);
#pragma unroll
                    for (int t = 0; t < 16; ++t) {   // U in place of Z
                        const float X = re[t] * inv, Y = im[t] * inv;
                        const float m2 = fmaf(X, X, Y * Y);
                        const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                        const float d = av[t] - m2 * rs;
                        acc[0] += d * d;
                        acc[1] += av[t] * av[t];
                        bad |= (int)bad_amplitude(av[t]);
                        if (m2 > 0.f) {
                            const float f = fmaf(cp * av[t], rs, b);
                            re[t] = X * f;
                            im[t] = Y * f;
                        } else {
                            re[t] = cp * av[t];
                            im[t] = 0.f;
                        }
                        um = fmaxf(um, fmaxf(fabsf(re[t]), fabsf(im[t])));
                    }
                    float r8[8], i8[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) { r8[t] = re[t]; i8[t] = im[t]; }
                    tmem_st8x2(x.tl + RA + k0, x.tl + RA + 128 + k0, r8, i8);
#pragma unroll
                    for (int t = 0; t < 8; ++t) { r8[t] = re[8 + t]; i8[t] = im[8 + t]; }
                    tmem_st8x2(x.tl + RA + k0 + 8, x.tl + RA + 128 + k0 + 8, r8, i8);
                }
            }
            tmem_wait_st();
            if constexpr (G::F16) g2 = mix_pow2_scale(mix_block_max<PREC>(x, um));
        }

        // ------------------------------------------------ inverse transform
        ok = mix_stage<PREC>(x, RA, RB, true, g2);
        if (!ok) break;
        if constexpr (G::F16) g3 = kMixStage2Scale;
        ok = mix_stage<PREC>(x, RB, RA, true, g3);
        if (!ok) break;

        // ------------------------------------------------ epilogue from RA
        // (the staging buffers are free: the load phase is done and the last
        // contraction's MMAs, which read the B buffer, have completed)
        if (x.leader) prefetch_frame(i + gridDim.x);
        if constexpr (G::STAGE) st_pending = i + (int)gridDim.x < a.K;
        {
            const float inv = 1.f / (g2 * g3);
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int s = 0; s < CW / 16; ++s) {
                    const int y0 = mix_col<PREC>(j, x.h) + 16 * s;
                    float re[16], im[16];
                    tmem_ld16x2(x.tl + RA + y0, x.tl + RA + 128 + y0, re, im);
                    if constexpr (RAAR) {
                        {
                            // C' += conj(w) (c_new - (1-b) w psi), relative to the object
                            const float rho = 1.f - a.beta;
#pragma unroll
                            for (int hf = 0; hf < 2; ++hf) {
                            float2 wp[8], pv[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                wp[k] = ld_hint(a.w_proj + (y0 + 8 * hf + k) * M + xcol, pol_keep);
                                pv[k] = ld_hint(a.psi + obj_index(py, px, y0 + 8 * hf + k, xcol, a.ny, a.nx, WRAP), pol_keep);
                            }
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int t = 8 * hf + k;
                                const int y = y0 + t;
                                const int o = obj_index(py, px, y, xcol, a.ny, a.nx, WRAP);
                                const float2 cn = make_float2(re[t] * inv, im[t] * inv);
                                st_hint(a.c + fo + y * M + xcol, cn, pol_stream);
                                if (!a.no_scatter)
                                    red_hint(a.accA + o, cmulc(wp[k], csub(cn, cscale(cmul(wp[k], pv[k]), rho))),
                                             pol_keep);
                                if (a.write_e) red_hint(a.ebuf + fo + y * M + xcol, cn, pol_stream);
                            }
                            }
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < 16; ++t)
                            st_hint(a.zout + fo + (y0 + t) * M + xcol, make_float2(re[t] * inv, im[t] * inv),
                                    pol_stream);
                    }
                }
            }
        }
        // each thread only touches its own lane and columns of the region,
        // so the next frame's load phase may overwrite them in program order
    }

    // A wait gave up: wait (bounded, full limit) once more for MMAs whose
    // commit was not waited for and for a staging copy still in flight, so
    // that nothing writes TMEM or shared memory after the block has left.
    if (x.mma_pending && x.leader) mbar_wait(x.bar, x.phase);
    if (st_pending && x.leader) mbar_wait(&cbar, cpar);
    if (am_pending && x.leader) mbar_wait(&abar, apar);
    const bool all_ok = __syncthreads_and(ok);
    if (!all_ok) {
        if (tid == 0) atomicExch(a.err, SHARP_ERR_TIMEOUT);   // flag the failure, leave the sums alone
    } else {
        if (__syncthreads_or(bad) && tid == 0) raise_error(a.err, SHARP_ERR_INVALID_ARG);
        block_sum<G::NT, 5>(acc, red);
        if (tid == 0) {
            if constexpr (RAAR) {
#pragma unroll
                for (int j = 0; j < 5; ++j) atomicAdd(a.sums + j, (double)acc[j]);
            } else {
                atomicAdd(a.sums, (double)acc[0]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(x.tbase, 512);
    }
}

template <int PREC, int MODE, int FLAGS, int WRAP>
static cudaError_t launch_mixed_one(const FrameArgs& a, cudaStream_t s) {
    using G = MixGeo<PREC>;
    auto kern = raar_mixed_kernel<PREC, MODE, FLAGS, WRAP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = a.K < sms ? a.K : sms;
    kern<<<grid, G::NT, G::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_mixed_prec(int mode, int flags, const FrameArgs& a, cudaStream_t s) {
    if (mode == MODE_PROJECT) return launch_mixed_one<PREC, MODE_PROJECT, 0, 0>(a, s);
    if (mode != MODE_RAAR) return cudaErrorInvalidValue;
    const int f = flags & (RF_FORM_B | RF_METRIC);
    if (a.wrap) {
        switch (f) {
            case 0: return launch_mixed_one<PREC, MODE_RAAR, 0, 1>(a, s);
            case RF_FORM_B: return launch_mixed_one<PREC, MODE_RAAR, RF_FORM_B, 1>(a, s);
            case RF_METRIC: return launch_mixed_one<PREC, MODE_RAAR, RF_METRIC, 1>(a, s);
            default: return launch_mixed_one<PREC, MODE_RAAR, RF_FORM_B | RF_METRIC, 1>(a, s);
        }
    }
    switch (f) {
        case 0: return launch_mixed_one<PREC, MODE_RAAR, 0, 0>(a, s);
        case RF_FORM_B: return launch_mixed_one<PREC, MODE_RAAR, RF_FORM_B, 0>(a, s);
        case RF_METRIC: return launch_mixed_one<PREC, MODE_RAAR, RF_METRIC, 0>(a, s);
        default: return launch_mixed_one<PREC, MODE_RAAR, RF_FORM_B | RF_METRIC, 0>(a, s);
    }
}

}  // namespace sharp
