// Tensor-core precision modes for 256 x 256 frames: the RAAR frame pass and
// the data projection P_a (Sec. 2.2 RAAR update; Eqs. 2, 5, 7-9; metrics of
// Eqs. 11-13) with the frame DFTs as FP16 (per-frame scaled) or BF16x3
// contractions with the 128 x 128 DFT matrix on tcgen05, FP32 accumulation in
// tensor memory (the contraction stages of raar_mixed.cuh).
//
// A 256^2 frame's FP32 accumulators (512 KB) exceed an SM's tensor memory
// (256 KB), so the unitary 256-point transform along each axis is split once,
// radix 2 in frequency: with n = nu + 128 p and k = 2 kappa + a (p, a in
// {0, 1}), omega = e^{-2 pi i / 256} and W = omega^2,
//   Z[2 kappa1 + a][2 kappa2 + b]
//     = 1/2 F128(y_ab)[kappa1][kappa2],
//   y_ab[nu1][nu2] = omega^(a nu1 + b nu2) sum_pq (-1)^(a p + b q) z[nu1 + 128 p][nu2 + 128 q],
// F128 the unitary 128^2 transform (128 = sqrt(256 * 256) / 2 accounts for
// the 1/2).  Each of the four sub-problems (a, b) is one 128^2 transform
// pair in tensor memory, exactly the 128^2 frame of raar_mixed.cuh: forward
// contractions, the Fourier-domain step on the frequencies (2 kappa1 + a,
// 2 kappa2 + b), inverse contractions.  The inverse undoes the split:
//   c[nu1 + 128 p][nu2 + 128 q]
//     = 1/2 sum_ab (-1)^(a p + b q) omega^-(a nu1 + b nu2) F128^-1(U_ab)[nu1][nu2].
// Both ends of the split need all four sub-problems at one (nu1, nu2): the
// load phase forms all four y_ab from the four quadrants of z; the final
// combination of the four inverse results also runs the epilogue (state
// store, overlap scatter relative to the object, as the FP32 frame pass).
// Sub-problems wait in the block's slab (FP32, 128 KB per slot,
// thread-private entries, so no synchronisation is needed between writer and
// reader):
//  - BF16X3 (out-of-place stages through both TMEM regions): y_00 in P,
//    y_01 / y_10 / y_11 in slots 1-3; the inverse results of the first three
//    sub-problems go back to slots 0-2, the last stays in P.
//  - FP16S (in-place stages, one region per sub-problem): y_00 in P, y_01 in
//    Q, y_10 / y_11 in slots 0 / 1; before sub-problem 1b the finished 0b
//    swaps places with it (region <-> slot b), so two slots suffice and the
//    final combination reads 00 and 01 from the slab, 10 and 11 from P and Q.
//
// Thread layout and TMEM regions as in raar_mixed.cuh: thread t owns lane
// r = nu2 (frame column within a quadrant) and 32 row indices nu1; regions P
// (columns 0-255) and Q (256-511), real then imaginary planes.
#pragma once

#include "raar_mixed.cuh"

namespace sharp {

template <int PREC, int MODE, int FLAGS, int WRAP>
__global__ void __launch_bounds__(512, 1) raar_mixed256_kernel(const FrameArgs ap, float2* slab) {
    using G = MixGeo<PREC>;
    constexpr int M = 256;        // frame size
    constexpr int H = 128;        // sub-problem size
    constexpr int MM = M * M;
    constexpr int HH = H * H;
    constexpr int CW = G::CW;
    constexpr bool RAAR = MODE == MODE_RAAR;
    constexpr int SMEM_MAIN = G::A_BYTES + G::B_BYTES;
    extern __shared__ __align__(128) unsigned char mix_smem[];
    __shared__ FrameArgs a;
    __shared__ __align__(8) uint64_t bar;    // MMAs completed
    __shared__ uint32_t s_tmem;
    __shared__ float s_max[16];
    __shared__ float red[32 * 5];
    __shared__ float2 s_om[M];               // omega^k, k < 256
    const int tid = threadIdx.x, warp = tid >> 5;

    MixCtx x;
    x.sA = (smem_addr(mix_smem) + 127u) & ~127u;
    x.sB = x.sA + G::A_BYTES;
    x.r = 32 * (warp & 3) + (tid & 31);
    x.h = warp >> 2;
    x.leader = tid == 0;
    x.bar = &bar;
    x.s_max = s_max;
    x.phase = 0;
    x.polls = wait_polls(ap.spin);
    x.mma_pending = false;
    static_assert(SMEM_MAIN + 128 <= 232448, "shared memory of one block");

    {   // the 128 x 128 DFT matrix parts, already in the operand layout
        const uint4* src = reinterpret_cast<const uint4*>(ap.dft_tab);
        uint4* dst = reinterpret_cast<uint4*>(mix_smem + (x.sA - smem_addr(mix_smem)));
        for (int k = tid; k < G::A_BYTES / 16; k += G::NT) dst[k] = __ldg(src + k);
    }
    for (int k = tid; k < M; k += G::NT) {
        double sn, cs;
        sincospi(-2.0 * k / M, &sn, &cs);
        s_om[k] = make_float2((float)cs, (float)sn);
    }
    if (tid == 0) {
        a = ap;
        mbar_init(&bar, 1);
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
    const uint32_t RA = 0u;
    const uint32_t RB = 256u;

    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const float b = RAAR ? a.beta : 0.f;
    const float cp = 1.f - 2.f * b;
    const int nu2 = x.r;                      // quadrant column owned by this thread
    float2* const slot = slab + (size_t)blockIdx.x * MM;   // 4 slots of H x H
    auto slab_at = [&](int s, int nu1) { return slot + (size_t)s * HH + nu1 * H + nu2; };
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    bool ok = true;

    auto prefetch_frame = [&](int f) {         // leader: the frame's streamed input into L2
        if (f >= a.K) return;
        const float2* src = (RAAR ? a.c : a.zin) + (size_t)f * MM;
        for (int k = 0; k < 4; ++k) bulk_prefetch_l2(src + k * (MM / 4), (unsigned)(MM / 4 * sizeof(float2)));
    };
    if (x.leader) prefetch_frame(blockIdx.x);

    for (int i = blockIdx.x; i < a.K; i += gridDim.x) {
        const size_t fo = (size_t)i * MM;
        if (x.leader)
            for (int k = 0; k < 2; ++k)
                bulk_prefetch_l2(a.amp + fo + k * (MM / 2), (unsigned)(MM / 2 * sizeof(float)));
        const int py = RAAR ? a.pos[2 * i] : 0;
        const int px = RAAR ? a.pos[2 * i + 1] : 0;

        // ---------------------------------------------- load: the four y_ab
        // y_00 into P; FP16S: y_01 into Q, y_10 / y_11 into slab slots 0 / 1;
        // BF16X3: y_01 / y_10 / y_11 into slab slots 1-3
        float mx = 0.f, mx1 = 0.f;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll 1
            for (int hh = 0; hh < CW / 8; ++hh) {
                const int n0 = mix_col<PREC>(j, x.h) + 8 * hh;
                float zr[8], zi[8], zr1[8], zi1[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int nu1 = n0 + k;
                    float2 z[4];   // quadrant (p, q) at index 2 p + q
                    if constexpr (RAAR) {
                        float2 cv[4], wf[4], yv[4], wp[4], pv[4], ev[4];
#pragma unroll
                        for (int pq = 0; pq < 4; ++pq) {
                            const int y = nu1 + H * (pq >> 1), xx = nu2 + H * (pq & 1);
                            const int o = obj_index(py, px, y, xx, a.ny, a.nx, WRAP);
                            cv[pq] = ld_hint(a.c + fo + y * M + xx, pol_stream);
                            wf[pq] = ld_hint(a.w_form + y * M + xx, pol_keep);
                            yv[pq] = ld_hint(a.psiy + o, pol_keep);
                            if constexpr (FLAGS & RF_FORM_B) wp[pq] = ld_hint(a.w_proj + y * M + xx, pol_keep);
                            if constexpr (FLAGS & (RF_METRIC | RF_FORM_B)) pv[pq] = ld_hint(a.psi + o, pol_keep);
                            if constexpr (FLAGS & RF_METRIC)
                                ev[pq] = a.read_e ? ld_hint(a.ebuf + fo + y * M + xx, pol_stream)
                                                  : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int pq = 0; pq < 4; ++pq) {
                            const int y = nu1 + H * (pq >> 1), xx = nu2 + H * (pq & 1);
                            const float2 wy = cmul(wf[pq], yv[pq]);
                            z[pq] = cadd(wy, cv[pq]);
                            acc[2] += cabs2(z[pq]);
                            if constexpr (FLAGS & RF_METRIC) {
                                acc[3] += cabs2(csub(cmul(wf[pq], pv[pq]), z[pq]));
                                acc[4] += cabs2(cadd(wy, ev[pq]));
                            }
                            if constexpr (FLAGS & RF_FORM_B) {
                                const int o = obj_index(py, px, y, xx, a.ny, a.nx, WRAP);
                                if (!a.no_scatter)
                                    red_hint(a.accB + o, cmulc(wp[pq], csub(z[pq], cmul(wp[pq], pv[pq]))), pol_keep);
                            }
                            if (a.write_e)
                                st_hint(a.ebuf + fo + y * M + xx, make_float2(-z[pq].x, -z[pq].y), pol_stream);
                        }
                    } else {
#pragma unroll
                        for (int pq = 0; pq < 4; ++pq)
                            z[pq] = ld_hint(a.zin + fo + (nu1 + H * (pq >> 1)) * M + nu2 + H * (pq & 1), pol_stream);
                    }
                    // butterflies over the quadrants, then the twiddles
                    const float2 s0 = cadd(z[0], z[1]), d0 = csub(z[0], z[1]);   // row quadrant p = 0
                    const float2 s1 = cadd(z[2], z[3]), d1 = csub(z[2], z[3]);   // p = 1
                    const float2 y00 = cadd(s0, s1);
                    const float2 y01 = cmul(s_om[nu2], cadd(d0, d1));
                    const float2 y10 = cmul(s_om[nu1], csub(s0, s1));
                    const float2 y11 = cmul(s_om[nu1 + nu2], csub(d0, d1));
                    zr[k] = y00.x;
                    zi[k] = y00.y;
                    mx = fmaxf(mx, fmaxf(fabsf(y00.x), fabsf(y00.y)));
                    if constexpr (G::F16) {
                        zr1[k] = y01.x;
                        zi1[k] = y01.y;
                        mx1 = fmaxf(mx1, fmaxf(fabsf(y01.x), fabsf(y01.y)));
                        st_hint(slab_at(0, nu1), y10, pol_keep);
                        st_hint(slab_at(1, nu1), y11, pol_keep);
                    } else {
                        st_hint(slab_at(1, nu1), y01, pol_keep);
                        st_hint(slab_at(2, nu1), y10, pol_keep);
                        st_hint(slab_at(3, nu1), y11, pol_keep);
                    }
                }
                tmem_st8x2(x.tl + RA + n0, x.tl + RA + 128 + n0, zr, zi);
                if constexpr (G::F16) tmem_st8x2(x.tl + RB + n0, x.tl + RB + 128 + n0, zr1, zi1);
            }
        }
        tmem_wait_st();

        // ---------------------------------------------- four sub-problems
        const float rho = 1.f - b;
        // combination of the four inverse sub-problems at row nu1 (y'_ab, the
        // twiddles applied here) and the epilogue of its four frame samples
        auto finish_row = [&](int nu1, float2 y00, float2 y01, float2 y10, float2 y11) {
            const float2 u00 = y00;
            const float2 u01 = cmulc(s_om[nu2], y01);
            const float2 u10 = cmulc(s_om[nu1], y10);
            const float2 u11 = cmulc(s_om[nu1 + nu2], y11);
            const float2 e0 = cadd(u00, u10), e1 = csub(u00, u10);   // row quadrant p = 0, 1
            const float2 f0 = cadd(u01, u11), f1 = csub(u01, u11);
            float2 cn[4];
            cn[0] = cscale(cadd(e0, f0), 0.5f);   // (p, q) = (0, 0)
            cn[1] = cscale(csub(e0, f0), 0.5f);   // (0, 1)
            cn[2] = cscale(cadd(e1, f1), 0.5f);   // (1, 0)
            cn[3] = cscale(csub(e1, f1), 0.5f);   // (1, 1)
            if constexpr (RAAR) {
                float2 wp[4], pv[4];
#pragma unroll
                for (int pq = 0; pq < 4; ++pq) {
                    const int y = nu1 + H * (pq >> 1), xx = nu2 + H * (pq & 1);
                    wp[pq] = ld_hint(a.w_proj + y * M + xx, pol_keep);
                    pv[pq] = ld_hint(a.psi + obj_index(py, px, y, xx, a.ny, a.nx, WRAP), pol_keep);
                }
#pragma unroll
                for (int pq = 0; pq < 4; ++pq) {
                    const int y = nu1 + H * (pq >> 1), xx = nu2 + H * (pq & 1);
                    const int o = obj_index(py, px, y, xx, a.ny, a.nx, WRAP);
                    st_hint(a.c + fo + y * M + xx, cn[pq], pol_stream);
                    // C' += conj(w) (c_new - (1-b) w psi), relative to the object
                    if (!a.no_scatter)
                        red_hint(a.accA + o, cmulc(wp[pq], csub(cn[pq], cscale(cmul(wp[pq], pv[pq]), rho))),
                                 pol_keep);
                    if (a.write_e) red_hint(a.ebuf + fo + y * M + xx, cn[pq], pol_stream);
                }
            } else {
#pragma unroll
                for (int pq = 0; pq < 4; ++pq)
                    st_hint(a.zout + fo + (nu1 + H * (pq >> 1)) * M + nu2 + H * (pq & 1), cn[pq],
                            pol_stream);
            }
        };
        if constexpr (G::F16) {
            // Each sub-problem is transformed in place in one TMEM region (a
            // stage converts both K-chunks of its source into shared memory
            // before its MMAs overwrite it): sub-problems 00 and 10 in P, 01
            // and 11 in Q.  Before sub-problems 10 and 11 a finished
            // sub-problem leaves its region for the slab slot that held the
            // pending one, entry by entry (thread-private), scaled on the way.
            float invs[4];
#pragma unroll 1
            for (int sub = 0; sub < 4 && ok; ++sub) {
                const int sa = sub >> 1, sb = sub & 1;
                const uint32_t R = sb ? RB : RA;
                float msub = sb ? mx1 : mx;
                if (sub >= 2) {   // y'_{0 sb} out to slab slot sb, y_{1 sb} in
                    msub = 0.f;
                    const float so = invs[sub - 2];
#pragma unroll 1
                    for (int j = 0; j < 2; ++j) {
#pragma unroll 1
                        for (int hh = 0; hh < CW / 8; ++hh) {
                            const int n0 = mix_col<PREC>(j, x.h) + 8 * hh;
                            float ore[8], oim[8], zr[8], zi[8];
                            tmem_ld_cols2<8>(x.tl + R + n0, x.tl + R + 128 + n0, ore, oim);
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float2 v = ld_hint(slab_at(sb, n0 + k), pol_keep);
                                zr[k] = v.x;
                                zi[k] = v.y;
                                msub = fmaxf(msub, fmaxf(fabsf(v.x), fabsf(v.y)));
                            }
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                st_hint(slab_at(sb, n0 + k), make_float2(ore[k] * so, oim[k] * so), pol_keep);
                            tmem_st8x2(x.tl + R + n0, x.tl + R + 128 + n0, zr, zi);
                        }
                    }
                    tmem_wait_st();
                }
                const float g0 = mix_pow2_scale(mix_block_max<PREC>(x, msub));
                const float g1 = kMixStage2Scale;
                if (!(ok = mix_stage_ip<PREC>(x, R, false, g0))) break;
                if (!(ok = mix_stage_ip<PREC>(x, R, false, g1))) break;
                float g2;
                {   // Fourier step on R: lane kappa2, column kappa1 -> frequency
                    // (2 kappa1 + a, 2 kappa2 + b); Z = X / 2 on the unitary scale
                    const float inv = 0.5f / (g0 * g1);
                    float um = 0.f;
                    const int kx = 2 * nu2 + sb;
#pragma unroll 1
                    for (int j = 0; j < 2; ++j) {
#pragma unroll
                        for (int s = 0; s < CW / 16; ++s) {
                            const int k0 = mix_col<PREC>(j, x.h) + 16 * s;
                            float re[16], im[16];
                            tmem_ld16x2(x.tl + R + k0, x.tl + R + 128 + k0, re, im);
                            float av[16];
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                av[t] = __ldcs(a.amp + fo + (size_t)(2 * (k0 + t) + sa) * M + kx);
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
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
                            tmem_st8x2(x.tl + R + k0, x.tl + R + 128 + k0, r8, i8);
#pragma unroll
                            for (int t = 0; t < 8; ++t) { r8[t] = re[8 + t]; i8[t] = im[8 + t]; }
                            tmem_st8x2(x.tl + R + k0 + 8, x.tl + R + 128 + k0 + 8, r8, i8);
                        }
                    }
                    tmem_wait_st();
                    g2 = mix_pow2_scale(mix_block_max<PREC>(x, um));
                }
                const float g3 = kMixStage2Scale;
                if (!(ok = mix_stage_ip<PREC>(x, R, true, g2))) break;
                if (!(ok = mix_stage_ip<PREC>(x, R, true, g3))) break;
                invs[sub] = 1.f / (g2 * g3);
            }
            if (ok) {   // ---------------------------------- combination + epilogue
                if (x.leader) prefetch_frame(i + gridDim.x);
                const float i2 = invs[2], i3 = invs[3];
#pragma unroll 1
                for (int j = 0; j < 2; ++j) {
#pragma unroll 1
                    for (int hh = 0; hh < CW / 8; ++hh) {
                        const int n0 = mix_col<PREC>(j, x.h) + 8 * hh;
                        float are[8], aim[8], bre[8], bim[8];
                        tmem_ld_cols2<8>(x.tl + RA + n0, x.tl + RA + 128 + n0, are, aim);
                        tmem_ld_cols2<8>(x.tl + RB + n0, x.tl + RB + 128 + n0, bre, bim);
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            finish_row(n0 + t, ld_hint(slab_at(0, n0 + t), pol_keep),
                                       ld_hint(slab_at(1, n0 + t), pol_keep), make_float2(are[t] * i2, aim[t] * i2),
                                       make_float2(bre[t] * i3, bim[t] * i3));
                    }
                }
            }
        } else {
#pragma unroll 1
            for (int sub = 0; sub < 4 && ok; ++sub) {
                const int sa = sub >> 1, sb = sub & 1;
                if (sub > 0) {   // y_ab from the slab into P
                    mx = 0.f;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
#pragma unroll 1
                        for (int hh = 0; hh < CW / 8; ++hh) {
                            const int n0 = mix_col<PREC>(j, x.h) + 8 * hh;
                            float zr[8], zi[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float2 v = ld_hint(slab_at(sub, n0 + k), pol_keep);
                                zr[k] = v.x;
                                zi[k] = v.y;
                                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
                            }
                            tmem_st8x2(x.tl + RA + n0, x.tl + RA + 128 + n0, zr, zi);
                        }
                    }
                    tmem_wait_st();
                }
                float g0 = 1.f, g1 = 1.f, g2 = 1.f, g3 = 1.f;
                if constexpr (G::F16) g0 = mix_pow2_scale(mix_block_max<PREC>(x, mx));
                if (!(ok = mix_stage<PREC>(x, RA, RB, false, g0))) break;
                if constexpr (G::F16) g1 = kMixStage2Scale;
                if (!(ok = mix_stage<PREC>(x, RB, RA, false, g1))) break;

                // Fourier step on P: lane kappa2, column kappa1 -> frequency
                // (2 kappa1 + a, 2 kappa2 + b) of the frame; Z = X / 2 on the
                // unitary 256^2 scale
                {
                    const float inv = 0.5f / (g0 * g1);   // exact: powers of two
                    float um = 0.f;
                    const int kx = 2 * nu2 + sb;
#pragma unroll 1
                    for (int j = 0; j < 2; ++j) {
#pragma unroll
                        for (int s = 0; s < CW / 16; ++s) {
                            const int k0 = mix_col<PREC>(j, x.h) + 16 * s;
                            float re[16], im[16];
                            tmem_ld16x2(x.tl + RA + k0, x.tl + RA + 128 + k0, re, im);
                            float av[16];
#pragma unroll
                            for (int t = 0; t < 16; ++t) av[t] = __ldcs(a.amp + fo + (size_t)(2 * (k0 + t) + sa) * M + kx);
                            float ur[16], ui[16];
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                const float X = re[t] * inv, Y = im[t] * inv;
                                const float m2 = fmaf(X, X, Y * Y);
                                const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                                const float d = av[t] - m2 * rs;
                                acc[0] += d * d;
                                acc[1] += av[t] * av[t];
                                bad |= (int)bad_amplitude(av[t]);
                                if (m2 > 0.f) {
                                    const float f = fmaf(cp * av[t], rs, b);
                                    ur[t] = X * f;
                                    ui[t] = Y * f;
                                } else {
                                    ur[t] = cp * av[t];
                                    ui[t] = 0.f;
                                }
                                um = fmaxf(um, fmaxf(fabsf(ur[t]), fabsf(ui[t])));
                            }
                            float r8[8], i8[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) { r8[t] = ur[t]; i8[t] = ui[t]; }
                            tmem_st8x2(x.tl + RA + k0, x.tl + RA + 128 + k0, r8, i8);
#pragma unroll
                            for (int t = 0; t < 8; ++t) { r8[t] = ur[8 + t]; i8[t] = ui[8 + t]; }
                            tmem_st8x2(x.tl + RA + k0 + 8, x.tl + RA + 128 + k0 + 8, r8, i8);
                        }
                    }
                    tmem_wait_st();
                    if constexpr (G::F16) g2 = mix_pow2_scale(mix_block_max<PREC>(x, um));
                }

                if (!(ok = mix_stage<PREC>(x, RA, RB, true, g2))) break;
                if constexpr (G::F16) g3 = kMixStage2Scale;
                if (!(ok = mix_stage<PREC>(x, RB, RA, true, g3))) break;
                const float inv = 1.f / (g2 * g3);

                if (sub < 3) {   // F128^-1(U_ab) into slab slot sub (its y_ab is consumed)
#pragma unroll 1
                    for (int j = 0; j < 2; ++j) {
#pragma unroll
                        for (int s = 0; s < CW / 16; ++s) {
                            const int n0 = mix_col<PREC>(j, x.h) + 16 * s;
                            float re[16], im[16];
                            tmem_ld16x2(x.tl + RA + n0, x.tl + RA + 128 + n0, re, im);
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                st_hint(slab_at(sub, n0 + t), make_float2(re[t] * inv, im[t] * inv), pol_keep);
                        }
                    }
                    continue;
                }

                // ------------------------------------------ combination + epilogue
                if (x.leader) prefetch_frame(i + gridDim.x);
#pragma unroll 1
                for (int j = 0; j < 2; ++j) {
#pragma unroll
                    for (int s = 0; s < CW / 16; ++s) {
                        const int n0 = mix_col<PREC>(j, x.h) + 16 * s;
                        float re[16], im[16];
                        tmem_ld16x2(x.tl + RA + n0, x.tl + RA + 128 + n0, re, im);
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const int nu1 = n0 + t;
                            finish_row(nu1, ld_hint(slab_at(0, nu1), pol_keep), ld_hint(slab_at(1, nu1), pol_keep),
                                       ld_hint(slab_at(2, nu1), pol_keep), make_float2(re[t] * inv, im[t] * inv));
                        }
                    }
                }
            }
        }
        if (!ok) break;
    }

    // A wait gave up: wait (bounded, full limit) once more for MMAs whose
    // commit was not waited for, so that nothing writes TMEM after the block
    // has left.
    if (x.mma_pending && x.leader) mbar_wait(x.bar, x.phase);
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
static cudaError_t launch_mixed256_one(const FrameArgs& a, float2* slab, cudaStream_t s) {
    using G = MixGeo<PREC>;
    constexpr int SMEM = G::A_BYTES + G::B_BYTES + 128;
    auto kern = raar_mixed256_kernel<PREC, MODE, FLAGS, WRAP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = a.K < sms ? a.K : sms;   // one block (and one slab of 4 H x H slots) per SM
    kern<<<grid, G::NT, SMEM, s>>>(a, slab);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_mixed256_prec(int mode, int flags, const FrameArgs& a, float2* slab, cudaStream_t s) {
    if (!slab) return cudaErrorInvalidValue;
    if (mode == MODE_PROJECT) return launch_mixed256_one<PREC, MODE_PROJECT, 0, 0>(a, slab, s);
    if (mode != MODE_RAAR) return cudaErrorInvalidValue;
    const int f = flags & (RF_FORM_B | RF_METRIC);
    if (a.wrap) {
        switch (f) {
            case 0: return launch_mixed256_one<PREC, MODE_RAAR, 0, 1>(a, slab, s);
            case RF_FORM_B: return launch_mixed256_one<PREC, MODE_RAAR, RF_FORM_B, 1>(a, slab, s);
            case RF_METRIC: return launch_mixed256_one<PREC, MODE_RAAR, RF_METRIC, 1>(a, slab, s);
            default: return launch_mixed256_one<PREC, MODE_RAAR, RF_FORM_B | RF_METRIC, 1>(a, slab, s);
        }
    }
    switch (f) {
        case 0: return launch_mixed256_one<PREC, MODE_RAAR, 0, 0>(a, slab, s);
        case RF_FORM_B: return launch_mixed256_one<PREC, MODE_RAAR, RF_FORM_B, 0>(a, slab, s);
        case RF_METRIC: return launch_mixed256_one<PREC, MODE_RAAR, RF_METRIC, 0>(a, slab, s);
        default: return launch_mixed256_one<PREC, MODE_RAAR, RF_FORM_B | RF_METRIC, 0>(a, slab, s);
    }
}

}  // namespace sharp
