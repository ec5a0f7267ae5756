// Image-side kernels: illumination sum D = Q*Q, normalisation (Q*Q)^{-1},
// split Q, overlap Q* by per-tile gathers, probe update (Eq. 10), metric
// finalisation (Eqs. 11-13) and the solution metric (Eq. 14).
//
// Q* and Q*Q are gathered per 32 x 32 image tile over the list of frames that
// touch the tile (built once per plan), so every image pixel is written by
// exactly one thread: no atomics and a fixed summation order; Q*Q is summed
// in FP64 across groups of FP32 terms, Q* z with compensated (Kahan) FP32.
#include <cuda_runtime.h>
#include <math.h>

#include <cstring>

#include "sharp_common.cuh"

namespace sharp {

namespace {

constexpr int GATHER_THREADS = 256;       // 32 columns x 8 row groups

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Offset of image coordinate g inside a frame starting at p (wrap-aware);
// returns a value >= m when g is outside the frame.
__device__ __forceinline__ int local_offset(int g, int p, int n, int wrap, int m) {
    int d = g - p;
    if (wrap && d < 0) d += n;
    return (d < 0) ? m : d;
}

// ------------------------------------------------------------------ D = Q*Q
__global__ void w2_kernel(const float2* __restrict__ w, float* __restrict__ w2, int mm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mm; i += gridDim.x * blockDim.x)
        w2[i] = cabs2(w[i]);
}

// Frame list entries of a tile staged in shared memory per round.
constexpr int GATHER_STAGE = 512;
// Frames summed in plain FP32 before each FP64 add: D = Q*Q (Eq. 9) is
// accumulated in FP64 across groups (GB300's FP64 rate is low, so the per-term
// adds stay FP32) and rounded once to FP32; near the probe edges, where D is
// small and built from many tiny terms, that keeps it correctly rounded.
constexpr int GATHER_GROUP = 16;

template <int WRAP>
__global__ void __launch_bounds__(GATHER_THREADS)
illum_gather_kernel(const int32_t* __restrict__ pos, const int* __restrict__ tptr,
                    const int* __restrict__ tfr, const float* __restrict__ w2, float* __restrict__ D,
                    unsigned* __restrict__ dmax_bits, int m, int ny, int nx, int tiles_x) {
    __shared__ int2 sp[GATHER_STAGE];          // (row, col) of the staged frames
    const int tile = blockIdx.x;
    const int gx = (tile % tiles_x) * TILE + (threadIdx.x & 31);
    const int gy0 = (tile / tiles_x) * TILE + (threadIdx.x >> 5);
    double s[4] = {0.0, 0.0, 0.0, 0.0};        // FP64 sums of the FP32 group sums
    const int j0 = tptr[tile], j1 = tptr[tile + 1];
    for (int base = j0; base < j1; base += GATHER_STAGE) {
        const int n = min(GATHER_STAGE, j1 - base);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int f = __ldg(tfr + base + t);
            sp[t] = make_int2(__ldg(pos + 2 * f), __ldg(pos + 2 * f + 1));
        }
        __syncthreads();
        for (int t0 = 0; t0 < n; t0 += GATHER_GROUP) {
            const int t1 = min(n, t0 + GATHER_GROUP);
            float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int t = t0; t < t1; ++t) {
                const int2 p = sp[t];
                int lx = gx - p.y;
                if (WRAP && lx < 0) lx += nx;
                if ((unsigned)lx >= (unsigned)m) continue;   // column outside this frame
                const float* wr = w2 + lx;
                const int ly0 = gy0 - p.x;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    int ly = ly0 + 8 * r;
                    if (WRAP && ly < 0) ly += ny;
                    if ((unsigned)ly < (unsigned)m) part[r] += __ldg(wr + ly * m);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) s[r] += (double)part[r];
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gy = gy0 + 8 * r;
        if (gy < ny && gx < nx) {
            const float d = (float)s[r];
            D[gy * nx + gx] = d;
            mx = fmaxf(mx, d);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dmax_bits, __float_as_uint(mx));
}

// 1/D above the threshold of reading R4, 0 below it.  A probe with no finite
// positive illumination anywhere (zero, or not finite) leaves every frame
// without an object pixel: that raises SHARP_ERR_INVALID_ARG on `err`.
__global__ void invd_kernel(const float* __restrict__ D, float* __restrict__ invD,
                            const unsigned* __restrict__ dmax_bits, int n, int* __restrict__ err) {
    const float dmax = __uint_as_float(*dmax_bits);
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(dmax > 0.f && dmax <= 3.402823466e38f))
        raise_error(err, SHARP_ERR_INVALID_ARG);
    const float thr = 1e-12f * dmax;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = D[i];
        invD[i] = d > thr ? 1.0f / d : 0.0f;
    }
}

// ------------------------------------------------------------------ Q* z
__global__ void __launch_bounds__(GATHER_THREADS)
overlap_gather_kernel(const int32_t* __restrict__ pos, const int* __restrict__ tptr,
                      const int* __restrict__ tfr, const float2* __restrict__ w,
                      const float2* __restrict__ z, float2* __restrict__ img, int m, int ny, int nx,
                      int tiles_x, int wrap) {
    const int tile = blockIdx.x;
    const int gx = (tile % tiles_x) * TILE + (threadIdx.x & 31);
    const int gy0 = (tile / tiles_x) * TILE + (threadIdx.x >> 5);
    float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    const size_t mm = (size_t)m * m;
    for (int j = tptr[tile]; j < tptr[tile + 1]; ++j) {
        const int f = tfr[j];
        const int py = pos[2 * f], px = pos[2 * f + 1];
        const int lx = local_offset(gx, px, nx, wrap, m);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ly = local_offset(gy0 + 8 * r, py, ny, wrap, m);
            if (lx < m && ly < m) {
                const int l = ly * m + lx;
                const float2 t = cmulc(__ldg(w + l), __ldg(z + f * mm + l));
                kahan_add(sr[r], cr[r], t.x);
                kahan_add(si[r], ci[r], t.y);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gy = gy0 + 8 * r;
        if (gy < ny && gx < nx) img[gy * nx + gx] = make_float2(sr[r], si[r]);
    }
}

// The overlap sums of the RAAR step relative to the object, gathered per
// image tile over the frames covering it in a fixed order (the deterministic
// mode of the frame pass, which then scatters nothing):
//   out(x) = sum_i conj(w_p(r_i)) (u_i(r_i) - rho w_p(r_i) psi(x)),  r_i = x - x_i,
// with u_i = c_i (the new state: C', rho = 1 - b) or u_i = w_f(r_i) psi_y(x)
// + c_i (the iterate z before the step: B', rho = 1; w_f and psi_y given).
// Terms are summed in FP32 with compensation, as Q* z above.
__global__ void __launch_bounds__(GATHER_THREADS)
overlap_delta_gather_kernel(const int32_t* __restrict__ pos, const int* __restrict__ tptr,
                            const int* __restrict__ tfr, const float2* __restrict__ wp,
                            const float2* __restrict__ wf, const float2* __restrict__ c,
                            const float2* __restrict__ psiy, const float2* __restrict__ psi, float rho,
                            float2* __restrict__ img, int m, int ny, int nx, int tiles_x, int wrap) {
    const int tile = blockIdx.x;
    const int gx = (tile % tiles_x) * TILE + (threadIdx.x & 31);
    const int gy0 = (tile / tiles_x) * TILE + (threadIdx.x >> 5);
    float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    float2 ps[4], py4[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gy = gy0 + 8 * r;
        const bool in = gy < ny && gx < nx;
        ps[r] = in ? psi[gy * nx + gx] : make_float2(0.f, 0.f);
        py4[r] = (in && psiy) ? psiy[gy * nx + gx] : make_float2(0.f, 0.f);
    }
    const size_t mm = (size_t)m * m;
    for (int j = tptr[tile]; j < tptr[tile + 1]; ++j) {
        const int f = tfr[j];
        const int py = pos[2 * f], px = pos[2 * f + 1];
        const int lx = local_offset(gx, px, nx, wrap, m);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ly = local_offset(gy0 + 8 * r, py, ny, wrap, m);
            if (lx < m && ly < m) {
                const int l = ly * m + lx;
                const float2 w = __ldg(wp + l);
                float2 u = __ldg(c + f * mm + l);
                if (wf) u = cadd(u, cmul(__ldg(wf + l), py4[r]));
                const float2 t = cmulc(w, csub(u, cscale(cmul(w, ps[r]), rho)));
                kahan_add(sr[r], cr[r], t.x);
                kahan_add(si[r], ci[r], t.y);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gy = gy0 + 8 * r;
        if (gy < ny && gx < nx) img[gy * nx + gx] = make_float2(sr[r], si[r]);
    }
}

__global__ void scale_invd_kernel(float2* __restrict__ img, const float* __restrict__ invD, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        img[i] = cscale(img[i], invD[i]);
}

// ------------------------------------------------------------------ Q psi
__global__ void q_gather_kernel(const int32_t* __restrict__ pos, const float2* __restrict__ obj,
                                const float2* __restrict__ w, float2* __restrict__ frames, int K, int m,
                                int ny, int nx, int wrap) {
    const size_t mm = (size_t)m * m;
    const size_t total = (size_t)K * mm;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / mm);
        const int l = (int)(e - (size_t)f * mm);
        const int y = l / m, x = l - y * m;
        const int o = obj_index(pos[2 * f], pos[2 * f + 1], y, x, ny, nx, wrap);
        frames[e] = cmul(__ldg(w + l), __ldg(obj + o));
    }
}

// ------------------------------------------------------------------ RAAR image pass
// The frame pass scattered its overlap sums relative to the object psi of
// the previous step (the image this kernel overwrites):
//   C' = Q*(c_new - (1-b) w psi)   with c_new = (1-2b) P_a z + b z,
//   B' = Q*(z - w psi)             only after a probe change; otherwise
//                                   Q* z = D psi exactly and B' = 0.
// Then C = Q* c_new = C' + (1-b) D psi and B = Q* z = B' + D psi, so with
// A = Q* P_a z = (C - b B)/(1-2b) (Sec. 2.2 RAAR update, Luke form):
//   A/D   = psi + (C' - b B') / ((1-2b) D)          -> psi (Eq. 9)
//   psi_y = (2b A - b B)/D = b psi + 2b (A/D - psi) - b B'/D
// Only the corrections C', B' pass through the 1/(1-2b) factor, so FP32
// rounding of the overlap sums is not amplified from full-size values.
// Both images are 0 where D is below the threshold; the sums are cleared
// for the next step.
__global__ void normalise_kernel(float2* __restrict__ C, float2* __restrict__ B,
                                 const float* __restrict__ invD, float2* __restrict__ psiy,
                                 float2* __restrict__ psi, float beta, int form_b, int n) {
    const float k = 1.f / (1.f - 2.f * beta);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float id = invD[i];
        const float2 cs = C[i];
        const float2 bs = form_b ? B[i] : make_float2(0.f, 0.f);
        float2 ny_ = make_float2(0.f, 0.f), np_ = make_float2(0.f, 0.f);
        if (id > 0.f) {
            const float2 ps = psi[i];
            const float kd = k * id;
            // dA = A/D - psi
            const float2 dA = make_float2(kd * fmaf(-beta, bs.x, cs.x), kd * fmaf(-beta, bs.y, cs.y));
            np_ = cadd(ps, dA);
            const float2 bd = cscale(bs, id);
            ny_ = make_float2(fmaf(beta, ps.x, beta * fmaf(2.f, dA.x, -bd.x)),
                              fmaf(beta, ps.y, beta * fmaf(2.f, dA.y, -bd.y)));
        }
        psi[i] = np_;
        psiy[i] = ny_;
        C[i] = make_float2(0.f, 0.f);
        if (form_b) B[i] = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------ Eq. 10
// Partial sums over a chunk of frames, one thread per probe pixel:
//   num = sum conj(psi(r + x_i)) z_i(r),  den = sum |psi(r + x_i)|^2
// with z_i = w . psi_y(r + x_i) + c_i (state) or z_i given (frames).
__global__ void probe_partial_kernel(const int32_t* __restrict__ pos, const float2* __restrict__ psi,
                                     const float2* __restrict__ zc, const float2* __restrict__ psiy,
                                     const float2* __restrict__ w, float* __restrict__ part, int K, int m,
                                     int ny, int nx, int wrap, int chunk_frames) {
    constexpr int U = 8;   // frames in flight per thread
    const int mm = m * m;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= mm) return;
    const int chunk = blockIdx.y;
    const int y = l / m, x = l - y * m;
    const int f0 = chunk * chunk_frames;
    const int f1 = min(K, f0 + chunk_frames);
    const float2 wl = psiy ? __ldg(w + l) : make_float2(0.f, 0.f);
    float nr = 0.f, ni = 0.f, dn = 0.f;
    for (int f = f0; f < f1; f += U) {
        float2 ps[U], zz[U], yy[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = min(f + u, f1 - 1);
            const int o = obj_index(__ldg(pos + 2 * g), __ldg(pos + 2 * g + 1), y, x, ny, nx, wrap);
            ps[u] = __ldg(psi + o);
            zz[u] = __ldcs(zc + (size_t)g * mm + l);
            yy[u] = psiy ? __ldg(psiy + o) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (f + u >= f1) break;
            const float2 z = psiy ? cadd(zz[u], cmul(wl, yy[u])) : zz[u];
            const float2 t = cmulc(ps[u], z);
            nr += t.x;
            ni += t.y;
            dn += cabs2(ps[u]);
        }
    }
    float* pc = part + (size_t)chunk * 3 * mm;
    pc[l] = nr;
    pc[mm + l] = ni;
    pc[2 * mm + l] = dn;
}

// FP64 sum over chunks of the FP32 partials: 32 probe pixels per block, the
// chunks split over the block's 8 warps, then combined in a fixed order; the
// largest denominator goes to dmax (as ordered bits: it is >= 0).
__global__ void __launch_bounds__(256) probe_reduce_kernel(const float* __restrict__ part, double* __restrict__ acc,
                                                           int chunks, int mm, unsigned long long* __restrict__ dmax) {
    __shared__ double sh[3][8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = blockIdx.x * 32 + lane;
    double nr = 0.0, ni = 0.0, dn = 0.0;
    if (l < mm) {
        for (int c = warp; c < chunks; c += 8) {
            const float* pc = part + (size_t)c * 3 * mm;
            nr += pc[l];
            ni += pc[mm + l];
            dn += pc[2 * mm + l];
        }
    }
    sh[0][warp][lane] = nr;
    sh[1][warp][lane] = ni;
    sh[2][warp][lane] = dn;
    __syncthreads();
    if (warp < 3) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[warp][k][lane];
        if (l < mm) acc[warp * mm + l] = t;
        if (warp == 2) {
            unsigned long long bits = (unsigned long long)__double_as_longlong(l < mm ? t : 0.0);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
                bits = ob > bits ? ob : bits;
            }
            if (lane == 0) atomicMax(dmax, bits);
        }
    }
}

// w_new = num / den, or w_old where den <= 1e-12 of the largest (reading R6).
__global__ void probe_final_kernel(const double* __restrict__ acc, const float2* __restrict__ w_old,
                                   float2* __restrict__ w_new, int mm,
                                   const unsigned long long* __restrict__ dmax) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= mm) return;
    const double thr = 1e-12 * __longlong_as_double((long long)*dmax);
    const double dn = acc[2 * mm + l];
    w_new[l] = dn > thr ? make_float2((float)(acc[l] / dn), (float)(acc[mm + l] / dn)) : w_old[l];
}

// ------------------------------------------------------------------ metrics
__global__ void metrics_final_kernel(const double* __restrict__ sums, double* __restrict__ out, int have_q,
                                     int have_d, int delta_is_norm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double a2 = sums[S_A2];
    const double na = sqrt(a2);
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    out[0] = sqrt(sums[S_RESID]) / na;
    out[1] = have_q ? sqrt(sums[S_Q]) / na : nan;
    out[2] = have_d ? sqrt(delta_is_norm ? sums[S_Z2] : sums[S_D]) / na : nan;
    out[3] = na;
}

// ------------------------------------------------------------------ illumination refinement
// Centre of mass of |w|^2 (Sec. 2.2 drift pathology): one block, FP64 sums of
// |w|^2, row * |w|^2 and col * |w|^2 into out[0..2].
__global__ void probe_moments_kernel(const float2* __restrict__ w, int m, double* __restrict__ out) {
    __shared__ double sh[3][32];
    // FP32 per thread (a few dozen terms), FP64 across threads (GB300's FP64
    // rate is low, so the per-element work stays in FP32)
    float f0 = 0.f, fy = 0.f, fx = 0.f;
    const int mm = m * m;
    for (int l = threadIdx.x; l < mm; l += blockDim.x) {
        const float v = cabs2(w[l]);
        f0 += v;
        fy = fmaf(v, (float)(l / m), fy);
        fx = fmaf(v, (float)(l % m), fx);
    }
    double s0 = f0, sy = fy, sx = fx;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sh[0][warp] = s0;
        sh[1][warp] = sy;
        sh[2][warp] = sx;
    }
    __syncthreads();
    if (warp == 0) {
        double t0 = lane < nw ? sh[0][lane] : 0.0, ty = lane < nw ? sh[1][lane] : 0.0,
               tx = lane < nw ? sh[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            ty += __shfl_xor_sync(0xffffffffu, ty, o);
            tx += __shfl_xor_sync(0xffffffffu, tx, o);
        }
        if (lane == 0) {
            out[0] = t0;
            out[1] = ty;
            out[2] = tx;
        }
    }
}

// out(r) = in((r + d) mod m) with d = floor(centroid - m/2 + 1/2) per axis:
// the roll that moves the centroid to the frame centre.  A zero probe is
// copied unchanged.
__global__ void probe_roll_kernel(const float2* __restrict__ in, float2* __restrict__ out, int m,
                                  const double* __restrict__ mom) {
    int dy = 0, dx = 0;
    if (mom[0] > 0.0) {
        dy = (int)floor(mom[1] / mom[0] - 0.5 * m + 0.5);
        dx = (int)floor(mom[2] / mom[0] - 0.5 * m + 0.5);
    }
    dy = ((dy % m) + m) % m;
    dx = ((dx % m) + m) % m;
    const int mm = m * m;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < mm; l += gridDim.x * blockDim.x) {
        int y = l / m + dy, x = l % m + dx;
        y -= (y >= m) ? m : 0;
        x -= (x >= m) ? m : 0;
        out[l] = in[y * m + x];
    }
}

// Mean intensity of the frames: acc[l] += sum over this block's chunk of
// frames of amp^2 (FP64 atomics, one per pixel per chunk).
__global__ void mean_frame_partial_kernel(const float* __restrict__ amp, int K, int mm, int chunk,
                                          double* __restrict__ acc) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= mm) return;
    const int f0 = blockIdx.y * chunk, f1 = min(K, f0 + chunk);
    double s = 0.0;
    for (int f = f0; f < f1; ++f) {
        const float v = __ldcs(amp + (size_t)f * mm + l);
        s += (double)v * v;
    }
    atomicAdd(acc + l, s);
}

// sqrt of the mean frame, or of its thresholded version (values below
// t * max -> 0, the others -> their mean), into a_w; and the centred unit
// impulse into z (its unitary transform has modulus 1/m and phase
// (-1)^(qy+qx), so P_a of it with amplitudes a_w is the centred inverse
// transform of a_w).  One block.
__global__ void mean_frame_final_kernel(const double* __restrict__ acc, int K, int m, float threshold,
                                        float* __restrict__ a_w, float2* __restrict__ z) {
    __shared__ double sh[2][32];
    const int mm = m * m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double level = -1.0;   // < 0: no threshold
    if (threshold > 0.f) {
        double mx = 0.0;
        for (int l = threadIdx.x; l < mm; l += blockDim.x) mx = fmax(mx, acc[l] / K);
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) sh[0][warp] = mx;
        __syncthreads();
        mx = 0.0;
        for (int i = 0; i < nw; ++i) mx = fmax(mx, sh[0][i]);
        __syncthreads();
        const double thr = (double)threshold * mx;
        double sum = 0.0, cnt = 0.0;
        for (int l = threadIdx.x; l < mm; l += blockDim.x) {
            const double v = acc[l] / K;
            if (v >= thr) {
                sum += v;
                cnt += 1.0;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) {
            sh[0][warp] = sum;
            sh[1][warp] = cnt;
        }
        __syncthreads();
        sum = 0.0;
        cnt = 0.0;
        for (int i = 0; i < nw; ++i) {
            sum += sh[0][i];
            cnt += sh[1][i];
        }
        level = cnt > 0.0 ? sum / cnt : 0.0;
        for (int l = threadIdx.x; l < mm; l += blockDim.x)
            a_w[l] = acc[l] / K >= thr ? (float)sqrt(level) : 0.f;
    } else {
        for (int l = threadIdx.x; l < mm; l += blockDim.x) a_w[l] = (float)sqrt(acc[l] / K);
    }
    const int c = (m / 2) * m + m / 2;
    for (int l = threadIdx.x; l < mm; l += blockDim.x) z[l] = make_float2(l == c ? 1.f : 0.f, 0.f);
}

__global__ void copy_scaled_kernel(const double* src, double* dst, double scale) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src * scale;
}

// ------------------------------------------------------------------ Eq. 14
// sums: 0,1 Re/Im <u,v>, 2 |v|^2, 3,4 Re/Im <psi,psi_t>_sel, 5 |psi_t|^2_sel,
//       6 |phi u - v|^2, 7 |phi' psi - psi_t|^2_sel ; u = D psi, v = D psi_t
__device__ __forceinline__ void block_add_double(double (&v)[6], double* sh, double* dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) sh[j * 32 + warp] = v[j];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            double s = lane < nw ? sh[j * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0 && s != 0.0) atomicAdd(dst + j, s);
        }
    }
}

__global__ void sol_pass1_kernel(const float2* __restrict__ psi, const float2* __restrict__ pt,
                                 const float* __restrict__ D, const unsigned* __restrict__ dmax_bits,
                                 double* __restrict__ sums, int n) {
    __shared__ double sh[6 * 32];
    const double sel_thr = 0.1 * (double)__uint_as_float(*dmax_bits);
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = D[i];
        const double ur = d * psi[i].x, ui = d * psi[i].y;
        const double vr = d * pt[i].x, vi = d * pt[i].y;
        v[0] += ur * vr + ui * vi;
        v[1] += ur * vi - ui * vr;
        v[2] += vr * vr + vi * vi;
        if (d >= sel_thr) {
            const double ar = psi[i].x, ai = psi[i].y, br = pt[i].x, bi = pt[i].y;
            v[3] += ar * br + ai * bi;
            v[4] += ar * bi - ai * br;
            v[5] += br * br + bi * bi;
        }
    }
    block_add_double(v, sh, sums);
}

__global__ void sol_pass2_kernel(const float2* __restrict__ psi, const float2* __restrict__ pt,
                                 const float* __restrict__ D, const unsigned* __restrict__ dmax_bits,
                                 double* __restrict__ sums, int n) {
    __shared__ double sh[6 * 32];
    const double sel_thr = 0.1 * (double)__uint_as_float(*dmax_bits);
    double p1r = sums[0], p1i = sums[1];
    double a1 = sqrt(p1r * p1r + p1i * p1i);
    if (a1 > 0) { p1r /= a1; p1i /= a1; } else { p1r = 1; p1i = 0; }
    double p2r = sums[3], p2i = sums[4];
    double a2 = sqrt(p2r * p2r + p2i * p2i);
    if (a2 > 0) { p2r /= a2; p2i /= a2; } else { p2r = 1; p2i = 0; }
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = D[i];
        const double ar = psi[i].x, ai = psi[i].y, br = pt[i].x, bi = pt[i].y;
        const double er = d * (p1r * ar - p1i * ai - br), ei = d * (p1r * ai + p1i * ar - bi);
        v[0] += er * er + ei * ei;
        if (d >= sel_thr) {
            const double fr = p2r * ar - p2i * ai - br, fi = p2r * ai + p2i * ar - bi;
            v[1] += fr * fr + fi * fi;
        }
    }
    block_add_double(v, sh, sums + 6);
}

__global__ void sol_final_kernel(const double* __restrict__ sums, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[0] = sqrt(sums[6] / sums[2]);
        out[1] = sqrt(sums[7] / sums[5]);
    }
}

inline int grid_for(size_t n, int threads, int cap = 152 * 16) {
    size_t g = (n + threads - 1) / threads;
    if (g > (size_t)cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

// ----------------------------------------------------------------------- launchers
static cudaError_t illum_for(const Plan& p, const float2* w, float* w2, float* D, unsigned* dmax,
                             cudaStream_t s) {
    const int mm = p.m * p.m;
    w2_kernel<<<grid_for(mm, 256), 256, 0, s>>>(w, w2, mm);
    cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (p.prm.wrap)
        illum_gather_kernel<1><<<p.tiles_y * p.tiles_x, GATHER_THREADS, 0, s>>>(
            p.pos, p.tile_ptr, p.tile_frames, w2, D, dmax, p.m, p.ny, p.nx, p.tiles_x);
    else
        illum_gather_kernel<0><<<p.tiles_y * p.tiles_x, GATHER_THREADS, 0, s>>>(
            p.pos, p.tile_ptr, p.tile_frames, w2, D, dmax, p.m, p.ny, p.nx, p.tiles_x);
    return cudaGetLastError();
}

cudaError_t launch_illumination(const Plan& p, const float2* w, float* w2, float* D, float* invD,
                                unsigned* dmax_bits, cudaStream_t s) {
    cudaError_t e = illum_for(p, w, w2, D, dmax_bits, s);
    if (e != cudaSuccess) return e;
    const int n = p.ny * p.nx;
    invd_kernel<<<grid_for(n, 256), 256, 0, s>>>(D, invD, dmax_bits, n, p.errflag);
    return cudaGetLastError();
}

cudaError_t launch_normalise(Plan& p, float2* psiy, float2* psi, int form_b, cudaStream_t s) {
    const int n = p.ny * p.nx;
    normalise_kernel<<<grid_for(n, 256), 256, 0, s>>>(p.accA, p.accB, p.invD, psiy, psi, p.prm.beta, form_b, n);
    return cudaGetLastError();
}

cudaError_t launch_q_gather(const Plan& p, const float2* obj, const float2* probe, float2* frames,
                            cudaStream_t s) {
    const size_t total = (size_t)p.K * p.m * p.m;
    q_gather_kernel<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(p.pos, obj, probe, frames, p.K, p.m, p.ny,
                                                                   p.nx, p.prm.wrap);
    return cudaGetLastError();
}

cudaError_t launch_overlap_gather(const Plan& p, const float2* probe, const float2* z, float2* img,
                                  cudaStream_t s) {
    overlap_gather_kernel<<<p.tiles_y * p.tiles_x, GATHER_THREADS, 0, s>>>(
        p.pos, p.tile_ptr, p.tile_frames, probe, z, img, p.m, p.ny, p.nx, p.tiles_x, p.prm.wrap);
    return cudaGetLastError();
}

cudaError_t launch_overlap_delta_gather(const Plan& p, const float2* wp, const float2* wf, const float2* c,
                                        const float2* psiy, const float2* psi, float rho, float2* img,
                                        cudaStream_t s) {
    overlap_delta_gather_kernel<<<p.tiles_y * p.tiles_x, GATHER_THREADS, 0, s>>>(
        p.pos, p.tile_ptr, p.tile_frames, wp, wf, c, psiy, psi, rho, img, p.m, p.ny, p.nx, p.tiles_x, p.prm.wrap);
    return cudaGetLastError();
}

cudaError_t launch_scale_invD(const Plan& p, float2* img, const float* invD, cudaStream_t s) {
    const int n = p.ny * p.nx;
    scale_invd_kernel<<<grid_for(n, 256), 256, 0, s>>>(img, invD, n);
    return cudaGetLastError();
}

static cudaError_t probe_common(Plan& p, const float2* psi, const float2* zc, const float2* psiy,
                                const float2* wform, const float2* w_old, float2* w_out, cudaStream_t s) {
    const int mm = p.m * p.m;
    dim3 g((mm + 255) / 256, p.probe_chunks);
    probe_partial_kernel<<<g, 256, 0, s>>>(p.pos, psi, zc, psiy, wform, p.probe_part, p.K, p.m, p.ny, p.nx,
                                          p.prm.wrap, p.probe_chunk_frames);
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(p.scal);
    cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    probe_reduce_kernel<<<(mm + 31) / 32, 256, 0, s>>>(p.probe_part, p.probe_acc, p.probe_chunks, mm, dmax);
    probe_final_kernel<<<(mm + 255) / 256, 256, 0, s>>>(p.probe_acc, w_old, w_out, mm, dmax);
    return cudaGetLastError();
}

cudaError_t launch_probe_update_state(Plan& p, const float2* c, const float2* psiy, const float2* psi,
                                      cudaStream_t s) {
    // z^(l) = w_cur . psi_y + c.  The current probe is copied to w_form (it
    // formed the iterate) and the refined probe is written to w_cur; the
    // buffers keep their addresses, so recorded CUDA graphs stay valid.
    cudaError_t e = cudaMemcpyAsync(p.w_form, p.w_cur, sizeof(float2) * p.m * p.m, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return probe_common(p, psi, c, psiy, p.w_form, p.w_form, p.w_cur, s);
}

cudaError_t launch_probe_update_frames(Plan& p, const float2* obj, const float2* z, const float2* w_old,
                                       float2* w_out, cudaStream_t s) {
    return probe_common(p, obj, z, nullptr, nullptr, w_old, w_out, s);
}

cudaError_t launch_metrics_finalize(const Plan& p, double* metrics, int have_q, int have_d, int delta_is_norm,
                                    cudaStream_t s) {
    metrics_final_kernel<<<1, 32, 0, s>>>(p.sums, metrics, have_q, have_d, delta_is_norm);
    return cudaGetLastError();
}

// Frame-kernel arguments for a single m x m "frame" (the probe).
static FrameArgs probe_frame_args(const Plan& p, const float2* zin, float2* zout, const float* amp) {
    FrameArgs a;
    memset(&a, 0, sizeof(a));
    a.K = 1;
    a.m = p.m;
    a.ny = p.ny;
    a.nx = p.nx;
    a.pos = p.pos;
    a.zin = zin;
    a.zout = zout;
    a.amp = amp;
    a.sums = p.scal + 16;   // residual slot of the single-frame launches
    a.err = p.errflag;
    a.counter = p.counter;
    a.scratch = p.big_scratch;
    return a;
}

cudaError_t launch_probe_refine(Plan& p, const float2* w_in, float2* w_out, cudaStream_t s) {
    const int mm = p.m * p.m;
    cudaError_t e = cudaSuccess;
    const float2* cur = w_in;
    if (p.probe_cons_kind != 0 && p.probe_cons) {
        const int mode = p.probe_cons_kind == SHARP_PROBE_CONSTRAINT_MASK ? MODE_MASK : MODE_PROJECT;
        e = launch_frames(mode, 0, probe_frame_args(p, cur, w_out, p.probe_cons), s);
        if (e != cudaSuccess) return e;
        cur = w_out;
    }
    if (p.probe_com) {
        double* mom = p.scal + 20;
        probe_moments_kernel<<<1, 1024, 0, s>>>(cur, p.m, mom);
        probe_roll_kernel<<<grid_for(mm, 256), 256, 0, s>>>(cur, p.w_tmp, p.m, mom);
        e = cudaMemcpyAsync(w_out, p.w_tmp, sizeof(float2) * mm, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        cur = w_out;
    }
    if (cur != w_out) e = cudaMemcpyAsync(w_out, cur, sizeof(float2) * mm, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_probe_init_mean(Plan& p, const float* amp, float threshold, float2* w_out, cudaStream_t s) {
    const int mm = p.m * p.m;
    double* acc = p.probe_acc;   // first m*m doubles; not live outside a probe update
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * mm, s);
    if (e != cudaSuccess) return e;
    const int chunk = 64;
    dim3 g((mm + 255) / 256, (p.K + chunk - 1) / chunk);
    mean_frame_partial_kernel<<<g, 256, 0, s>>>(amp, p.K, mm, chunk, acc);
    mean_frame_final_kernel<<<1, 1024, 0, s>>>(acc, p.K, p.m, threshold, p.w2tmp, p.w_tmp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_frames(MODE_PROJECT, 0, probe_frame_args(p, p.w_tmp, w_out, p.w2tmp), s);
}

cudaError_t launch_copy_scaled(const double* src, double* dst, double scale, cudaStream_t s) {
    copy_scaled_kernel<<<1, 32, 0, s>>>(src, dst, scale);
    return cudaGetLastError();
}

cudaError_t launch_solution_error(Plan& p, const float2* psi, const float2* psi_true, const float2* probe,
                                  double* out, cudaStream_t s) {
    // D of the given probe goes to the plan's scratch images (the RAAR
    // state's own D is untouched).
    const int n = p.ny * p.nx;
    float* D = p.Dtmp;
    unsigned* dmax = reinterpret_cast<unsigned*>(p.scal + 2);
    cudaError_t e = illum_for(p, probe, p.w2tmp, D, dmax, s);
    if (e != cudaSuccess) return e;
    double* sums = p.scal + 4;   // 12 doubles
    e = cudaMemsetAsync(sums, 0, 8 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n, 256, 152 * 4);
    sol_pass1_kernel<<<g, 256, 0, s>>>(psi, psi_true, D, dmax, sums, n);
    sol_pass2_kernel<<<g, 256, 0, s>>>(psi, psi_true, D, dmax, sums, n);
    sol_final_kernel<<<1, 32, 0, s>>>(sums, out);
    return cudaGetLastError();
}

}  // namespace sharp
