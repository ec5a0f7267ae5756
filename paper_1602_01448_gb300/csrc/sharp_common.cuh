// Shared device helpers and the internal (C++) interface between the
// translation units of the library.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sharp.h"

namespace sharp {

// ---------------------------------------------------------------- complex
// Complex add / subtract on the packed FP32x2 pipe of sm_100-class GPUs: one
// instruction per complex operation (a float2 already occupies an aligned
// register pair).  b * (-1) + a rounds exactly like a - b.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// A measured Fourier amplitude (Eq. 1: a = |F z| >= 0) that is NaN, infinite
// or negative; the frame passes raise SHARP_ERR_INVALID_ARG on the plan.
__device__ __forceinline__ bool bad_amplitude(float a) { return !(a >= 0.f && a <= 3.402823466e38f); }

// Record a kernel-side error on a plan's flag unless one is already set.
__device__ __forceinline__ void raise_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// 1/sqrt(x) for x > 0: the hardware estimate refined by one Newton step for
// f(r) = r^-2 - x, r <- r + r (1 - x r^2) / 2, evaluated with a fused
// multiply-add.  The result is within about one unit in the last place and
// carries no systematic bias, so |P_a z| (Eq. 7) matches the measured
// amplitude on average; a biased estimate shifts the RAAR fixed point.
__device__ __forceinline__ float rsqrt_refined(float x) {
    const float r = rsqrtf(x);
    const float e = fmaf(-(x * r), r, 1.0f);
    return fmaf(0.5f * r, e, r);
}

// Vector reductions into global memory (sm_90+): one red.global per pixel.
__device__ __forceinline__ void red_add_f2(float2* p, float2 v) {
    atomicAdd(p, v);
}

// Object pixel index of frame-local (y, x) for a frame at (py, px).  With wrap
// the positions are pre-reduced to [0, n) and m <= n, so one subtraction is
// enough.
__device__ __forceinline__ int obj_index(int py, int px, int y, int x, int ny, int nx, int wrap) {
    int r = py + y, c = px + x;
    if (wrap) {
        r = (r >= ny) ? r - ny : r;
        c = (c >= nx) ? c - nx : c;
    }
    return r * nx + c;
}

// Block-wide sum of NV floats per thread; result valid in thread 0.  `red`
// must hold 32 * NV floats of shared memory.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* red) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) red[j * 32 + warp] = v[j];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float s = (lane < NW) ? red[j * 32 + lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            v[j] = s;
        }
    }
}

// ---------------------------------------------------------------- plan
// Device-resident scratch owned by a plan.  All pointers are device pointers.
struct Plan {
    int K, m, ny, nx;
    sharp_params prm;
    int32_t* pos;            // K x 2, normalised (wrap) positions
    // per-tile frame lists (CSR over TILE x TILE image tiles)
    int tiles_y, tiles_x;
    int* tile_ptr;           // tiles + 1
    int* tile_frames;        // nnz
    int tile_nnz;
    // illumination
    float2* w_cur;           // probe used by the next projection
    float2* w_form;          // probe that formed the current iterate
    float* w2;               // |w_cur|^2 (m*m)
    float* Dsum;             // Q*Q (ny*nx), FP32 compensated sum
    float* invD;             // 1/D or 0 below the threshold
    unsigned* dmax_bits;     // max D as float bits
    // overlap sums (float2 images), relative to the current object psi:
    // accA = Q*(c_new - (1-b) w psi) (c_new the new frame state), accB =
    // Q*(z - w psi) (only after a probe change)
    float2* accA;
    float2* accB;
    bool b_valid;            // B/D equals the previous object (no probe change)
    bool initialised;
    // eps_Delta support: e = c^(l) - z^(l-1)
    float2* ebuf;            // K*m*m or nullptr
    int e_written_iter;      // step that last wrote ebuf (0 = none)
    int last_iter;           // last step run (0 = none)
    // reductions
    double* sums;            // 16 doubles of per-step sums
    int probe_chunks;        // chunks of frames in the partial sums of Eq. 10
    int probe_chunk_frames;  // frames per chunk
    float* probe_part;       // FP32 partial sums of Eq. 10 per chunk of frames (chunks x 3 x m*m)
    double* probe_acc;       // 3 x m*m doubles (FP64 sums over the chunks)
    double* scal;            // 32 doubles of misc scalars
    // scratch for operations on a caller-given probe (standalone operators)
    float* w2tmp;            // m*m
    float* Dtmp;             // ny*nx
    float* invDtmp;          // ny*nx
    bool form_differs;       // w_form != w_cur (a probe update happened)
    void* prof;              // kernel-timing state (sharp_api.cu), nullptr when off
    int* errflag;            // device int: sticky error raised inside kernels
    int* counter;            // device int: work counter of the persistent frame pass
    float2* big_scratch;     // m = 256: one m*m slab per SM (frame transposition)
    // illumination refinement after each probe update (Sec. 2.2, step 7)
    float* probe_cons;       // m*m Fourier mask or Fourier amplitudes (nullptr = none)
    int probe_cons_kind;     // SHARP_PROBE_CONSTRAINT_*
    int probe_com;           // centre the probe after each update
    float2* w_tmp;           // m*m scratch probe
    // tensor-core precision modes: the m x m DFT matrix parts in the operand
    // layout of the contraction kernels (nullptr in FP32 mode)
    void* dft_tab;
    // poll limit of the frame passes' bounded waits (FrameArgs::spin encoding)
    unsigned wait_spin;
    // deterministic overlap sums: gathered per tile in a fixed order instead
    // of scattered with atomics (bit-identical steps)
    int deterministic;
};

constexpr int TILE = 32;

// ------------------------------------------------ launchers (frame_kernels.cu)
enum FrameMode { MODE_RAAR = 0, MODE_PROJECT = 1, MODE_AMPS = 2, MODE_LOSS = 3, MODE_GRAD = 4,
                 MODE_PROJECT_PF = 5 /* P_a with one residual per frame in sums[i] */,
                 MODE_MASK = 6 /* F^-1{(F z) mask}, mask in `amp` */ };

struct FrameArgs {
    int K, m, ny, nx, wrap;
    const int32_t* pos;
    // RAAR state
    float2* c;               // K*m*m state (in/out)
    const float2* psiy;      // image
    const float2* psi;       // image (eps_Q gather)
    float2* ebuf;            // eps_Delta buffer
    const float2* w_form;
    const float2* w_proj;
    float2* accA;
    float2* accB;
    float beta;
    int read_e;              // accumulate |w_f psi_y + e|^2 (needs RF_METRIC)
    int write_e;             // store e = c_new - z
    // explicit-frame modes
    const float2* zin;
    float2* zout;
    const float* amp;
    float* amp_out;
    const float2* obj;
    const float2* probe;
    float2* g_obj;
    float2* g_probe;
    float gscale;
    double* sums;            // per-mode accumulators
    int* err;                // device error flag (SHARP_ERR_TIMEOUT on a bounded-wait failure)
    int* counter;            // frame counter of the persistent RAAR pass (zeroed per launch)
    float2* scratch;         // 256^2 frames: one m*m slab per block of the frame kernels
    const void* dft_tab;     // tensor-core precision modes: DFT matrix parts (raar_mixed.cuh layout)
    unsigned spin;           // poll limit of the first bounded waits (wait_polls: 0 default, kNoPolls none)
    int no_scatter;          // deterministic mode: the overlap sums are gathered after the pass instead
};

// compile-time flags of MODE_RAAR
enum RaarFlags { RF_FORM_B = 1, RF_METRIC = 2 };

template <int M>
cudaError_t launch_frames_m(int mode, int flags, const FrameArgs& a, cudaStream_t s);
template <int M, int WRAP>
cudaError_t launch_raar_w(int flags, const FrameArgs& a, cudaStream_t s);
template <int M>
inline cudaError_t launch_raar_m(int flags, const FrameArgs& a, cudaStream_t s) {
    return a.wrap ? launch_raar_w<M, 1>(flags, a, s) : launch_raar_w<M, 0>(flags, a, s);
}

// Tensor-core precision modes (raar_mixed.cuh; m = 128): the RAAR frame pass
// (MODE_RAAR) and the data projection (MODE_PROJECT) with the frame DFTs as
// FP16 / BF16x3 contractions.
template <int PREC>
cudaError_t launch_mixed_prec(int mode, int flags, const FrameArgs& a, cudaStream_t s);
// The same for 256^2 frames (raar_mixed256.cuh): the transforms split once,
// radix 2, into four 128^2 sub-problems; `slab` holds m*m scratch per block.
template <int PREC>
cudaError_t launch_mixed256_prec(int mode, int flags, const FrameArgs& a, float2* slab, cudaStream_t s);
cudaError_t launch_mixed(int prec, int mode, int flags, const FrameArgs& a, cudaStream_t s);  // sharp_api.cu

// 256^2 frames, the standalone modes (frame256_ops.cu): line passes through
// slabs of m*m scratch, one per block, at most one block per SM.
cudaError_t launch_big_ops(int mode, const FrameArgs& a, cudaStream_t s);
// The RAAR pass of 256^2 frames through four 128^2 register transforms
// (raar_split256.cuh) for one scan, or for the scans of a batch with `ch`
// rows per round trip (2, 4); `slab` holds m*m scratch per block.
cudaError_t launch_split256(int flags, const FrameArgs& a, float2* slab, cudaStream_t s);
struct BatchTable;
cudaError_t launch_split256_batch(int flags, const BatchTable& bt, int grid, float2* slab, cudaStream_t s, int ch);

inline cudaError_t launch_frames(int mode, int flags, const FrameArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    switch (a.m) {
        case 64: return launch_frames_m<64>(mode, flags, a, s);
        case 128: return launch_frames_m<128>(mode, flags, a, s);
        case 256:
            return mode == MODE_RAAR ? launch_split256(flags, a, a.scratch, s) : launch_big_ops(mode, a, s);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------ launchers (image_kernels.cu)
cudaError_t launch_illumination(const Plan& p, const float2* w, float* w2, float* D, float* invD,
                                unsigned* dmax_bits, cudaStream_t s);   // D = Q*Q of w, invD
cudaError_t launch_normalise(Plan& p, float2* psiy, float2* psi, int form_b, cudaStream_t s);
cudaError_t launch_q_gather(const Plan& p, const float2* obj, const float2* probe, float2* frames,
                            cudaStream_t s);
cudaError_t launch_overlap_gather(const Plan& p, const float2* probe, const float2* z, float2* img,
                                  cudaStream_t s);   // Q* z
cudaError_t launch_scale_invD(const Plan& p, float2* img, const float* invD, cudaStream_t s);  // img *= invD
// Deterministic overlap sums relative to the object (per-tile gathers in a
// fixed frame order): img = sum_i conj(wp) (u_i - rho wp psi), u_i = c_i, or
// wf psi_y + c_i when wf and psiy are given.
cudaError_t launch_overlap_delta_gather(const Plan& p, const float2* wp, const float2* wf, const float2* c,
                                        const float2* psiy, const float2* psi, float rho, float2* img,
                                        cudaStream_t s);
cudaError_t launch_probe_update_state(Plan& p, const float2* c, const float2* psiy, const float2* psi,
                                      cudaStream_t s);  // Eq. 10 on z = w_cur psiy + c -> w_cur
cudaError_t launch_probe_update_frames(Plan& p, const float2* obj, const float2* z,
                                       const float2* w_old, float2* w_out, cudaStream_t s);
cudaError_t launch_metrics_finalize(const Plan& p, double* metrics, int have_q, int have_d,
                                    int delta_is_norm, cudaStream_t s);
cudaError_t launch_solution_error(Plan& p, const float2* psi, const float2* psi_true, const float2* probe,
                                  double* out, cudaStream_t s);
cudaError_t launch_copy_scaled(const double* src, double* dst, double scale, cudaStream_t s);
// Fourier constraint (if configured) then centring (if configured) of probe
// w_in -> w_out (may alias), Sec. 2.2 step 7.
cudaError_t launch_probe_refine(Plan& p, const float2* w_in, float2* w_out, cudaStream_t s);
// Initial illumination from the mean frame of amp (Sec. 2.2 step 2, Sec. 3.2).
cudaError_t launch_probe_init_mean(Plan& p, const float* amp, float threshold, float2* w_out, cudaStream_t s);

// Message returned by sharp_last_error() on this thread (sharp_api.cu).
void set_last_error(const char* msg);

// Host-side schedule of one RAAR step of a plan (what the launches need).
struct StepInfo {
    int flags;           // RF_FORM_B | RF_METRIC
    int have_q, have_d, delta_is_norm, read_e, write_e, probe_due;
};
// sharp_api.cu: argument/state checks, scratch setup and the frame-pass
// arguments of step `iter`.  No GPU work is queued (the step's sums are
// cleared by raar_step_clear).
int raar_step_prepare(Plan& p, float2* c, float2* psiy, float2* psi, const float* amp, int iter, FrameArgs* a,
                      StepInfo* info);
cudaError_t raar_step_clear(Plan& p, cudaStream_t s);
// Launches after the frame pass (image pass, metrics, probe update) and the
// plan's bookkeeping.  mode 0: launch and update the bookkeeping; mode 1:
// bookkeeping only (a recorded graph issues the launches).  With
// `record_times` false no timing events are used.
int raar_step_finish(Plan& p, float2* c, float2* psiy, float2* psi, float2* probe, double* metrics, int iter,
                     const StepInfo& info, cudaStream_t s, bool record_times, int mode = 0);

// Batch frame pass (raar_batch_64.cu, raar_batch_128.cu)
// Frames of several scans in one persistent launch: scan s owns global frame
// indices base[s] .. base[s+1]-1.
struct BatchTable {
    const FrameArgs* scans;   // device array, one per scan
    const int* base;          // device array, nscans + 1 prefix sums of K
    int nscans;
    int total;                // base[nscans]
    int* counter;             // global frame counter (zeroed per launch)
    int* err;                 // batch status; a timeout also sets the scan's plan flag
    int stagger_ns;           // block b starts (b % 4) * stagger_ns after the launch (tile shape)
};
// The batch frame pass of frame size M with CH rows per load / epilogue
// round trip (64, 128: CH in {4, 8, 16}, one translation unit per pair).
template <int M, int CH>
cudaError_t launch_raar_batch_mc(int flags, const BatchTable& bt, int grid, cudaStream_t s);
inline cudaError_t launch_raar_batch(int m, int ch, int flags, const BatchTable& bt, int grid, cudaStream_t s) {
    if (m == 64) {
        if (ch == 4) return launch_raar_batch_mc<64, 4>(flags, bt, grid, s);
        if (ch == 8) return launch_raar_batch_mc<64, 8>(flags, bt, grid, s);
        if (ch == 16) return launch_raar_batch_mc<64, 16>(flags, bt, grid, s);
    } else if (m == 128) {
        if (ch == 4) return launch_raar_batch_mc<128, 4>(flags, bt, grid, s);
        if (ch == 8) return launch_raar_batch_mc<128, 8>(flags, bt, grid, s);
        if (ch == 16) return launch_raar_batch_mc<128, 16>(flags, bt, grid, s);
    }
    return cudaErrorInvalidValue;
}
template <int M>
cudaError_t raar_batch_max_grid(int* grid);

// slots of Plan::sums
enum SumSlot {
    S_RESID = 0,   // sum (a - |Fz|)^2  = ||P_a z - z||^2
    S_A2 = 1,      // sum a^2
    S_Z2 = 2,      // sum |z|^2
    S_Q = 3,       // sum |w_f psi - z|^2
    S_D = 4,       // sum |w_f psi_y + e|^2
};

}  // namespace sharp

// The opaque handle of the C ABI.
struct sharp_plan_s {
    sharp::Plan p;
};
