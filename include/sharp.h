/*
 * sharp.h -- C ABI of the GB300 (sm_103a) RAAR ptychography hot path.
 *
 * The library implements one iteration of RAAR (relaxed averaged alternating
 * reflections) over all diffraction frames of a ptychographic scan, as set out
 * in Marchesini et al., "SHARP: a distributed, GPU-based ptychographic
 * solver", arXiv:1602.01448, Sec. 2 (forward model, Eqs. 1-6; projections and
 * updates, Eqs. 7-10 and the reconstruction sequence of Sec. 2.2; metrics,
 * Eqs. 11-14).
 *
 * Notation (Sec. 2.1): K frames of m x m pixels, object psi of ny x nx pixels,
 * illumination (probe) w of m x m pixels, integer frame positions x_(i).
 *
 * Conventions for every entry point:
 *  - Array pointers are DEVICE pointers unless a comment says HOST.  They are
 *    owned by the caller, row-major and contiguous.  Complex values are
 *    float2 {re, im} (complex64).  Frames are stored frame-major: K x m x m.
 *  - Positions are int32 pairs (row, col): the top-left object pixel of each
 *    frame (the grid x_(i) = (r mu', r nu') of Sec. 2.1).
 *  - Fourier amplitudes are on the unitary scale of Eq. 2: a = sqrt(I) / m
 *    when I = |DFT|^2 of the unnormalised e^{-2 pi i} transform.  The forward
 *    DFT is the unitary e^{-2 pi i q.r} transform.
 *  - Work is queued on the given stream; no call synchronises it unless its
 *    comment says so.  A plan holds scratch buffers, so calls on one plan
 *    must not overlap on the GPU (use one stream per plan).
 *  - Every call returns SHARP_OK or an error code; the message of the last
 *    error of the calling thread is available from sharp_last_error().
 *    Sizes the kernels do not implement return SHARP_ERR_UNSUPPORTED_SIZE:
 *    there is no CPU fallback.
 *  - Scalar results (losses, residuals, metrics) are written to DEVICE
 *    doubles so that calls stay asynchronous.
 */
#ifndef SHARP_H
#define SHARP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHARP_OK                   0
#define SHARP_ERR_INVALID_ARG      1  /* null pointer, bad size, position out of range, ... */
#define SHARP_ERR_UNSUPPORTED_SIZE 2  /* frame size without a kernel (m not in {64,128,256}) */
#define SHARP_ERR_CUDA             3  /* a CUDA runtime call or launch failed */
#define SHARP_ERR_TIMEOUT          4  /* a bounded device-side wait gave up */
#define SHARP_ERR_STATE            5  /* call order violated (e.g. step before init) */

#define SHARP_PREC_FP32            0  /* FP32 data and transforms, FP64 global sums */
/*
 * Tensor-core precision modes (m = 128 or 256).  The 2D DFTs of the RAAR
 * frame pass (sharp_raar_step) and of the data projection
 * (sharp_fourier_project) run as contractions with the 128 x 128 DFT matrix
 * of Eq. 2 on the tensor cores, FP32 accumulation (a 256-point transform is
 * split once, radix 2, into 128-point ones); data, metrics and every other
 * operator stay FP32 / FP64.
 *   SHARP_PREC_FP16S  : FP16 operands scaled per frame by powers of two so
 *                       that FP16's range is never left: each transform's
 *                       input by the one that maps its largest component into
 *                       [2^14, 2^15), the intermediate between the
 *                       transform's two contractions by 2^-4 (its components
 *                       are at most 16 times the input's largest).
 *                       Relative error of one transform ~1e-3 (RMS ~3e-4).
 *   SHARP_PREC_BF16X3 : BF16 operands split x = hi + lo, three products
 *                       hi.hi + hi.lo + lo.hi per real product.  Relative
 *                       error of one transform ~1e-5.
 */
#define SHARP_PREC_FP16S           1
#define SHARP_PREC_BF16X3          2

typedef struct sharp_plan_s* sharp_plan;

/* Options of the reconstruction (Sec. 2.3 user options; Sec. 2.2 sequence). */
typedef struct {
    float beta;          /* RAAR relaxation beta in (0.5, 1]; 0.75 by default (Sec. 2.2) */
    int   wrap;          /* 1: object indexed modulo its size (periodic boundary, Fig. 3) */
    int   probe_every;   /* refine the probe (Eq. 10) on steps with iter % probe_every == 0; 0 = never */
    int   residual_every;/* eps_Q and eps_Delta (Eqs. 12, 13) on steps with iter % residual_every == 0; 0 = never */
    int   precision;     /* SHARP_PREC_FP32, or SHARP_PREC_FP16S / SHARP_PREC_BF16X3 (m = 128, 256) */
} sharp_params;

/* Message of the last failed call on this thread ("" if none).  Never NULL. */
const char* sharp_last_error(void);

/* Library version string, e.g. "sharp-gb300 0.1 (sm_103a)". */
const char* sharp_version(void);

/* Fills *p with the defaults: beta 0.75, wrap 0, probe_every 0,
 * residual_every 1, precision FP32. */
void sharp_default_params(sharp_params* p);

/*
 * Create a plan for K frames of m x m over an ny x nx object.
 *   pos    : DEVICE int32[K][2] (row, col) top-left corners.  Copied; the call
 *            synchronises `stream` to read them.  Without wrap every frame must
 *            lie inside the object (0 <= row <= ny-m, 0 <= col <= nx-m); with
 *            wrap positions are reduced modulo (ny, nx).
 *   params : copied; NULL means sharp_default_params().
 * Allocates the plan's scratch (illumination sum, overlap accumulators,
 * per-tile frame lists, reduction buffers; for m = 256 also one m x m
 * transposition slab per SM, 78 MB on 152 SMs).  The per-block lists of frames
 * that touch each image block (Sec. 2.3) are built here once, on the host.
 * With a tensor-core precision mode the plan also holds the 128 x 128 DFT
 * matrix parts (64 KB for FP16S, 128 KB for BF16X3).
 * Errors: INVALID_ARG (K < 1, ny or nx < m, bad position, beta outside
 * (0.5, 1], unknown precision), UNSUPPORTED_SIZE (m without a kernel, or a
 * tensor-core mode with m = 64).
 */
int sharp_plan_create(sharp_plan* plan, int K, int m, int ny, int nx,
                      const int32_t* pos, const sharp_params* params,
                      cudaStream_t stream);

/* Release a plan and its scratch (synchronises the device). NULL is a no-op. */
int sharp_plan_destroy(sharp_plan plan);

/*
 * Split operator Q (Sec. 2.1, Eqs. 5-6): frames[i](r) = probe(r) * obj(r + x_(i)).
 *   obj    : float2[ny][nx];  probe : float2[m][m];  frames : float2[K][m][m] (output).
 */
int sharp_q_gather(sharp_plan plan, const float2* obj, const float2* probe,
                   float2* frames, cudaStream_t stream);

/*
 * Data projection P_a (Eq. 7): out = F* (F z / |F z|) a, frame by frame, with
 * phase 1 where F z = 0.  in-place (out == z) is allowed.
 *   z, out   : float2[K][m][m];  amp : float[K][m][m] (unitary scale).
 *   resid_sq : DEVICE double[1] or NULL; receives ||P_a z - z||^2 (overwritten).
 * In the tensor-core precision modes z and amp must be 16-byte aligned (INVALID_ARG).
 */
int sharp_fourier_project(sharp_plan plan, const float2* z, const float* amp,
                          float2* out, double* resid_sq, cudaStream_t stream);

/*
 * Object update and overlap projection (Eqs. 8-9):
 *   obj_out = (Q*Q)^{-1} Q* z, 0 where Q*Q <= 1e-12 max(Q*Q);
 *   z_out   = Q obj_out = P_Q z (may be NULL).
 * Q* z is gathered per 32x32 image tile over the frames covering that tile
 * (no atomics, deterministic).
 *   probe : float2[m][m];  z : float2[K][m][m];  obj_out : float2[ny][nx].
 */
int sharp_overlap_project(sharp_plan plan, const float2* probe, const float2* z,
                          float2* obj_out, float2* z_out, cudaStream_t stream);

/*
 * Probe update on explicit frames (Eq. 10):
 *   probe_out(r) = sum_i conj(obj(r+x_i)) z_i(r) / sum_i |obj(r+x_i)|^2,
 * keeping probe_old(r) where the denominator is <= 1e-12 of its maximum.
 *   obj : float2[ny][nx];  z : float2[K][m][m];  probe_old, probe_out : float2[m][m].
 */
int sharp_probe_update(sharp_plan plan, const float2* obj, const float2* z,
                       const float2* probe_old, float2* probe_out, cudaStream_t stream);

/*
 * Illumination refinement after each probe update (Sec. 2.2: the real-space
 * drift and Fourier-space pathologies; reconstruction sequence step 7).
 * With F the unitary transform of Eq. 2:
 *   SHARP_PROBE_CONSTRAINT_MASK      : w <- F^-1{(F w) m_w}
 *   SHARP_PROBE_CONSTRAINT_AMPLITUDE : w <- F^-1{a_w (F w)/|F w|}  (phase 1 where F w = 0)
 * then, with center_of_mass != 0, w is rolled periodically within the frame
 * by -d, d = floor(c - m/2 + 1/2) per axis, c the centre of mass of |w|^2 over
 * frame indices 0..m-1 (the object follows through the next object update).
 *   values : float[m][m] device array (mask or amplitudes), copied into the
 *            plan; NULL with SHARP_PROBE_CONSTRAINT_NONE.
 * sharp_plan_set_probe_refinement configures what sharp_raar_step (and the
 * batch) applies after Eq. 10; sharp_probe_refine applies it to a given probe
 * (probe_out may equal probe_in).  Set it before a batch records its steps.
 * Errors: INVALID_ARG (unknown kind, values missing), CUDA.
 */
#define SHARP_PROBE_CONSTRAINT_NONE 0
#define SHARP_PROBE_CONSTRAINT_MASK 1
#define SHARP_PROBE_CONSTRAINT_AMPLITUDE 2
int sharp_plan_set_probe_refinement(sharp_plan plan, int constraint, const float* values, int center_of_mass,
                                    cudaStream_t stream);
int sharp_probe_refine(sharp_plan plan, const float2* probe_in, float2* probe_out, cudaStream_t stream);

/*
 * Initial illumination from the average frame (Sec. 2.2 reconstruction
 * sequence step 2; threshold variant of Sec. 3.2):
 *   I(q)   = (1/K) sum_i amp_i(q)^2                (amplitudes on the unitary scale)
 *   I'(q)  = I(q), or with 0 < threshold <= 1: 0 where I < threshold * max I and
 *            the mean of the remaining values elsewhere
 *   probe_out = F^-1 sqrt(I') rolled by m/2 per axis (centred in the frame).
 *   amp : float[K][m][m];  probe_out : float2[m][m].
 * Errors: INVALID_ARG (threshold outside [0, 1]), CUDA.
 */
int sharp_probe_init_mean(sharp_plan plan, const float* amp, float threshold, float2* probe_out,
                          cudaStream_t stream);

/*
 * Start a RAAR reconstruction from z^(0) = Q psi^(0) (Sec. 2.2 sequence).
 * The frames are kept implicitly as z = w_f . psi_y(r + x_i) + c_i, where w_f
 * is the probe that formed them; this call sets c = 0, psi_y = psi0, psi = psi0
 * and makes probe0 the plan's current probe (computing Q*Q).
 *   psi0 : float2[ny][nx];  probe0 : float2[m][m]
 *   state_c : float2[K][m][m] (output);  psi_y, psi : float2[ny][nx] (outputs).
 */
int sharp_raar_init(sharp_plan plan, const float2* psi0, const float2* probe0,
                    float2* state_c, float2* psi_y, float2* psi, cudaStream_t stream);

/*
 * One RAAR step, iteration number `iter` (1-based):
 *   z^(l) = [2b P_Q P_a + (1-2b) P_a + b (I - P_Q)] z^(l-1)       (Sec. 2.2, Luke form)
 *   psi^(l) = Q* z^(l) / Q*Q                                        (Eq. 9)
 *   if probe_every > 0 and iter % probe_every == 0: probe from Eq. 10.
 * One fused frame pass (gather, FFT, magnitude projection, inverse FFT,
 * overlap scatter-add, state update) plus one image pass.
 *   state_c, psi_y : in/out state from sharp_raar_init or the previous step.
 *   psi     : in: psi^(l-1) (read for eps_Q); out: psi^(l).
 *   probe   : float2[m][m] or NULL; receives the plan's current probe.
 *   amp     : float[K][m][m] measured amplitudes (unitary scale).
 *   metrics : DEVICE double[4] or NULL; for the iterate z^(l-1) entering the step:
 *             [0] eps_a (Eq. 11)  [1] eps_Q (Eq. 12, projector of the probe that
 *             formed z^(l-1))  [2] eps_Delta = ||z^(l-1) - z^(l-2)|| / ||a|| (Eq. 13,
 *             z^(-1) = 0)  [3] ||a||.  [1] and [2] are NaN off the residual cadence,
 *             and [2] is NaN when step iter-1 was not run on this plan.
 * Errors: STATE if the plan was not initialised with sharp_raar_init.
 */
int sharp_raar_step(sharp_plan plan, float2* state_c, float2* psi_y, float2* psi,
                    float2* probe, const float* amp, double* metrics, int iter,
                    cudaStream_t stream);

/*
 * Deterministic overlap sums.  By default the frame pass adds each frame's
 * contribution to the overlap sums Q*(.) of Eq. 9 with atomic additions, so
 * their FP32 rounding depends on the order in which frames finish and two
 * runs differ at rounding level.  With enable != 0 the frame pass scatters
 * nothing; the sums are gathered afterwards per 32 x 32 image tile over the
 * frames covering it, in a fixed order (one more read of the frame state per
 * step, and of the iterate on steps after a probe update), so the iterate,
 * object and probe of every step are bit-identical from run to run.  The
 * metrics are not: each block adds up its terms in FP32 over the frames it
 * happened to take, so they differ at FP32 rounding (about 1e-7 relative).
 * Single scans only
 * (sharp_batch_create rejects such plans).  Errors: INVALID_ARG.
 */
int sharp_plan_set_deterministic(sharp_plan plan, int enable);

/*
 * Checkpoint and resume of a RAAR reconstruction (the state of Sec. 2.2's
 * iteration).  The caller owns and saves state_c, psi_y and psi; the plan
 * holds the current probe, the probe that formed the iterate and the step
 * bookkeeping:
 *   sharp_raar_checkpoint copies the two probes (DEVICE float2[m][m] each)
 *   and fills info (HOST int[4]: last step run, whether the object equals
 *   Q* z / Q*Q, whether the probe changed at the last step, 0);
 *   sharp_raar_restore makes a plan over the same scan continue from such a
 *   record (probes copied, Q*Q recomputed), after the caller has restored
 *   state_c, psi_y and psi.  The next step must be info[0] + 1.  The buffer of
 *   eps_Delta is not part of the record: the first step after a restore that
 *   would read it reports eps_Delta as NaN.  With deterministic sums the
 *   resumed steps are bit-identical to uninterrupted ones.
 * Errors: INVALID_ARG, STATE (checkpoint before sharp_raar_init).
 */
int sharp_raar_checkpoint(sharp_plan plan, float2* probe_cur, float2* probe_form, int* info, cudaStream_t stream);
int sharp_raar_restore(sharp_plan plan, const float2* probe_cur, const float2* probe_form, const int* info,
                       cudaStream_t stream);

/*
 * Solution metric eps_0 (Eq. 14) at z = Q psi, z0 = Q psi_true:
 *   out[0] = min_phi ||D (e^{i phi} psi - psi_true)|| / ||D psi_true||, D = Q*Q of `probe`;
 *   out[1] = object NRMSE over pixels with D >= 0.1 max D, same phase rule.
 *   out : DEVICE double[2].
 */
int sharp_solution_error(sharp_plan plan, const float2* psi, const float2* psi_true,
                         const float2* probe, double* out, cudaStream_t stream);

/*
 * Forward model (Eq. 1): amp_out[i] = |F (probe . obj(r + x_i))| on the unitary scale.
 */
int sharp_forward_amplitudes(sharp_plan plan, const float2* obj, const float2* probe,
                             float* amp_out, cudaStream_t stream);

/*
 * Amplitude loss L = sum_i || |F Q(obj, probe)_i| - amp_i ||^2 (the least-squares
 * form of Eq. 1).  loss : DEVICE double[1] (overwritten).
 */
int sharp_amp_loss(sharp_plan plan, const float2* obj, const float2* probe,
                   const float* amp, double* loss, cudaStream_t stream);

/*
 * Adjoint of sharp_amp_loss.  With r_i = z_i - P_a z_i (frame FFTs recomputed):
 *   g_obj   = grad_scale * Q* r                   (dL/d conj(obj))
 *   g_probe = grad_scale * sum_i conj(obj(r+x_i)) r_i   (dL/d conj(probe))
 * Outputs are overwritten.  grad_scale = 2 gives PyTorch's convention for a
 * real loss of complex inputs.  g_probe may be NULL.
 */
int sharp_amp_loss_backward(sharp_plan plan, const float2* obj, const float2* probe,
                            const float* amp, double grad_scale, float2* g_obj,
                            float2* g_probe, cudaStream_t stream);

/*
 * Batched RAAR: independent scans (the multi-scan workloads of a streaming
 * beamline, Sec. 3.3) stepped together.  Each scan keeps its own plan, state,
 * amplitudes and probe; every sharp_batch_step(iter) performs one RAAR step
 * (as sharp_raar_step) for every scan with one persistent frame-pass launch
 * per frame size over the frames of all scans of that size, then each scan's
 * image pass, metrics and probe update.  The launch sequence of each distinct
 * step schedule is recorded as a CUDA graph on first use and replayed
 * afterwards.  The launch shape of each frame size is chosen by an autotuner
 * on the first steps: blocks per SM, rows per round trip of the frame pass's
 * gathers and scatter (4, 8, 16; 2, 4 for 256^2 frames) and the block-start
 * stagger, one parameter at a time, each candidate timed once; while it runs,
 * steps go without graphs and synchronise the stream.  The choice is kept for
 * the process per frame size and batch size class (frames rounded down to a
 * power of two), so later batches of the class start tuned.  Results do not
 * depend on the shape or on graphs beyond the order of the atomic sums.
 *   plans : nscans plans, already set up with sharp_raar_init; they must share
 *           probe_every and residual_every and be stepped only through the
 *           batch, and use SHARP_PREC_FP32.  The batch does not own them.
 * sharp_batch_bind gives scan `scan` its state buffers (as sharp_raar_step;
 * probe and metrics may be NULL); rebinding drops the recorded graphs.
 * sharp_batch_tuned_grid returns the grid chosen for frame size m (or -1);
 * sharp_batch_tuned_shape gives the whole shape (STATE while still tuning);
 * sharp_batch_set_shape fixes it instead (INVALID_ARG outside the
 * candidates; drops the recorded graphs).
 * sharp_batch_status synchronises `stream` and returns SHARP_ERR_TIMEOUT
 * (once) if a bounded wait of a batched frame pass gave up, or
 * SHARP_ERR_INVALID_ARG if a scan's measured amplitudes hold a value that is
 * not finite and non-negative; the affected scan's plan reports it through
 * sharp_plan_status as well.
 * Errors: INVALID_ARG, STATE (unbound scan, diverging schedules), CUDA.
 */
typedef struct sharp_batch_s* sharp_batch;
int sharp_batch_create(sharp_batch* batch, int nscans, const sharp_plan* plans);
int sharp_batch_bind(sharp_batch batch, int scan, float2* state_c, float2* psi_y, float2* psi, float2* probe,
                     const float* amp, double* metrics);
int sharp_batch_step(sharp_batch batch, int iter, cudaStream_t stream);
int sharp_batch_set_graphs(sharp_batch batch, int enable);
int sharp_batch_tuned_grid(sharp_batch batch, int m);
int sharp_batch_tuned_shape(sharp_batch batch, int m, int* grid, int* rows, int* stagger_ns);
int sharp_batch_set_shape(sharp_batch batch, int m, int grid, int rows, int stagger_ns);
int sharp_batch_status(sharp_batch batch, cudaStream_t stream);
int sharp_batch_destroy(sharp_batch batch);

/*
 * Data projection without device allocation.  The paper has no counterpart:
 * this entry point serves callers that must not allocate device memory while
 * they run -- hosts that own every device allocation, or real-time loops that
 * cannot risk the synchronisation an allocation may cause.  It needs no plan.
 *   z, out   : float2[K][m][m] (out == z allowed);  amp : float[K][m][m];
 *   resid_sq : DEVICE double[1] or NULL; receives ||P_a z - z||^2, summed over
 *              frames in frame order.
 *   Same result as sharp_fourier_project (Eq. 7, phase 1 where F z = 0).
 * Its only scratch, one residual per frame, lives in a fixed library-owned
 * device array of SHARP_NOALLOC_MAX_FRAMES doubles (512 KiB) that every GPU
 * using the library keeps until the process exits; K above that limit
 * returns SHARP_ERR_INVALID_ARG.  The first call on each device looks up the
 * array's device address (make it before any stream capture).  All calls
 * share the array: calls that overlap on the GPU race, so serialise them.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE (m not 64 or 128), CUDA.
 */
#define SHARP_NOALLOC_MAX_FRAMES 65536
int sharp_fourier_project_noalloc(const float2* z, const float* amp, float2* out, double* resid_sq,
                                  int K, int m, cudaStream_t stream);

/*
 * Synchronise `stream` and report a sticky device-side failure of the plan's
 * kernels, then clear it:
 *   SHARP_ERR_TIMEOUT     a bounded wait for a bulk copy or for tensor-core
 *                         work gave up (the affected step's results are invalid);
 *   SHARP_ERR_INVALID_ARG a frame pass read a measured amplitude that is not
 *                         finite and non-negative (Eq. 1: a = |F z|), or the
 *                         probe gives no finite positive illumination Q*Q
 *                         anywhere (all zero or not finite; sharp_raar_init,
 *                         probe updates, sharp_overlap_project).
 * The first error raised since the last call is reported.
 */
int sharp_plan_status(sharp_plan plan, cudaStream_t stream);

/*
 * Poll limit of the bounded device-side waits of the plan's frame passes
 * (the first wait for each bulk copy of frame data and for each group of
 * tensor-core MMAs).  Not part of the method: a watchdog setting.
 *   polls < 0 : the default, 2^26 polls (seconds of waiting);
 *   polls = 0 : no polling, so every such wait gives up at once (a frame
 *               pass then stops early and sharp_plan_status reports
 *               SHARP_ERR_TIMEOUT; used to exercise the error path);
 *   polls > 0 : that many polls (at most 2^32 - 2).
 * Whatever the setting, a kernel whose wait gave up waits with the default
 * limit for its own copies and MMAs still in flight before it exits, and
 * releases its tensor memory.  Applies to the launches queued after the call.
 * Errors: INVALID_ARG.
 */
int sharp_plan_set_wait_limit(sharp_plan plan, long long polls);

/*
 * Kernel timing (tracing aid; the paper reports per-kernel time shares in the
 * Fig. 3 caption).  When enabled, every kernel launch of the plan is bracketed
 * by CUDA events on the launching stream, classified as
 *   0 frame pass (fused gather/FFT/projection/scatter), 1 image pass
 *   (normalisation), 2 probe update (Eq. 10), 3 illumination sum Q*Q,
 *   4 other (metrics, split, overlap gather, small kernels).
 * sharp_plan_kernel_times synchronises the recorded events and returns, per
 * class, ms_out[c] = total milliseconds and launches_out[c] = number of
 * launches since the last call (both arrays of 5; either may be NULL), then
 * resets the counters.  Profiling adds an event pair per launch; leave it off
 * for production runs.
 */
#define SHARP_KCLASS_COUNT 5
int sharp_plan_set_profiling(sharp_plan plan, int enable);
int sharp_plan_kernel_times(sharp_plan plan, double* ms_out, int* launches_out);

#ifdef __cplusplus
}
#endif

#endif /* SHARP_H */
