// C ABI of the library (include/sharp.h): argument checks, plan scratch,
// per-block frame lists, and the order of kernel launches of each call.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sharp_common.cuh"
#include "tma.cuh"

using sharp::Plan;

namespace {

// Kernel timing: an event pair per launch, read back on demand.
struct Prof {
    struct Rec { int cls, kernels; cudaEvent_t a, b; };
    std::vector<Rec> live;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

enum KClass { K_FRAME = 0, K_IMAGE = 1, K_PROBE = 2, K_ILLUM = 3, K_OTHER = 4 };

// Bracket the launches issued by `body` with events when profiling is on.
template <class F>
cudaError_t timed(Plan& p, int cls, int kernels, cudaStream_t s, F body) {
    Prof* pr = static_cast<Prof*>(p.prof);
    if (!pr) return body();
    cudaEvent_t a = pr->get(), b = pr->get();
    cudaEventRecord(a, s);
    cudaError_t e = body();
    cudaEventRecord(b, s);
    pr->live.push_back({cls, kernels, a, b});
    return e;
}

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define SHARP_CK(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(SHARP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define SHARP_NONNULL(ptr)                                                               \
    do {                                                                                 \
        if (!(ptr)) return fail(SHARP_ERR_INVALID_ARG, "%s: %s is NULL", __func__, #ptr); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

bool supported_m(int m) { return m == 64 || m == 128 || m == 256; }

void free_plan(Plan& p) {
    void* ptrs[] = {p.pos,   p.tile_ptr,   p.tile_frames, p.w_cur, p.w_form,     p.w2,
                    p.Dsum,  p.invD,       p.dmax_bits,   p.accA,  p.accB,       p.ebuf,
                    p.sums,  p.probe_part, p.probe_acc,   p.scal,  p.w2tmp,      p.Dtmp,
                    p.invDtmp, p.errflag, p.counter, p.big_scratch, p.probe_cons, p.w_tmp,
                    p.dft_tab};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    std::memset(&p, 0, sizeof(p));
}

sharp::FrameArgs base_args(const Plan& p) {
    sharp::FrameArgs a;
    std::memset(&a, 0, sizeof(a));
    a.K = p.K;
    a.m = p.m;
    a.ny = p.ny;
    a.nx = p.nx;
    a.wrap = p.prm.wrap;
    a.pos = p.pos;
    a.beta = p.prm.beta;
    a.sums = p.sums;
    a.err = p.errflag;
    a.scratch = p.big_scratch;
    a.counter = p.counter;
    a.dft_tab = p.dft_tab;
    a.spin = p.wait_spin;
    return a;
}

// The m x m unitary DFT matrix F[k][n] = e^{-2 pi i kn/m} / sqrt(m) (Eq. 2) as
// the A operand of the tensor-core contraction kernels: parts {F_r, F_i} in
// FP16 (SHARP_PREC_FP16S) or {F_r hi, F_r lo, F_i hi, F_i lo} in BF16
// (SHARP_PREC_BF16X3, lo = bf16(F - hi)), each part in the canonical K-major
// no-swizzle layout: core matrix (k/8, n/8) of 8 rows x 8 values at byte
// ((n/8) * (m/8) + k/8) * 128, row k%8 at +16 (k%8), value n%8 at +2 (n%8).
std::vector<uint16_t> dft_table(int prec, int m) {
    const int parts = prec == SHARP_PREC_FP16S ? 2 : 4;
    const size_t mm = (size_t)m * m;
    std::vector<uint16_t> t(parts * mm, 0);
    const double pi = 3.14159265358979323846, s = 1.0 / std::sqrt((double)m);
    for (int k = 0; k < m; ++k)
        for (int n = 0; n < m; ++n) {
            const double ang = 2.0 * pi * (double)(((long long)k * n) % m) / m;
            const double v[2] = {std::cos(ang) * s, -std::sin(ang) * s};
            const size_t off = ((size_t)(n / 8) * (m / 8) + k / 8) * 64 + (k % 8) * 8 + (n % 8);
            for (int c = 0; c < 2; ++c) {
                if (prec == SHARP_PREC_FP16S) {
                    const __half_raw h = __double2half(v[c]);
                    t[c * mm + off] = h.x;
                } else {
                    const __nv_bfloat16 hi = __double2bfloat16(v[c]);
                    const __nv_bfloat16 lo = __double2bfloat16(v[c] - (double)__bfloat162float(hi));
                    t[(2 * c) * mm + off] = static_cast<__nv_bfloat16_raw>(hi).x;
                    t[(2 * c + 1) * mm + off] = static_cast<__nv_bfloat16_raw>(lo).x;
                }
            }
        }
    return t;
}

bool mixed(const Plan& p) { return p.prm.precision != SHARP_PREC_FP32; }

int check_plan(sharp_plan plan) {
    if (!plan) return fail(SHARP_ERR_INVALID_ARG, "plan is NULL");
    return SHARP_OK;
}

}  // namespace

void sharp::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

cudaError_t sharp::launch_mixed(int prec, int mode, int flags, const FrameArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    if (!a.dft_tab) return cudaErrorInvalidValue;
    if (a.m == 128) {
        if (prec == SHARP_PREC_FP16S) return launch_mixed_prec<SHARP_PREC_FP16S>(mode, flags, a, s);
        if (prec == SHARP_PREC_BF16X3) return launch_mixed_prec<SHARP_PREC_BF16X3>(mode, flags, a, s);
    } else if (a.m == 256) {
        if (prec == SHARP_PREC_FP16S) return launch_mixed256_prec<SHARP_PREC_FP16S>(mode, flags, a, a.scratch, s);
        if (prec == SHARP_PREC_BF16X3) return launch_mixed256_prec<SHARP_PREC_BF16X3>(mode, flags, a, a.scratch, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t sharp::raar_step_clear(Plan& p, cudaStream_t s) {
    return cudaMemsetAsync(p.sums, 0, 8 * sizeof(double), s);
}

int sharp::raar_step_prepare(Plan& p, float2* state_c, float2* psi_y, float2* psi, const float* amp, int iter,
                             sharp::FrameArgs* out, sharp::StepInfo* info) {
    SHARP_NONNULL(state_c); SHARP_NONNULL(psi_y); SHARP_NONNULL(psi); SHARP_NONNULL(amp);
    if (!p.initialised) return fail(SHARP_ERR_STATE, "RAAR step before sharp_raar_init");
    if ((reinterpret_cast<uintptr_t>(state_c) | reinterpret_cast<uintptr_t>(amp)) & 15)
        return fail(SHARP_ERR_INVALID_ARG, "state_c and amp must be 16-byte aligned (bulk copies)");
    if (iter < 1) return fail(SHARP_ERR_INVALID_ARG, "iter = %d < 1", iter);
    const size_t mm = (size_t)p.m * p.m;
    const int R = p.prm.residual_every;
    const bool cadence = R > 0 && iter % R == 0;
    sharp::StepInfo in;
    std::memset(&in, 0, sizeof(in));
    in.write_e = (R > 0 && (iter + 1) % R == 0) ? 1 : 0;
    if (!p.b_valid) in.flags |= sharp::RF_FORM_B;
    if (cadence) {
        in.flags |= sharp::RF_METRIC;
        in.have_q = 1;
        if (p.last_iter == 0) {
            in.have_d = 1;
            in.delta_is_norm = 1;   // z^(-1) = 0
        } else if (p.e_written_iter == iter - 1 && p.last_iter == iter - 1) {
            in.have_d = 1;
            in.read_e = 1;
        }
    }
    in.probe_due = (p.prm.probe_every > 0 && iter % p.prm.probe_every == 0) ? 1 : 0;
    if ((in.read_e || in.write_e) && !p.ebuf) {
        SHARP_CK(dalloc(&p.ebuf, (size_t)p.K * mm));
    }
    sharp::FrameArgs a = base_args(p);
    a.c = state_c;
    a.psiy = psi_y;
    a.psi = psi;
    a.ebuf = p.ebuf;
    a.w_form = p.w_form;
    a.w_proj = p.w_cur;
    a.accA = p.accA;
    a.accB = p.accB;
    a.amp = amp;
    a.read_e = in.read_e;
    a.write_e = in.write_e;
    a.no_scatter = p.deterministic;
    *out = a;
    *info = in;
    return SHARP_OK;
}

int sharp::raar_step_finish(Plan& p, float2* state_c, float2* psi_y, float2* psi, float2* probe, double* metrics,
                            int iter, const sharp::StepInfo& in, cudaStream_t s, bool record_times, int mode) {
    void* prof = p.prof;
    if (!record_times) p.prof = nullptr;
    const size_t mm = (size_t)p.m * p.m;
    const int form_b = (in.flags & sharp::RF_FORM_B) ? 1 : 0;
    int rc = SHARP_OK;
    const bool dry = mode == 1;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == SHARP_OK) rc = fail(SHARP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    // in bookkeeping-only mode every launch below is skipped
    auto timed_or_skip = [&](int cls, int kernels, auto body) -> cudaError_t {
        return dry ? cudaSuccess : timed(p, cls, kernels, s, body);
    };
    ck(timed_or_skip(K_IMAGE, 1, [&] { return sharp::launch_normalise(p, psi_y, psi, form_b, s); }), "normalise");
    p.b_valid = true;   // Q* z^(l) / D = psi^(l) for the next step
    if (p.form_differs) {
        if (!dry)
            ck(cudaMemcpyAsync(p.w_form, p.w_cur, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s), "probe copy");
        p.form_differs = false;
    }
    if (metrics)
        ck(timed_or_skip(K_OTHER, 1, [&] {
               return sharp::launch_metrics_finalize(p, metrics, in.have_q, in.have_d, in.delta_is_norm, s);
           }), "metrics");
    if (in.probe_due) {
        ck(timed_or_skip(K_PROBE, 3, [&] { return sharp::launch_probe_update_state(p, state_c, psi_y, psi, s); }),
           "probe update");
        if (p.probe_com || (p.probe_cons_kind && p.probe_cons))
            ck(timed_or_skip(K_PROBE, 2, [&] { return sharp::launch_probe_refine(p, p.w_cur, p.w_cur, s); }),
               "probe refinement");
        ck(timed_or_skip(K_ILLUM, 3, [&] {
               return sharp::launch_illumination(p, p.w_cur, p.w2, p.Dsum, p.invD, p.dmax_bits, s);
           }), "illumination");
        p.b_valid = false;
        p.form_differs = true;
    }
    if (probe && !dry)
        ck(cudaMemcpyAsync(probe, p.w_cur, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s), "probe out");
    p.e_written_iter = in.write_e ? iter : 0;
    p.last_iter = iter;
    p.prof = prof;
    return rc;
}

extern "C" {

const char* sharp_last_error(void) { return g_err.c_str(); }

const char* sharp_version(void) { return "sharp-gb300 0.1 (sm_103a)"; }

void sharp_default_params(sharp_params* p) {
    if (!p) return;
    p->beta = 0.75f;
    p->wrap = 0;
    p->probe_every = 0;
    p->residual_every = 1;
    p->precision = SHARP_PREC_FP32;
}

int sharp_plan_create(sharp_plan* out, int K, int m, int ny, int nx, const int32_t* pos,
                      const sharp_params* params, cudaStream_t stream) {
    g_err.clear();
    SHARP_NONNULL(out);
    *out = nullptr;
    SHARP_NONNULL(pos);
    if (K < 1) return fail(SHARP_ERR_INVALID_ARG, "K = %d < 1", K);
    if (m < 1 || ny < m || nx < m) return fail(SHARP_ERR_INVALID_ARG, "need 1 <= m <= ny, nx (m=%d ny=%d nx=%d)", m, ny, nx);
    if (!supported_m(m)) return fail(SHARP_ERR_UNSUPPORTED_SIZE, "frame size m=%d has no kernel (64, 128, 256)", m);
    if ((long long)ny * nx > (1LL << 30) || (long long)K * m * m > (1LL << 34))
        return fail(SHARP_ERR_INVALID_ARG, "problem too large for 32-bit pixel indexing");
    sharp_params prm;
    sharp_default_params(&prm);
    if (params) prm = *params;
    // RAAR's relaxation range (Sec. 2.2).  At b = 1/2 the new state
    // (1-2b) P_a z + b z carries no trace of P_a z, and the image pass
    // recovers Q* P_a z with the factor 1/(1-2b).
    if (!(prm.beta > 0.5f && prm.beta <= 1.f))
        return fail(SHARP_ERR_INVALID_ARG, "beta = %g outside (0.5, 1]", prm.beta);
    if (prm.probe_every < 0 || prm.residual_every < 0) return fail(SHARP_ERR_INVALID_ARG, "negative cadence");
    if (prm.precision != SHARP_PREC_FP32 && prm.precision != SHARP_PREC_FP16S && prm.precision != SHARP_PREC_BF16X3)
        return fail(SHARP_ERR_INVALID_ARG, "unknown precision %d", prm.precision);
    if (prm.precision != SHARP_PREC_FP32 && m != 128 && m != 256)
        return fail(SHARP_ERR_UNSUPPORTED_SIZE, "tensor-core precision modes need m = 128 or 256 (m = %d)", m);

    std::vector<int32_t> hpos((size_t)K * 2);
    SHARP_CK(cudaMemcpyAsync(hpos.data(), pos, hpos.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    SHARP_CK(cudaStreamSynchronize(stream));
    for (int i = 0; i < K; ++i) {
        int r = hpos[2 * i], c = hpos[2 * i + 1];
        if (prm.wrap) {
            r %= ny; if (r < 0) r += ny;
            c %= nx; if (c < 0) c += nx;
            hpos[2 * i] = r;
            hpos[2 * i + 1] = c;
        } else if (r < 0 || c < 0 || r > ny - m || c > nx - m) {
            return fail(SHARP_ERR_INVALID_ARG, "frame %d at (%d, %d) leaves the %dx%d object (no wrap)", i, r, c, ny, nx);
        }
    }
    // per-tile frame lists: the tiles each frame touches (wrap-aware)
    const int tiles_y = (ny + sharp::TILE - 1) / sharp::TILE;
    const int tiles_x = (nx + sharp::TILE - 1) / sharp::TILE;
    std::vector<std::vector<int>> rows_of(K), cols_of(K);
    std::vector<int> count((size_t)tiles_y * tiles_x + 1, 0);
    std::vector<char> mark_y(tiles_y), mark_x(tiles_x);
    for (int i = 0; i < K; ++i) {
        std::fill(mark_y.begin(), mark_y.end(), 0);
        std::fill(mark_x.begin(), mark_x.end(), 0);
        for (int d = 0; d < m; ++d) {
            mark_y[((hpos[2 * i] + d) % ny) / sharp::TILE] = 1;
            mark_x[((hpos[2 * i + 1] + d) % nx) / sharp::TILE] = 1;
        }
        for (int t = 0; t < tiles_y; ++t) if (mark_y[t]) rows_of[i].push_back(t);
        for (int t = 0; t < tiles_x; ++t) if (mark_x[t]) cols_of[i].push_back(t);
        for (int ty : rows_of[i]) for (int tx : cols_of[i]) count[(size_t)ty * tiles_x + tx + 1]++;
    }
    for (size_t t = 1; t < count.size(); ++t) count[t] += count[t - 1];
    const int nnz = count.back();
    std::vector<int> frames(nnz), fill(count.begin(), count.end() - 1);
    for (int i = 0; i < K; ++i)
        for (int ty : rows_of[i]) for (int tx : cols_of[i]) frames[fill[(size_t)ty * tiles_x + tx]++] = i;

    sharp_plan h = new sharp_plan_s;
    Plan& p = h->p;
    std::memset(&p, 0, sizeof(p));
    p.K = K; p.m = m; p.ny = ny; p.nx = nx; p.prm = prm;
    p.tiles_y = tiles_y; p.tiles_x = tiles_x; p.tile_nnz = nnz;
    {
        // 64 frames per chunk of the Eq. 10 partial sums (fewer, longer chunks
        // measured faster than 8-32 once the reduction is counted), more when
        // the partial buffer would pass 64 MB
        const long long max_chunks = std::max(1LL, (64LL << 20) / (12LL * m * m));
        p.probe_chunk_frames = std::max(64, (int)((K + max_chunks - 1) / max_chunks));
        p.probe_chunks = (K + p.probe_chunk_frames - 1) / p.probe_chunk_frames;
    }
    const size_t n = (size_t)ny * nx, mm = (size_t)m * m;
    cudaError_t e = cudaSuccess;
#define SHARP_ALLOC(field, count)                   \
    if (e == cudaSuccess) e = dalloc(&p.field, (count));
    SHARP_ALLOC(pos, (size_t)K * 2)
    SHARP_ALLOC(tile_ptr, count.size())
    SHARP_ALLOC(tile_frames, (size_t)std::max(nnz, 1))
    SHARP_ALLOC(w_cur, mm)
    SHARP_ALLOC(w_form, mm)
    SHARP_ALLOC(w2, mm)
    SHARP_ALLOC(Dsum, n)
    SHARP_ALLOC(invD, n)
    SHARP_ALLOC(dmax_bits, 4)
    SHARP_ALLOC(accA, n)
    SHARP_ALLOC(accB, n)
    SHARP_ALLOC(sums, 16)
    SHARP_ALLOC(probe_part, (size_t)p.probe_chunks * 3 * mm)
    SHARP_ALLOC(probe_acc, 3 * mm)
    SHARP_ALLOC(scal, 32)
    SHARP_ALLOC(w2tmp, mm)
    SHARP_ALLOC(Dtmp, n)
    SHARP_ALLOC(invDtmp, n)
    SHARP_ALLOC(errflag, 1)
    SHARP_ALLOC(counter, 1)
    SHARP_ALLOC(w_tmp, mm)
    if (m == 256) {   // one frame slab per SM for the line-pass transform
        int dev = 0, sms = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        SHARP_ALLOC(big_scratch, (size_t)sms * mm)
    }
    std::vector<uint16_t> dft;
    if (prm.precision != SHARP_PREC_FP32) {
        dft = dft_table(prm.precision, m == 256 ? 128 : m);   // 256^2 frames: four 128^2 sub-problems
        if (e == cudaSuccess) e = cudaMalloc(&p.dft_tab, dft.size() * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.dft_tab, dft.data(), dft.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, stream);
    }
#undef SHARP_ALLOC
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.pos, hpos.data(), hpos.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.tile_ptr, count.data(), count.size() * sizeof(int), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(p.tile_frames, frames.data(), (size_t)nnz * sizeof(int), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.scal, 0, 32 * sizeof(double), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.errflag, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host vectors die here
    if (e != cudaSuccess) {
        free_plan(p);
        delete h;
        return fail(SHARP_ERR_CUDA, "plan allocation: %s", cudaGetErrorString(e));
    }
    *out = h;
    return SHARP_OK;
}

int sharp_plan_status(sharp_plan plan, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    int flag = 0;
    SHARP_CK(cudaMemcpyAsync(&flag, plan->p.errflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SHARP_CK(cudaStreamSynchronize(s));
    if (flag != 0) {
        SHARP_CK(cudaMemsetAsync(plan->p.errflag, 0, sizeof(int), s));
        SHARP_CK(cudaStreamSynchronize(s));
        if (flag == SHARP_ERR_TIMEOUT)
            return fail(flag, "a bounded device-side wait gave up (the step's results are invalid)");
        if (flag == SHARP_ERR_INVALID_ARG)
            return fail(flag, "invalid data seen on the device: a measured amplitude that is not finite and "
                              "non-negative, or a probe without finite positive illumination");
        return fail(flag, "device-side error %d", flag);
    }
    return SHARP_OK;
}

int sharp_plan_set_deterministic(sharp_plan plan, int enable) {
    if (int r = check_plan(plan)) return r;
    plan->p.deterministic = enable ? 1 : 0;
    return SHARP_OK;
}

int sharp_raar_checkpoint(sharp_plan plan, float2* probe_cur, float2* probe_form, int* info, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(probe_cur); SHARP_NONNULL(probe_form); SHARP_NONNULL(info);
    Plan& p = plan->p;
    if (!p.initialised) return fail(SHARP_ERR_STATE, "checkpoint before sharp_raar_init");
    const size_t mm = (size_t)p.m * p.m;
    SHARP_CK(cudaMemcpyAsync(probe_cur, p.w_cur, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(cudaMemcpyAsync(probe_form, p.w_form, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    info[0] = p.last_iter;
    info[1] = p.b_valid ? 1 : 0;
    info[2] = p.form_differs ? 1 : 0;
    info[3] = 0;
    return SHARP_OK;
}

int sharp_raar_restore(sharp_plan plan, const float2* probe_cur, const float2* probe_form, const int* info,
                       cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(probe_cur); SHARP_NONNULL(probe_form); SHARP_NONNULL(info);
    Plan& p = plan->p;
    if (info[0] < 0 || (info[1] != 0 && info[1] != 1) || (info[2] != 0 && info[2] != 1))
        return fail(SHARP_ERR_INVALID_ARG, "checkpoint record out of range");
    const size_t n = (size_t)p.ny * p.nx, mm = (size_t)p.m * p.m;
    SHARP_CK(cudaMemcpyAsync(p.w_cur, probe_cur, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(cudaMemcpyAsync(p.w_form, probe_form, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(sharp::launch_illumination(p, p.w_cur, p.w2, p.Dsum, p.invD, p.dmax_bits, s));
    SHARP_CK(cudaMemsetAsync(p.accA, 0, n * sizeof(float2), s));
    SHARP_CK(cudaMemsetAsync(p.accB, 0, n * sizeof(float2), s));
    p.last_iter = info[0];
    p.b_valid = info[1] != 0;
    p.form_differs = info[2] != 0;
    p.e_written_iter = 0;   // the eps_Delta buffer is not part of a checkpoint
    p.initialised = true;
    return SHARP_OK;
}

int sharp_plan_set_wait_limit(sharp_plan plan, long long polls) {
    if (int r = check_plan(plan)) return r;
    if (polls > 0xfffffffeLL) return fail(SHARP_ERR_INVALID_ARG, "wait limit %lld above 2^32 - 2 polls", polls);
    plan->p.wait_spin = polls < 0 ? 0u : (polls == 0 ? sharp::kNoPolls : (unsigned)polls);
    return SHARP_OK;
}

int sharp_plan_set_profiling(sharp_plan plan, int enable) {
    if (int r = check_plan(plan)) return r;
    Plan& p = plan->p;
    if (enable && !p.prof) p.prof = new Prof();
    if (!enable && p.prof) {
        Prof* pr = static_cast<Prof*>(p.prof);
        cudaDeviceSynchronize();
        for (auto& r : pr->live) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pr->pool) cudaEventDestroy(e);
        delete pr;
        p.prof = nullptr;
    }
    return SHARP_OK;
}

int sharp_plan_kernel_times(sharp_plan plan, double* ms_out, int* launches_out) {
    if (int r = check_plan(plan)) return r;
    double ms[SHARP_KCLASS_COUNT] = {0, 0, 0, 0, 0};
    int cnt[SHARP_KCLASS_COUNT] = {0, 0, 0, 0, 0};
    Prof* pr = static_cast<Prof*>(plan->p.prof);
    if (pr) {
        for (auto& r : pr->live) {
            SHARP_CK(cudaEventSynchronize(r.b));
            float t = 0.f;
            SHARP_CK(cudaEventElapsedTime(&t, r.a, r.b));
            ms[r.cls] += t;
            cnt[r.cls] += r.kernels;
            pr->pool.push_back(r.a);
            pr->pool.push_back(r.b);
        }
        pr->live.clear();
    }
    for (int c = 0; c < SHARP_KCLASS_COUNT; ++c) {
        if (ms_out) ms_out[c] = ms[c];
        if (launches_out) launches_out[c] = cnt[c];
    }
    return SHARP_OK;
}

int sharp_plan_destroy(sharp_plan plan) {
    if (!plan) return SHARP_OK;
    cudaDeviceSynchronize();
    sharp_plan_set_profiling(plan, 0);
    free_plan(plan->p);
    delete plan;
    return SHARP_OK;
}

int sharp_q_gather(sharp_plan plan, const float2* obj, const float2* probe, float2* frames, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(obj); SHARP_NONNULL(probe); SHARP_NONNULL(frames);
    SHARP_CK(sharp::launch_q_gather(plan->p, obj, probe, frames, s));
    return SHARP_OK;
}

int sharp_fourier_project(sharp_plan plan, const float2* z, const float* amp, float2* out, double* resid_sq,
                          cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(z); SHARP_NONNULL(amp); SHARP_NONNULL(out);
    Plan& p = plan->p;
    SHARP_CK(cudaMemsetAsync(p.sums, 0, sizeof(double), s));
    sharp::FrameArgs a = base_args(p);
    a.zin = z;
    a.zout = out;
    a.amp = amp;
    if (mixed(p) && ((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(amp)) & 15))
        return fail(SHARP_ERR_INVALID_ARG, "z and amp must be 16-byte aligned in the tensor-core modes (bulk copies)");
    if (mixed(p)) SHARP_CK(sharp::launch_mixed(p.prm.precision, sharp::MODE_PROJECT, 0, a, s));
    else SHARP_CK(sharp::launch_frames(sharp::MODE_PROJECT, 0, a, s));
    if (resid_sq) SHARP_CK(sharp::launch_copy_scaled(p.sums, resid_sq, 1.0, s));
    return SHARP_OK;
}

int sharp_overlap_project(sharp_plan plan, const float2* probe, const float2* z, float2* obj_out, float2* z_out,
                          cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(probe); SHARP_NONNULL(z); SHARP_NONNULL(obj_out);
    Plan& p = plan->p;
    unsigned* dmax = reinterpret_cast<unsigned*>(p.scal + 3);
    SHARP_CK(sharp::launch_illumination(p, probe, p.w2tmp, p.Dtmp, p.invDtmp, dmax, s));
    SHARP_CK(sharp::launch_overlap_gather(p, probe, z, obj_out, s));
    SHARP_CK(sharp::launch_scale_invD(p, obj_out, p.invDtmp, s));
    if (z_out) SHARP_CK(sharp::launch_q_gather(p, obj_out, probe, z_out, s));
    return SHARP_OK;
}

int sharp_probe_update(sharp_plan plan, const float2* obj, const float2* z, const float2* probe_old,
                       float2* probe_out, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(obj); SHARP_NONNULL(z); SHARP_NONNULL(probe_old); SHARP_NONNULL(probe_out);
    if (probe_out == probe_old) return fail(SHARP_ERR_INVALID_ARG, "probe_out must not alias probe_old");
    SHARP_CK(sharp::launch_probe_update_frames(plan->p, obj, z, probe_old, probe_out, s));
    return SHARP_OK;
}

int sharp_plan_set_probe_refinement(sharp_plan plan, int constraint, const float* values, int center_of_mass,
                                    cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    Plan& p = plan->p;
    if (constraint < SHARP_PROBE_CONSTRAINT_NONE || constraint > SHARP_PROBE_CONSTRAINT_AMPLITUDE)
        return fail(SHARP_ERR_INVALID_ARG, "unknown probe constraint %d", constraint);
    if (constraint != SHARP_PROBE_CONSTRAINT_NONE && !values)
        return fail(SHARP_ERR_INVALID_ARG, "the probe constraint needs its m x m values");
    const size_t mm = (size_t)p.m * p.m;
    if (constraint != SHARP_PROBE_CONSTRAINT_NONE) {
        if (!p.probe_cons) SHARP_CK(dalloc(&p.probe_cons, mm));
        SHARP_CK(cudaMemcpyAsync(p.probe_cons, values, mm * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    p.probe_cons_kind = constraint;
    p.probe_com = center_of_mass ? 1 : 0;
    return SHARP_OK;
}

int sharp_probe_refine(sharp_plan plan, const float2* probe_in, float2* probe_out, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(probe_in); SHARP_NONNULL(probe_out);
    SHARP_CK(sharp::launch_probe_refine(plan->p, probe_in, probe_out, s));
    return SHARP_OK;
}

int sharp_probe_init_mean(sharp_plan plan, const float* amp, float threshold, float2* probe_out, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(amp); SHARP_NONNULL(probe_out);
    if (!(threshold >= 0.f && threshold <= 1.f))
        return fail(SHARP_ERR_INVALID_ARG, "threshold = %g outside [0, 1]", threshold);
    SHARP_CK(sharp::launch_probe_init_mean(plan->p, amp, threshold, probe_out, s));
    return SHARP_OK;
}

int sharp_raar_init(sharp_plan plan, const float2* psi0, const float2* probe0, float2* state_c, float2* psi_y,
                    float2* psi, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(psi0); SHARP_NONNULL(probe0); SHARP_NONNULL(state_c); SHARP_NONNULL(psi_y); SHARP_NONNULL(psi);
    Plan& p = plan->p;
    const size_t n = (size_t)p.ny * p.nx, mm = (size_t)p.m * p.m;
    SHARP_CK(cudaMemcpyAsync(p.w_cur, probe0, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(cudaMemcpyAsync(p.w_form, probe0, mm * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(sharp::launch_illumination(p, p.w_cur, p.w2, p.Dsum, p.invD, p.dmax_bits, s));
    SHARP_CK(cudaMemsetAsync(state_c, 0, (size_t)p.K * mm * sizeof(float2), s));
    if (psi_y != psi0) SHARP_CK(cudaMemcpyAsync(psi_y, psi0, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (psi != psi0) SHARP_CK(cudaMemcpyAsync(psi, psi0, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SHARP_CK(cudaMemsetAsync(p.accA, 0, n * sizeof(float2), s));
    SHARP_CK(cudaMemsetAsync(p.accB, 0, n * sizeof(float2), s));
    p.b_valid = true;   // z^(0) = Q psi0, so Q* z^(0) / D = psi0 = psi
    p.form_differs = false;
    p.e_written_iter = 0;
    p.last_iter = 0;
    p.initialised = true;
    return SHARP_OK;
}

int sharp_raar_step(sharp_plan plan, float2* state_c, float2* psi_y, float2* psi, float2* probe, const float* amp,
                    double* metrics, int iter, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    Plan& p = plan->p;
    sharp::FrameArgs a;
    sharp::StepInfo info;
    if (int r = sharp::raar_step_prepare(p, state_c, psi_y, psi, amp, iter, &a, &info)) return r;
    SHARP_CK(sharp::raar_step_clear(p, s));
    if (p.deterministic && (info.flags & sharp::RF_FORM_B)) {
        // B' = Q*(z - w psi) from the iterate entering the step (the frame
        // pass overwrites its state)
        SHARP_CK(timed(p, K_OTHER, 1, s, [&] {
            return sharp::launch_overlap_delta_gather(p, p.w_cur, p.w_form, state_c, psi_y, psi, 1.f, p.accB, s);
        }));
    }
    SHARP_CK(timed(p, K_FRAME, 1, s, [&] {
        return mixed(p) ? sharp::launch_mixed(p.prm.precision, sharp::MODE_RAAR, info.flags, a, s)
                        : sharp::launch_frames(sharp::MODE_RAAR, info.flags, a, s);
    }));
    if (p.deterministic) {
        // C' = Q*(c_new - (1-b) w psi) from the new state
        SHARP_CK(timed(p, K_OTHER, 1, s, [&] {
            return sharp::launch_overlap_delta_gather(p, p.w_cur, nullptr, state_c, nullptr, psi,
                                                      1.f - p.prm.beta, p.accA, s);
        }));
    }
    return sharp::raar_step_finish(p, state_c, psi_y, psi, probe, metrics, iter, info, s, true);
}

int sharp_solution_error(sharp_plan plan, const float2* psi, const float2* psi_true, const float2* probe,
                         double* out, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(psi); SHARP_NONNULL(psi_true); SHARP_NONNULL(probe); SHARP_NONNULL(out);
    SHARP_CK(sharp::launch_solution_error(plan->p, psi, psi_true, probe, out, s));
    return SHARP_OK;
}

int sharp_forward_amplitudes(sharp_plan plan, const float2* obj, const float2* probe, float* amp_out,
                             cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(obj); SHARP_NONNULL(probe); SHARP_NONNULL(amp_out);
    sharp::FrameArgs a = base_args(plan->p);
    a.obj = obj;
    a.probe = probe;
    a.amp_out = amp_out;
    SHARP_CK(sharp::launch_frames(sharp::MODE_AMPS, 0, a, s));
    return SHARP_OK;
}

int sharp_amp_loss(sharp_plan plan, const float2* obj, const float2* probe, const float* amp, double* loss,
                   cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(obj); SHARP_NONNULL(probe); SHARP_NONNULL(amp); SHARP_NONNULL(loss);
    Plan& p = plan->p;
    SHARP_CK(cudaMemsetAsync(p.sums, 0, sizeof(double), s));
    sharp::FrameArgs a = base_args(p);
    a.obj = obj;
    a.probe = probe;
    a.amp = amp;
    SHARP_CK(sharp::launch_frames(sharp::MODE_LOSS, 0, a, s));
    SHARP_CK(sharp::launch_copy_scaled(p.sums, loss, 1.0, s));
    return SHARP_OK;
}

int sharp_amp_loss_backward(sharp_plan plan, const float2* obj, const float2* probe, const float* amp,
                            double grad_scale, float2* g_obj, float2* g_probe, cudaStream_t s) {
    if (int r = check_plan(plan)) return r;
    SHARP_NONNULL(obj); SHARP_NONNULL(probe); SHARP_NONNULL(amp); SHARP_NONNULL(g_obj);
    Plan& p = plan->p;
    SHARP_CK(cudaMemsetAsync(g_obj, 0, (size_t)p.ny * p.nx * sizeof(float2), s));
    if (g_probe) SHARP_CK(cudaMemsetAsync(g_probe, 0, (size_t)p.m * p.m * sizeof(float2), s));
    SHARP_CK(cudaMemsetAsync(p.sums, 0, sizeof(double), s));
    sharp::FrameArgs a = base_args(p);
    a.obj = obj;
    a.probe = probe;
    a.amp = amp;
    a.g_obj = g_obj;
    a.g_probe = g_probe;
    a.gscale = (float)grad_scale;
    SHARP_CK(sharp::launch_frames(sharp::MODE_GRAD, 0, a, s));
    return SHARP_OK;
}

}  // extern "C"
