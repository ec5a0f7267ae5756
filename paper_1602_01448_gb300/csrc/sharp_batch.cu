// Batched RAAR: many independent scans stepped together.
//
// A batch groups plans (one per scan, each with its own state, amplitudes and
// probe).  Each step runs one persistent frame-pass launch per frame size over
// the frames of all scans of that size (raar_batch_kernel), then every scan's
// image pass, metrics and probe update.  The launch sequence of a step depends
// only on the step's schedule (flags, metric cadence, probe update), so it is
// recorded once per schedule as a CUDA graph and replayed afterwards.
//
// The launch shape of each frame-size group is chosen online by a small
// autotuner: the number of resident blocks per SM, the rows each thread loads
// and stores per round trip of the gathers and the scatter (the frame pass's
// tile shape: 4, 8 or 16 rows for 64^2 and 128^2 frames, 2 or 4 row pairs of
// the four quadrants for 256^2),
// and whether block starts are staggered.  The first steps time one
// candidate each with events around the group's frame pass, one parameter
// at a time (coordinate descent: grid, then rows, then stagger, each from the
// best so far), and keep the fastest.  None of these changes the arithmetic
// of a frame; only the order of the atomic overlap sums differs.  The choice
// is kept for the process, per frame size and size class of the batch
// (frames rounded down to a power of two), so later batches of that class
// start tuned.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "sharp_common.cuh"

namespace {

struct Bind {
    float2* c = nullptr;
    float2* psiy = nullptr;
    float2* psi = nullptr;
    float2* probe = nullptr;
    const float* amp = nullptr;
    double* metrics = nullptr;
};

struct Shape {                    // launch shape of a group's frame pass
    int grid = 0;                 // blocks (a multiple of the SM count)
    int ch = 8;                   // rows per load / epilogue round trip
    int stagger = 2000;           // ns between the starts of blocks b % 4 = 0, 1, 2, 3
};

struct Group {                    // scans of one frame size
    int m = 0;
    std::vector<int> scans;       // indices into the batch
    int total = 0;
    int* d_base = nullptr;
    float2* slab = nullptr;       // 256^2 frames: one frame of scratch per block
    int max_grid = 0;
    // autotuner: candidates of the current parameter, their times, the best so far
    int stage = 0;                // 0 grid, 1 rows, 2 stagger, 3 done
    std::vector<Shape> cand;
    std::vector<float> cand_ms;
    Shape best;
    float best_ms = -1.f;
    bool tuned = false;
};

// Tuned shapes of this process: (frame size, size class) -> shape.
std::mutex g_tuned_mutex;
std::map<std::pair<int, int>, Shape> g_tuned;

int size_class(int frames) {
    int c = 0;
    while ((frames >> (c + 1)) > 0) ++c;
    return c;
}

// Candidates of the next tuner stage (each differs from g.best in one
// parameter); false when no stage is left.
bool next_stage(Group& g, int sms) {
    g.cand.clear();
    while (g.cand.empty() && g.stage < 3) {
        if (g.stage == 0) {
            for (int k = 1; k * sms <= g.max_grid; ++k) {
                Shape s = g.best;
                s.grid = k * sms;
                g.cand.push_back(s);
            }
            if (g.cand.empty()) {
                Shape s = g.best;
                s.grid = g.max_grid;
                g.cand.push_back(s);
            }
        } else if (g.stage == 1) {
            for (int ch : (g.m == 256 ? std::vector<int>{2, 4} : std::vector<int>{4, 8, 16}))
                if (ch != g.best.ch) {
                    Shape s = g.best;
                    s.ch = ch;
                    g.cand.push_back(s);
                }
        } else {
            Shape s = g.best;
            s.stagger = g.best.stagger ? 0 : 2000;
            g.cand.push_back(s);
        }
        ++g.stage;
    }
    g.cand_ms.assign(g.cand.size(), -1.f);
    return !g.cand.empty();
}

// Record the time of candidate k; move on when the stage is complete.
void tuner_record(Group& g, int k, float ms, int sms) {
    g.cand_ms[k] = ms;
    for (float t : g.cand_ms)
        if (t < 0.f) return;
    for (size_t j = 0; j < g.cand.size(); ++j)
        if (g.best_ms < 0.f || g.cand_ms[j] < g.best_ms) {
            g.best_ms = g.cand_ms[j];
            g.best = g.cand[j];
        }
    if (!next_stage(g, sms)) {
        g.tuned = true;
        std::lock_guard<std::mutex> lk(g_tuned_mutex);
        g_tuned[{g.m, size_class(g.total)}] = g.best;
    }
}

struct Schedule {                 // one distinct step schedule
    cudaGraphExec_t exec = nullptr;            // its recorded launches (graphs on, tuning done)
    std::vector<sharp::FrameArgs*> tables;     // device FrameArgs of each group's scans
};

int bfail(int code, const std::string& msg) {
    sharp::set_last_error(msg.c_str());
    return code;
}

}  // namespace

struct sharp_batch_s {
    std::vector<sharp_plan> plans;
    std::vector<Bind> binds;
    std::vector<Group> groups;
    int* counter = nullptr;
    int* err = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<uint64_t, Schedule> schedules;
    int use_graphs = 1;
};

namespace {

cudaError_t launch_group(const Group& g, const sharp::FrameArgs* table, int flags, const Shape& sh, int* counter,
                         int* err, cudaStream_t s) {
    sharp::BatchTable bt;
    bt.scans = table;
    bt.base = g.d_base;
    bt.nscans = (int)g.scans.size();
    bt.total = g.total;
    bt.counter = counter;
    bt.err = err;
    bt.stagger_ns = sh.stagger;
    if (g.m == 256) return sharp::launch_split256_batch(flags, bt, sh.grid, g.slab, s, sh.ch);
    return sharp::launch_raar_batch(g.m, sh.ch, flags, bt, sh.grid, s);
}

void drop_schedules(sharp_batch b) {
    for (auto& kv : b->schedules) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto* t : kv.second.tables) cudaFree(t);
    }
    b->schedules.clear();
}

}  // namespace

extern "C" {

int sharp_batch_create(sharp_batch* out, int nscans, const sharp_plan* plans) {
    if (!out || !plans || nscans < 1) return bfail(SHARP_ERR_INVALID_ARG, "batch needs at least one plan");
    *out = nullptr;
    const sharp_params& p0 = plans[0] ? plans[0]->p.prm : sharp_params{};
    for (int i = 0; i < nscans; ++i) {
        if (!plans[i]) return bfail(SHARP_ERR_INVALID_ARG, "NULL plan in batch");
        const sharp_params& pi = plans[i]->p.prm;
        if (pi.probe_every != p0.probe_every || pi.residual_every != p0.residual_every)
            return bfail(SHARP_ERR_INVALID_ARG, "plans of a batch must share probe_every and residual_every");
        if (pi.precision != SHARP_PREC_FP32)
            return bfail(SHARP_ERR_INVALID_ARG, "batched scans run in SHARP_PREC_FP32 only");
        if (plans[i]->p.deterministic)
            return bfail(SHARP_ERR_INVALID_ARG, "batched scans scatter their overlap sums (no deterministic mode)");
    }
    sharp_batch b = new sharp_batch_s;
    b->plans.assign(plans, plans + nscans);
    b->binds.resize(nscans);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int m : {64, 128, 256}) {
        Group g;
        g.m = m;
        for (int i = 0; i < nscans; ++i)
            if (plans[i]->p.m == m) g.scans.push_back(i);
        if (g.scans.empty()) continue;
        std::vector<int> base(1, 0);
        for (int i : g.scans) base.push_back(base.back() + plans[i]->p.K);
        g.total = base.back();
        cudaError_t e = cudaMalloc(&g.d_base, base.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(g.d_base, base.data(), base.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            if (m == 256) {
                g.max_grid = sms;   // one block (and one slab) per SM
                e = cudaMalloc(&g.slab, (size_t)sms * m * m * sizeof(float2));
            } else {
                e = (m == 64) ? sharp::raar_batch_max_grid<64>(&g.max_grid)
                              : sharp::raar_batch_max_grid<128>(&g.max_grid);
            }
        }
        if (e != cudaSuccess) {
            b->groups.push_back(g);   // freed by destroy
            sharp_batch_destroy(b);
            return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
        }
        g.best.grid = std::min(sms, g.max_grid);
        g.best.ch = m == 256 ? 4 : 8;
        {
            std::lock_guard<std::mutex> lk(g_tuned_mutex);
            auto it = g_tuned.find({m, size_class(g.total)});
            if (it != g_tuned.end() && it->second.grid <= g.max_grid) {
                g.best = it->second;
                g.tuned = true;
            }
        }
        if (!g.tuned) next_stage(g, sms);
        b->groups.push_back(g);
    }
    cudaError_t e = cudaMalloc(&b->counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e != cudaSuccess) {
        sharp_batch_destroy(b);
        return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = b;
    return SHARP_OK;
}

int sharp_batch_bind(sharp_batch b, int scan, float2* state_c, float2* psi_y, float2* psi, float2* probe,
                     const float* amp, double* metrics) {
    if (!b || scan < 0 || scan >= (int)b->plans.size()) return bfail(SHARP_ERR_INVALID_ARG, "bad batch or scan index");
    if (!state_c || !psi_y || !psi || !amp) return bfail(SHARP_ERR_INVALID_ARG, "state, object and amplitudes needed");
    Bind& d = b->binds[scan];
    d.c = state_c;
    d.psiy = psi_y;
    d.psi = psi;
    d.probe = probe;
    d.amp = amp;
    d.metrics = metrics;
    // the argument tables and graphs hold the old addresses
    cudaDeviceSynchronize();
    drop_schedules(b);
    return SHARP_OK;
}

int sharp_batch_step(sharp_batch b, int iter, cudaStream_t stream) {
    if (!b) return bfail(SHARP_ERR_INVALID_ARG, "batch is NULL");
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; ++i)
        if (!b->binds[i].c) return bfail(SHARP_ERR_STATE, "scan " + std::to_string(i) + " not bound");
    // 1. host schedule and frame-pass arguments of every scan (no GPU work)
    std::vector<sharp::FrameArgs> args(n);
    std::vector<sharp::StepInfo> info(n);
    uint64_t sig = 1469598103934665603ull;
    for (int i = 0; i < n; ++i) {
        sharp::Plan& p = b->plans[i]->p;
        const int fd = p.form_differs ? 1 : 0;
        if (int r = sharp::raar_step_prepare(p, b->binds[i].c, b->binds[i].psiy, b->binds[i].psi, b->binds[i].amp,
                                             iter, &args[i], &info[i]))
            return r;
        const sharp::StepInfo& in = info[i];
        const uint64_t word = (uint64_t)(in.flags | in.have_q << 2 | in.have_d << 3 | in.delta_is_norm << 4 |
                                         in.read_e << 5 | in.write_e << 6 | in.probe_due << 7 | fd << 8 |
                                         p.probe_cons_kind << 9 | p.probe_com << 11);
        sig = (sig ^ word) * 1099511628211ull;
    }
    std::vector<int> gflags(b->groups.size(), 0);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group& g = b->groups[gi];
        gflags[gi] = info[g.scans[0]].flags;
        for (int i : g.scans)
            if (info[i].flags != gflags[gi]) return bfail(SHARP_ERR_STATE, "scans of a batch reached different schedules");
    }
    bool tuning = false;
    for (auto& g : b->groups) tuning |= !g.tuned;
    const bool use_graph = b->use_graphs && !tuning;
    // 2. device argument tables of this schedule (made once, outside any capture)
    Schedule& sch = b->schedules[sig];
    if (sch.tables.empty()) {
        sch.tables.assign(b->groups.size(), nullptr);
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            std::vector<sharp::FrameArgs> tab;
            for (int i : b->groups[gi].scans) tab.push_back(args[i]);
            cudaError_t e = cudaMalloc(&sch.tables[gi], tab.size() * sizeof(sharp::FrameArgs));
            if (e == cudaSuccess)
                e = cudaMemcpy(sch.tables[gi], tab.data(), tab.size() * sizeof(sharp::FrameArgs),
                               cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                for (auto* t : sch.tables) cudaFree(t);
                b->schedules.erase(sig);
                return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
            }
        }
    }
    int rc = SHARP_OK;
    if (use_graph && sch.exec) {
        // 3a. the recorded launches, then the bookkeeping of every scan
        cudaError_t e = cudaGraphLaunch(sch.exec, stream);
        if (e != cudaSuccess) return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
        for (int i = 0; i < n && rc == SHARP_OK; ++i)
            rc = sharp::raar_step_finish(b->plans[i]->p, b->binds[i].c, b->binds[i].psiy, b->binds[i].psi,
                                         b->binds[i].probe, b->binds[i].metrics, iter, info[i], stream, false, 1);
        return rc;
    }
    // 3b. issue the step: into a recording (first use of this schedule) or
    // directly (graphs off, or the autotuner still timing grids)
    cudaStream_t s = use_graph ? b->cap : stream;
    if (use_graph) {
        // recorded on a private stream; the graph is launched on the caller's
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    }
    for (int i = 0; i < n && rc == SHARP_OK; ++i) {
        cudaError_t e = sharp::raar_step_clear(b->plans[i]->p, s);
        if (e != cudaSuccess) rc = bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (size_t gi = 0; gi < b->groups.size() && rc == SHARP_OK; ++gi) {
        Group& g = b->groups[gi];
        const bool timing = !use_graph && !g.tuned;
        int cand = -1;
        if (timing)
            for (size_t k = 0; k < g.cand_ms.size(); ++k)
                if (g.cand_ms[k] < 0.f) { cand = (int)k; break; }
        const Shape sh = cand >= 0 ? g.cand[cand] : g.best;
        cudaError_t e = cudaSuccess;
        if (cand >= 0) e = cudaEventRecord(b->ev0, s);
        if (e == cudaSuccess) e = launch_group(g, sch.tables[gi], gflags[gi], sh, b->counter, b->err, s);
        if (e == cudaSuccess && cand >= 0) e = cudaEventRecord(b->ev1, s);
        if (e == cudaSuccess && cand >= 0) e = cudaEventSynchronize(b->ev1);
        if (e == cudaSuccess && cand >= 0) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, b->ev0, b->ev1);
            tuner_record(g, cand, ms, sms);
        }
        if (e != cudaSuccess) rc = bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    }
    for (int i = 0; i < n && rc == SHARP_OK; ++i)
        rc = sharp::raar_step_finish(b->plans[i]->p, b->binds[i].c, b->binds[i].psiy, b->binds[i].psi,
                                     b->binds[i].probe, b->binds[i].metrics, iter, info[i], s, false, 0);
    if (!use_graph) return rc;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc == SHARP_OK && e != cudaSuccess) rc = bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    if (rc == SHARP_OK) {
        e = cudaGraphInstantiate(&sch.exec, graph, 0);
        if (e != cudaSuccess) {
            sch.exec = nullptr;
            rc = bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != SHARP_OK) return rc;
    e = cudaGraphLaunch(sch.exec, stream);
    if (e != cudaSuccess) rc = bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    return rc;
}

int sharp_batch_status(sharp_batch b, cudaStream_t stream) {
    if (!b) return bfail(SHARP_ERR_INVALID_ARG, "batch is NULL");
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return bfail(SHARP_ERR_CUDA, cudaGetErrorString(e));
    if (flag != 0) {
        cudaMemsetAsync(b->err, 0, sizeof(int), stream);
        if (flag == SHARP_ERR_INVALID_ARG)
            return bfail(flag, "a measured amplitude of a scan is not finite and non-negative");
        return bfail(flag, "a bounded device-side wait gave up (the step's results are invalid)");
    }
    return SHARP_OK;
}

int sharp_batch_set_graphs(sharp_batch b, int enable) {
    if (!b) return bfail(SHARP_ERR_INVALID_ARG, "batch is NULL");
    b->use_graphs = enable ? 1 : 0;
    return SHARP_OK;
}

int sharp_batch_tuned_grid(sharp_batch b, int m) {
    if (!b) return -1;
    for (auto& g : b->groups)
        if (g.m == m) return g.tuned ? g.best.grid : -1;
    return -1;
}

int sharp_batch_tuned_shape(sharp_batch b, int m, int* grid, int* rows, int* stagger_ns) {
    if (!b) return bfail(SHARP_ERR_INVALID_ARG, "batch is NULL");
    for (auto& g : b->groups) {
        if (g.m != m) continue;
        if (!g.tuned) return bfail(SHARP_ERR_STATE, "the tuner has not finished for this frame size");
        if (grid) *grid = g.best.grid;
        if (rows) *rows = g.best.ch;
        if (stagger_ns) *stagger_ns = g.best.stagger;
        return SHARP_OK;
    }
    return bfail(SHARP_ERR_INVALID_ARG, "no scan of the batch has frames of size " + std::to_string(m));
}

int sharp_batch_set_shape(sharp_batch b, int m, int grid, int rows, int stagger_ns) {
    if (!b) return bfail(SHARP_ERR_INVALID_ARG, "batch is NULL");
    for (auto& g : b->groups) {
        if (g.m != m) continue;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const bool rows_ok = m == 256 ? (rows == 2 || rows == 4) : (rows == 4 || rows == 8 || rows == 16);
        if (grid < 1 || grid > g.max_grid || !rows_ok || stagger_ns < 0 || stagger_ns > 100000)
            return bfail(SHARP_ERR_INVALID_ARG, "launch shape outside the tuner's candidates");
        cudaDeviceSynchronize();
        drop_schedules(b);   // recorded graphs hold the old launches
        g.best.grid = grid;
        g.best.ch = rows;
        g.best.stagger = stagger_ns;
        g.tuned = true;
        g.stage = 3;
        g.cand.clear();
        g.cand_ms.clear();
        return SHARP_OK;
    }
    return bfail(SHARP_ERR_INVALID_ARG, "no scan of the batch has frames of size " + std::to_string(m));
}

int sharp_batch_destroy(sharp_batch b) {
    if (!b) return SHARP_OK;
    cudaDeviceSynchronize();
    drop_schedules(b);
    for (auto& g : b->groups) {
        if (g.d_base) cudaFree(g.d_base);
        if (g.slab) cudaFree(g.slab);
    }
    if (b->counter) cudaFree(b->counter);
    if (b->err) cudaFree(b->err);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
    return SHARP_OK;
}

}  // extern "C"
