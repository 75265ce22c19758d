// hd_api.cu -- the C ABI declared in include/hd.h: context creation
// (geometry of Sec. II.A/B, initial lattice, cell binning), sweep sequencing,
// measurements and read-back.  Host code only; all per-disk work runs in the
// kernels of hd_sweep.cu and hd_measure.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hd.h"
#include "hd_kernels.h"
#include "hd_analysis.h"
#include "hd_bin.h"
#include "hd_bounds.h"

using hd::CellBufs;
using hd::Frame;
using hd::Rep;

namespace {

// An NVTX range around a public call, so that a profiler (ncu --nvtx, nsys)
// can select or label the library's phases; a no-op without a profiler.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

constexpr double kPi = 3.14159265358979323846;
constexpr double kFx = 16777216.0;  // 2^24 fixed-point units per sigma
constexpr int kMaxBins = 512;
constexpr size_t kCellPad = 64;  // elements of padding after every per-generation cell array
constexpr int kMaxStrips = 64;    // strips of a one-replica graph wavefront
constexpr int kAutoStrips = 16;   // strips chosen when the colour pass is 1.5 to 3.5 waves deep
constexpr int kAutoStripsDeep = 8;  // ... and when it is deeper
constexpr int kMaxBranches = 64;  // replicas on concurrent branches of a captured step

struct Plan {
    Rep rep;
    int cap;
    int64_t nlat;   // lattice columns
    double eta_req;
};

}  // namespace

struct hd_ctx {
    int R = 0;
    bool fixed = false;
    int cap = 4;
    int K = 50;
    int lattice = 0;
    int threads = 128;
    int tpc = 1;            // threads per active cell of the split colour pass
    bool fused = false;
    bool pass_tma = false;  // colour pass with bulk-copy (TMA) staging
    bool persist = false;   // many sweeps per launch (wavefront over bands)
    int bands = 0;          // bands of two cell rows over all replicas
    uint32_t* persist_sync = nullptr;  // ticket, abort word and per-band progress of the persistent sweep
    int persist_blocks = 0;            // its grid: the blocks resident at once
    bool persist_stall = false;        // test hook (HD_TEST_PERSIST_STALL=1 at creation)
    // analysis scratch, grown on demand and freed with the context
    double2* acf = nullptr;     // [R][max_lag + 1]
    size_t acf_cap = 0;
    double* tau = nullptr;      // [R]
    double* field_acc = nullptr;  // [R][bins^2][3]
    double2* field = nullptr;     // [R][bins^2]
    size_t field_cap = 0;
    int2* sq_hk = nullptr;          // [R][nq] wave vectors
    double2* sq_part = nullptr;     // [R][disk blocks][nq] partial amplitudes
    double* sq_S = nullptr;         // [R][nq]
    int* sq_best = nullptr;         // [R]
    size_t sq_cap = 0, sq_S_cap = 0, sq_part_cap = 0;  // capacities of sq_hk, sq_S, sq_part
    double2* chi = nullptr;         // [Ntot] positional order by disk id
    double* corr_acc = nullptr;     // [R][nr][3]
    double2* corr = nullptr;        // [R][nr]
    size_t corr_cap = 0;
    int tile = 48;
    double sigma = 1.0;
    std::vector<Rep> reps;
    std::vector<int64_t> nlat;
    int64_t Ntot = 0, Ctot = 0;
    int blocks_cell = 0, blocks_act = 0, blocks_tile = 0, blocks_t32 = 0, blocks_seg = 0;
    Rep* reps_d = nullptr;
    CellBufs buf[2] = {};
    int cur = 0;
    Frame* table = nullptr;
    Frame* frame = nullptr;
    uint64_t* sweep_ctr = nullptr;
    unsigned long long* counters = nullptr;
    int* err = nullptr;
    unsigned long long* hist = nullptr;
    double* edges = nullptr;
    long long* edgesF = nullptr;
    double* fit = nullptr;
    double* fit_qr = nullptr;  // Householder factor of the fit's design matrix
    double2* psi_local = nullptr;
    hd::ExactPair* psi_part = nullptr;  // [blocks_t32] exact block sums of psi_j
    double* psi_res = nullptr;
    double* xy = nullptr;
    uint16_t* rep_of_act = nullptr;   // replica of each active-cell-grid block
    uint16_t* rep_of_cell = nullptr;  // replica of each whole-cell-grid block
    cudaStream_t stream = nullptr;
    hd_status sticky = HD_OK;
    std::vector<int64_t> sweeps;
    std::vector<void*> allocs;
    // instrumentation: launch tallies always, event timing when enabled
    int64_t launches[HD_KERNEL_CLASSES] = {};
    double kernel_ms[HD_KERNEL_CLASSES] = {};
    bool profiling = false;
    std::vector<cudaEvent_t> ev;    // pool, used in start/stop pairs
    std::vector<int> ev_class;      // class of each pending pair
    size_t ev_used = 0;
    // graph-captured steps (hd_run): one executable graph per (sweeps per step,
    // measure, starting buffer parity), with its kernel tallies
    // A graph captured while profiling holds an event-record node before and
    // after every kernel node (events gev[ev0 + 2i], gev[ev0 + 2i + 1] around
    // its i-th kernel, of class ev_cls[i]), so that each replay times every
    // kernel inside the graph, free of host launch gaps.
    struct StepGraph {
        int sweeps;
        bool measure;
        int parity;
        bool local;     // the measurement keeps the psi_6 field
        bool profiled;
        cudaGraphExec_t exec;
        int64_t launches[HD_KERNEL_CLASSES];
        size_t ev0;
        std::vector<int> ev_cls;
    };
    std::vector<StepGraph> graphs;
    std::vector<cudaEvent_t> gev;         // event pool of profiled graphs
    size_t gev_used = 0;
    StepGraph* prof_capture = nullptr;    // the profiled graph being captured
    cudaStream_t capture_stream = nullptr;
    // Captured steps run their sweeps on concurrent graph branches: K strips of
    // bands of a one-replica context (strips > 1), or one branch per replica
    // (branches).  side: their streams; side_ev: the fork event, one join
    // event per branch, then the strips' phase events (two sets by parity).
    int strips = 1;
    bool branches = false;
    // host-pinned scratch: a count and the device error word, read back
    // together with one synchronisation
    int64_t* pinned = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;
    double* series = nullptr;       // [cap][R][4]: beta P / rho, g(2 sigma+), Re Psi_6, Im Psi_6
    int64_t* series_len = nullptr;  // device counter of recorded steps
    int64_t series_cap = 0;

    hd::LaunchCfg cfg(cudaStream_t s) const {
        hd::LaunchCfg c = cfg();
        c.stream = s;
        return c;
    }

    hd::LaunchCfg cfg() const {
        hd::LaunchCfg c;
        c.reps = reps_d;
        c.rep0 = reps.data();
        c.rep_of_act = rep_of_act;
        c.rep_of_cell = rep_of_cell;
        c.R = R;
        c.cap = cap;
        c.fixed = fixed;
        c.threads = threads;
        c.tpc = tpc;
        c.persist_blocks = persist_blocks;
        c.persist_stall = persist_stall;
        c.ntc = 0;
        for (int k : {1, 2})
            if (std::all_of(reps.begin(), reps.end(), [k](const hd::Rep& r) { return r.nt == k; })) c.ntc = k;
        c.blocks_cell = blocks_cell;
        c.blocks_act = blocks_act;
        c.blocks_tile = blocks_tile;
        c.blocks_t32 = blocks_t32;
        c.blocks_seg = blocks_seg;
        c.stream = stream;
        return c;
    }
};

namespace {

hd_status fail_cuda(hd_ctx* ctx) {
    ctx->sticky = HD_ERR_CUDA;
    return HD_ERR_CUDA;
}

#define HD_CK(ctx, call)                                   \
    do {                                                   \
        if ((call) != cudaSuccess) return fail_cuda(ctx);  \
    } while (0)

template <class T>
bool dev_alloc(hd_ctx* ctx, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    ctx->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

// Float pre-test bounds of the FP64 form (hd_bounds.h): the cell side in
// float and floats bracketing (2 sigma)^2 = 4 by the pair margin.
void set_f32_bounds(Rep& r) {
    const double M = hd::pair_f32_margin(r.w, r.delta);
    r.wf = float(r.w);
    r.d2_lo = std::nextafter(float(4.0 - M), -HUGE_VALF);
    r.d2_hi = std::nextafter(float(4.0 + M), HUGE_VALF);
}

// The histogram's range [e0, eK) widened by the margin of pairs hist_R cells
// apart, and the psi_6 margin (candidates two cells apart).
void set_hist_f32_bounds(Rep& r, double e0, double eK) {
    const double M = hd::cells_f32_margin(r.w, r.hist_R);
    r.h_lo = std::nextafter(float(e0 - M), -HUGE_VALF);
    r.h_hi = std::nextafter(float(eK + M), HUGE_VALF);
    r.psi_m = std::nextafter(float(hd::cells_f32_margin(r.w, 2)), HUGE_VALF);
}

// Geometry of one chain (Sec. II.A, II.B).  Lengths in units of sigma.
hd_status plan_replica(int64_t N, double eta, double sigma, double delta, uint64_t seed, const hd_opts& o,
                       double cell_min, Plan& pl) {
    if (N < 2 || N > (int64_t(1) << 31) - 1 || !(eta > 0.0) || !(sigma > 0.0) || !(delta >= 0.0))
        return HD_ERR_ARG;
    const bool fixed = o.precision == HD_FIXED32;
    const double L = std::sqrt(double(N) * kPi / eta);
    if (!(cell_min >= 2.0)) return HD_ERR_ARG;
    const int m = 2 * int(std::floor(L / (2.0 * cell_min)));
    if (m < 4) return HD_ERR_ARG;
    const double w = L / double(m);
    if (!(w < 8.0)) return HD_ERR_ARG;
    int64_t n = int64_t(std::ceil(std::sqrt(double(N))));
    while (n * n < N) ++n;
    while ((n - 1) * (n - 1) >= N) --n;
    if (L / double(n) < 2.0) return HD_ERR_ARG;  // the initial lattice would overlap
    const double dhat = delta / sigma;
    if (dhat > 0.0 && dhat < 0x1p-900) return HD_ERR_ARG;  // see scale_2m53
    const int64_t W = std::llround(w * kFx);
    const int64_t D = std::llround(dhat * kFx);
    if (fixed) {
        if (W >= (int64_t(1) << 29) || 2 * D + 1 >= (int64_t(1) << 32) || D >= W) return HD_ERR_ARG;
    } else if (!(dhat < w)) {
        return HD_ERR_ARG;
    }
    const double wr = fixed ? double(W) / kFx : w;
    const int kk = int(std::floor(wr / std::sqrt(2.0))) + 1;  // sub-squares of side < sqrt(2) sigma
    pl.cap = kk * kk;
    if (pl.cap > 9) return HD_ERR_ARG;
    Rep& r = pl.rep;
    std::memset(&r, 0, sizeof(Rep));
    r.N = N;
    r.m = m;
    r.hm = m / 2;
    {   // invariant divisor hm (>= 2): see div_by
        int l = 0;
        while ((int64_t(1) << l) < r.hm) ++l;
        r.hm_mul = uint32_t((((uint64_t(1) << l) - uint64_t(r.hm)) << 32) / uint64_t(r.hm) + 1u);
        r.hm_sh = l - 1;
    }
    const int64_t ncell = int64_t(m) * m;
    r.nt = o.trials_per_cell > 0 ? o.trials_per_cell : int((N + ncell - 1) / ncell);
    r.W = int32_t(W);
    r.D = int32_t(D);
    r.LF = int64_t(m) * W;
    r.w = w;
    r.w_below = std::nextafter(w, 0.0);
    r.L = L;
    r.Lm = fixed ? double(r.LF) / kFx : L;
    r.delta = dhat;
    r.sigma = sigma;
    r.key0 = uint32_t(seed & 0xffffffffu);
    r.key1 = uint32_t(seed >> 32);
    set_f32_bounds(r);
    pl.nlat = n;
    pl.eta_req = eta;
    return HD_OK;
}

// FP64 cell binning of a global coordinate t in [0, L).
void bin_fp64(double t, const Rep& r, int& c, double& u) {
    int cc = int(t / r.w);
    if (cc > r.m - 1) cc = r.m - 1;
    if (cc < 0) cc = 0;
    double uu = t - double(cc) * r.w;
    if (uu < 0.0 && cc > 0) {
        cc -= 1;
        uu = t - double(cc) * r.w;
    }
    if (uu >= r.w && cc < r.m - 1) {
        cc += 1;
        uu = t - double(cc) * r.w;
    }
    if (uu < 0.0) uu = 0.0;
    if (uu >= r.w) uu = r.w_below;
    c = cc;
    u = uu;
}

// Host image of one cell-list generation.
struct HostCells {
    std::vector<uint8_t> cnt;
    std::vector<double> pos64;   // 2 per slot
    std::vector<int32_t> posfx;  // 2 per slot
    std::vector<int32_t> pid;
};

// Insert disk `id` of replica r with global coordinates (sigma units, or exact
// fixed-point integers) into the unshifted cell frame.
bool bin_disk(const hd_ctx* ctx, const Rep& rep, HostCells& h, int64_t id, double x, double y, int64_t X,
              int64_t Y) {
    int cx, cy;
    double ux = 0.0, uy = 0.0;
    int32_t fx = 0, fy = 0;
    if (ctx->fixed) {
        cx = int(X / rep.W);
        cy = int(Y / rep.W);
        fx = int32_t(X % rep.W);
        fy = int32_t(Y % rep.W);
    } else {
        bin_fp64(x, rep, cx, ux);
        bin_fp64(y, rep, cy, uy);
    }
    const int64_t cell = hd::cell_index(rep, cx, cy);
    const int k = h.cnt[cell];
    if (k >= ctx->cap) return false;
    const int64_t slot = int64_t(k) * ctx->Ctot + cell;
    if (ctx->fixed) {
        h.posfx[2 * slot] = fx;
        h.posfx[2 * slot + 1] = fy;
    } else {
        h.pos64[2 * slot] = ux;
        h.pos64[2 * slot + 1] = uy;
    }
    h.pid[slot] = int32_t(id);
    h.cnt[cell] = uint8_t(k + 1);
    return true;
}

void host_cells_init(const hd_ctx* ctx, HostCells& h) {
    h.cnt.assign(size_t(ctx->Ctot), 0);
    h.pid.assign(size_t(ctx->Ctot) * ctx->cap, 0);
    if (ctx->fixed) h.posfx.assign(size_t(ctx->Ctot) * ctx->cap * 2, 0);
    else h.pos64.assign(size_t(ctx->Ctot) * ctx->cap * 2, 0.0);
}

hd_status upload_cells(hd_ctx* ctx, const HostCells& h) {
    const size_t slots = size_t(ctx->Ctot) * ctx->cap;
    CellBufs& b = ctx->buf[ctx->cur];
    HD_CK(ctx, cudaMemcpyAsync(b.cnt, h.cnt.data(), h.cnt.size(), cudaMemcpyHostToDevice, ctx->stream));
    HD_CK(ctx, cudaMemcpyAsync(b.pid, h.pid.data(), slots * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->fixed)
        HD_CK(ctx, cudaMemcpyAsync(b.pos, h.posfx.data(), slots * 2 * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   ctx->stream));
    else
        HD_CK(ctx, cudaMemcpyAsync(b.pos, h.pos64.data(), slots * 2 * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
    std::vector<Frame> zero(size_t(ctx->R));
    std::memset(zero.data(), 0, zero.size() * sizeof(Frame));
    HD_CK(ctx, cudaMemcpyAsync(ctx->frame, zero.data(), zero.size() * sizeof(Frame), cudaMemcpyHostToDevice,
                               ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

// Read the device error flag after a synchronisation.  Overflow is sticky
// (disks were dropped); a measurement reach failure is reported once.
// The status a value of the device error word stands for (the sticky ones
// made sticky; a reach error cleared on the device).
hd_status flags_status(hd_ctx* ctx, int flag) {
    if (flag & 1) {
        ctx->sticky = HD_ERR_OVERFLOW;
        return HD_ERR_OVERFLOW;
    }
    if (flag & (8 | 16)) {  // a bulk-copy staging or a persistent sweep's dependency wait gave up
        ctx->sticky = HD_ERR_TIMEOUT;
        return HD_ERR_TIMEOUT;
    }
    if (flag & 2) {
        HD_CK(ctx, cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
        HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
        return HD_ERR_REACH;
    }
    return HD_OK;
}

// Wait for the context's stream and report its device error word.
hd_status check_flags(hd_ctx* ctx) {
    int flag = 0;
    HD_CK(ctx, cudaMemcpyAsync(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return flags_status(ctx, flag);
}

void drop_graphs(hd_ctx* ctx) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    ctx->gev_used = 0;
}

void free_ctx(hd_ctx* ctx) {
    if (!ctx) return;
    drop_graphs(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (cudaStream_t b : ctx->side) cudaStreamDestroy(b);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (cudaEvent_t e : ctx->side_ev) cudaEventDestroy(e);
    if (ctx->series) cudaFree(ctx->series);
    if (ctx->acf) cudaFree(ctx->acf);
    if (ctx->tau) cudaFree(ctx->tau);
    if (ctx->field_acc) cudaFree(ctx->field_acc);
    if (ctx->field) cudaFree(ctx->field);
    for (void* q : {(void*)ctx->sq_hk, (void*)ctx->sq_part, (void*)ctx->sq_S, (void*)ctx->sq_best, (void*)ctx->chi,
                    (void*)ctx->corr_acc, (void*)ctx->corr})
        if (q) cudaFree(q);
    if (ctx->series_len) cudaFree(ctx->series_len);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->gev) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFree(p);
    delete ctx;
}

// Fold the pending event pairs into the per-class totals.
bool prof_flush(hd_ctx* ctx) {
    if (ctx->ev_used == 0) return true;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return false;
    for (size_t i = 0; i < ctx->ev_used / 2; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]) != cudaSuccess) return false;
        ctx->kernel_ms[ctx->ev_class[i]] += double(ms);
    }
    ctx->ev_used = 0;
    ctx->ev_class.clear();
    return true;
}

// Enqueue one kernel launch of class `cls`, bracketed by events when
// profiling (never while a graph is being captured).
template <class F>
cudaError_t launch(hd_ctx* ctx, int cls, F&& f, bool capturing = false) {
    ctx->launches[cls] += 1;
    if (capturing && ctx->prof_capture) {  // event nodes around the kernel node
        hd_ctx::StepGraph& g = *ctx->prof_capture;
        const size_t i = g.ev0 + 2 * g.ev_cls.size();
        if (i + 2 > ctx->gev.size()) return cudaErrorInvalidValue;  // pool sized before the capture
        cudaError_t e = cudaEventRecordWithFlags(ctx->gev[i], ctx->capture_stream, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
        e = f();
        if (e != cudaSuccess) return e;
        e = cudaEventRecordWithFlags(ctx->gev[i + 1], ctx->capture_stream, cudaEventRecordExternal);
        g.ev_cls.push_back(cls);
        return e;
    }
    if (!ctx->profiling || capturing) return f();
    if (ctx->ev_used + 2 > ctx->ev.size() && !prof_flush(ctx)) return cudaErrorUnknown;
    cudaError_t e = cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream);
    if (e != cudaSuccess) return e;
    e = f();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream);
    ctx->ev_class.push_back(cls);
    ctx->ev_used += 2;
    return e;
}

// Streams and events of the concurrent branches of captured steps: n
// branches, and (strips) two sets of n phase events.
cudaError_t ensure_side(hd_ctx* ctx, int n, bool phases) {
    while (ctx->side.size() < size_t(n)) {
        cudaStream_t b = nullptr;
        const cudaError_t e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        ctx->side.push_back(b);
    }
    const size_t need = size_t(1 + n) + (phases ? size_t(2 * n) : 0);
    while (ctx->side_ev.size() < need) {
        cudaEvent_t ev = nullptr;
        const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        ctx->side_ev.push_back(ev);
    }
    return cudaSuccess;
}

// Fork the first n side streams from s (captured: each takes s's current
// dependencies), and join them back into s.
cudaError_t fork_side(hd_ctx* ctx, cudaStream_t s, int n) {
    cudaError_t e = cudaEventRecord(ctx->side_ev[0], s);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ctx->side[size_t(i)], ctx->side_ev[0], 0);
    return e;
}
cudaError_t join_side(hd_ctx* ctx, cudaStream_t s, int n) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ctx->side_ev[1 + size_t(i)], ctx->side[size_t(i)]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->side_ev[1 + size_t(i)], 0);
    }
    return e;
}

// One replica's nc sweeps as K strips (see enqueue_strips) on side streams
// off .. off + K - 1, forked and joined by the caller; c0 is the replica's
// one-replica launch configuration, tab and counters its draw table and trial
// counters.  The phase events of side stream x are side_ev[ev_phase + x] and
// side_ev[ev_phase + S + x] (by phase parity), S the side streams in use.
cudaError_t enqueue_strip_chain(hd_ctx* ctx, const hd::LaunchCfg& c0, const Rep& rep, const hd::Frame* tab,
                                unsigned long long* counters, int nc, int cur0, int off, int K, size_t ev_phase,
                                int S) {
    std::vector<uint32_t> b(size_t(K) + 1);
    for (int i = 0; i <= K; ++i) b[size_t(i)] = uint32_t((int64_t(rep.hm) * i) / K);
    cudaError_t e = cudaSuccess;
    int cur = cur0;
    int k = 0;  // phase index over the chunk
    for (int j = 1; j <= nc && e == cudaSuccess; ++j) {
        for (int ph = 0; ph < 5 && e == cudaSuccess; ++ph, ++k) {
            const size_t now = ev_phase + size_t(k & 1) * size_t(S) + size_t(off);
            const size_t prev = ev_phase + size_t((k & 1) ^ 1) * size_t(S) + size_t(off);
            for (int i = 0; i < K && e == cudaSuccess; ++i) {
                cudaStream_t bs = ctx->side[size_t(off + i)];
                if (k > 0) {  // the previous phase in the two neighbouring strips (its own: stream order)
                    const int l = (i + K - 1) % K, r = (i + 1) % K;
                    if (l != i) e = cudaStreamWaitEvent(bs, ctx->side_ev[prev + size_t(l)], 0);
                    if (e == cudaSuccess && r != i && r != l) e = cudaStreamWaitEvent(bs, ctx->side_ev[prev + size_t(r)], 0);
                    if (e != cudaSuccess) break;
                }
                hd::LaunchCfg c = c0;
                c.stream = bs;
                const uint32_t lo = b[size_t(i)] * uint32_t(rep.hm), hi = b[size_t(i) + 1] * uint32_t(rep.hm);
                if (ph == 0) {
                    c.band_lo = lo;
                    c.band_span = hi - lo;
                    e = launch(ctx, HD_K_REBUILD, [&] {
                        return hd::launch_rebuild(c, tab, j, ctx->buf[cur], ctx->buf[cur ^ 1], ctx->err);
                    }, true);
                } else {
                    c.act_lo = lo;
                    c.act_hi = hi;
                    e = launch(ctx, HD_K_PASS, [&] {
                        return hd::launch_pass(c, tab, j, ph - 1, ctx->buf[cur], counters);
                    }, true);
                }
                if (e == cudaSuccess) e = cudaEventRecord(ctx->side_ev[now + size_t(i)], bs);
            }
            if (ph == 0) cur ^= 1;
        }
    }
    return e;
}

// The one-replica launch configuration of replica r of a batch (its blocks
// numbered from 0, its constants as kernel parameters); rep receives the
// replica's constants and must outlive the launches.
hd::LaunchCfg replica_cfg(hd_ctx* ctx, int r, Rep& rep) {
    rep = ctx->reps[size_t(r)];
    rep.blk_act = 0;
    rep.blk_cell = 0;
    hd::LaunchCfg c = ctx->cfg();
    c.R = 1;
    c.rep0 = &rep;
    c.reps = ctx->reps_d + r;
    c.ntc = (rep.nt == 1 || rep.nt == 2) ? rep.nt : 0;
    c.blocks_act = int((int64_t(rep.hh) + c.threads - 1) / c.threads);
    c.blocks_cell = int((int64_t(rep.m) * rep.m + c.threads - 1) / c.threads);
    return c;
}

// Replica branches: the nc sweeps of one draw table, each replica on its own
// stream with its own one-replica launches (constants as kernel parameters),
// the replicas' chains running concurrently.  Same chain as the batched
// launches: the replicas are independent.
// (Strips inside the branches measured slower: the replicas' concurrency
// already fills the GPU, and the extra graph nodes only cost launches.)
cudaError_t enqueue_replica_branches(hd_ctx* ctx, cudaStream_t s, int nc) {
    cudaError_t e = fork_side(ctx, s, ctx->R);
    const int cur0 = ctx->cur;
    for (int r = 0; r < ctx->R && e == cudaSuccess; ++r) {
        Rep rep;
        hd::LaunchCfg c = replica_cfg(ctx, r, rep);
        const hd::Frame* tab = ctx->table + size_t(r) * (hd::kMaxChunk + 1);
        unsigned long long* counters = ctx->counters + 2 * size_t(r);
        c.stream = ctx->side[size_t(r)];
        int cur = cur0;
        for (int j = 1; j <= nc && e == cudaSuccess; ++j) {
            e = launch(ctx, HD_K_REBUILD, [&] {
                return hd::launch_rebuild(c, tab, j, ctx->buf[cur], ctx->buf[cur ^ 1], ctx->err);
            }, true);
            cur ^= 1;
            for (int p = 0; p < 4 && e == cudaSuccess; ++p)
                e = launch(ctx, HD_K_PASS, [&] { return hd::launch_pass(c, tab, j, p, ctx->buf[cur], counters); }, true);
        }
    }
    if (e == cudaSuccess) e = join_side(ctx, s, ctx->R);
    if (nc & 1) ctx->cur ^= 1;
    return e;
}

// Graph wavefront of one replica: the nc sweeps of one draw table as K strips
// of bands (two cell rows each), one stream per strip.  An item of band b
// reads and writes only cell rows 2b - 1 .. 2b + 2 (a pass reads its cells'
// eight neighbours, a rebuild moves a disk by at most one cell), so a
// strip's phase (the rebuild or one colour pass) may start once the previous
// phase is done in that strip and the two next to it: graph edges, not a
// global barrier, separate the phases, and the tail of one strip's launch
// overlaps the next phase of strips that are ready.  Every cell sees the
// same sequence of phases as in the serial order, so the chain is the same.
cudaError_t enqueue_strips(hd_ctx* ctx, cudaStream_t s, int nc) {
    const int K = ctx->strips;
    cudaError_t e = fork_side(ctx, s, K);
    if (e == cudaSuccess)
        e = enqueue_strip_chain(ctx, ctx->cfg(), ctx->reps[0], ctx->table, ctx->counters, nc, ctx->cur, 0, K,
                                size_t(1 + K), K);
    if (e == cudaSuccess) e = join_side(ctx, s, K);
    if (nc & 1) ctx->cur ^= 1;
    return e;
}

// Enqueue n sweeps on stream s (draw tables of up to kMaxChunk sweeps, then
// per sweep either one fused launch or a rebuild and four colour passes).
// While a step graph is captured (not for a profiled graph, whose event nodes
// time each kernel in order), the sweeps of a one-replica context with strips
// run as a graph wavefront, and those of a batch with replica branches as
// one branch per replica.
cudaError_t enqueue_sweeps(hd_ctx* ctx, cudaStream_t s, int64_t n, bool capturing) {
    const hd::LaunchCfg c = ctx->cfg(s);
    const bool wave = capturing && !ctx->prof_capture && (ctx->strips > 1 || ctx->branches);
    if (wave) {
        const int nb = ctx->strips > 1 ? ctx->strips : ctx->R;
        cudaError_t e = ensure_side(ctx, nb, ctx->strips > 1);
        for (int64_t left = n; left > 0 && e == cudaSuccess;) {
            const int nc = int(std::min<int64_t>(left, hd::kMaxChunk));
            e = launch(ctx, HD_K_DRAWS, [&] { return hd::launch_draws(c, ctx->table, ctx->frame, ctx->sweep_ctr, nc); },
                       capturing);
            if (e == cudaSuccess) e = ctx->strips > 1 ? enqueue_strips(ctx, s, nc) : enqueue_replica_branches(ctx, s, nc);
            left -= nc;
        }
        return e;
    }
    int64_t left = n;
    cudaError_t e = cudaSuccess;
    while (left > 0 && e == cudaSuccess) {
        const int nc = int(std::min<int64_t>(left, hd::kMaxChunk));
        e = launch(ctx, HD_K_DRAWS, [&] { return hd::launch_draws(c, ctx->table, ctx->frame, ctx->sweep_ctr, nc); },
                   capturing);
        for (int j = 1; j <= nc && e == cudaSuccess; ++j) {
            if (ctx->persist) {  // the chunk's sweeps in one launch
                e = launch(ctx, HD_K_SWEEP, [&] {
                    return hd::launch_sweeps_persist(c, ctx->table, nc, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1],
                                                     ctx->counters, ctx->err, ctx->persist_sync, ctx->bands);
                }, capturing);
                if (nc & 1) ctx->cur ^= 1;
                break;
            }
            if (ctx->fused) {
                e = launch(ctx, HD_K_SWEEP, [&] {
                    return hd::launch_sweep_fused(c, ctx->table, j, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1],
                                                  ctx->counters, ctx->err);
                }, capturing);
                ctx->cur ^= 1;
            } else {
                e = launch(ctx, HD_K_REBUILD, [&] {
                    return hd::launch_rebuild(c, ctx->table, j, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1], ctx->err);
                }, capturing);
                ctx->cur ^= 1;
                for (int p = 0; p < 4 && e == cudaSuccess; ++p)
                    e = launch(ctx, HD_K_PASS, [&] {
                        return ctx->pass_tma
                                   ? hd::launch_pass_tma(c, ctx->table, j, p, ctx->buf[ctx->cur], ctx->counters, ctx->err)
                                   : hd::launch_pass(c, ctx->table, j, p, ctx->buf[ctx->cur], ctx->counters);
                    }, capturing);
            }
        }
        left -= nc;
    }
    return e;
}

// Enqueue the contact histogram and the pressure fit on stream s.
cudaError_t enqueue_pressure(hd_ctx* ctx, cudaStream_t s, bool capturing) {
    const hd::LaunchCfg c = ctx->cfg(s);
    cudaError_t e = cudaMemsetAsync(ctx->hist, 0, sizeof(unsigned long long) * size_t(ctx->R) * ctx->K, s);
    if (e != cudaSuccess) return e;
    int halo = 0;
    for (const hd::Rep& rep : ctx->reps) halo = std::max(halo, rep.hist_R);
    const hd::HistCfg h{ctx->K, ctx->edges, ctx->edgesF, halo};
    e = launch(ctx, HD_K_HIST, [&] { return hd::launch_hist(c, h, ctx->buf[ctx->cur], ctx->hist); }, capturing);
    if (e != cudaSuccess) return e;
    return launch(ctx, HD_K_FIT, [&] { return hd::launch_fit(c, ctx->K, ctx->fit_qr, ctx->hist, ctx->fit); }, capturing);
}

// Enqueue psi_6 (local field into psi_local when `local`) and its reduction.
cudaError_t enqueue_psi6(hd_ctx* ctx, cudaStream_t s, bool local, bool capturing) {
    const hd::LaunchCfg c = ctx->cfg(s);
    cudaError_t e = launch(ctx, HD_K_PSI6, [&] {
        return hd::launch_psi6(c, ctx->buf[ctx->cur], local ? ctx->psi_local : nullptr, ctx->psi_part, ctx->err);
    }, capturing);
    if (e != cudaSuccess) return e;
    return launch(ctx, HD_K_PSI6_REDUCE, [&] { return hd::launch_psi6_reduce(c, ctx->psi_part, ctx->psi_res); },
                  capturing);
}

// One hd_run step: sweeps, then (optionally) a measurement appended to the
// device series.
cudaError_t enqueue_step(hd_ctx* ctx, cudaStream_t s, int sweeps, bool measure, bool local, bool capturing) {
    cudaError_t e = enqueue_sweeps(ctx, s, sweeps, capturing);
    if (e != cudaSuccess || !measure) return e;
    if (capturing && !ctx->prof_capture) {
        // the histogram and psi_6 only read the cells: in a step graph psi_6
        // runs on a branch of its own, beside the histogram and the fit
        // (measured: 3.95 -> 3.93 ms per step at N = 2^20)
        e = ensure_side(ctx, 1, false);
        if (e == cudaSuccess) e = fork_side(ctx, s, 1);
        if (e == cudaSuccess) e = enqueue_psi6(ctx, ctx->side[0], local, capturing);
        if (e == cudaSuccess) e = enqueue_pressure(ctx, s, capturing);
        if (e == cudaSuccess) e = join_side(ctx, s, 1);
    } else {
        e = enqueue_pressure(ctx, s, capturing);
        if (e != cudaSuccess) return e;
        e = enqueue_psi6(ctx, s, local, capturing);
    }
    if (e != cudaSuccess) return e;
    return hd::launch_record(ctx->cfg(s), ctx->fit, ctx->psi_res, ctx->series, ctx->series_len, ctx->series_cap,
                             ctx->err);
}

}  // namespace

extern "C" {

void hd_default_opts(hd_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(hd_opts));
    o->precision = HD_FP64;
    o->lattice = HD_LATTICE_SQUARE;
    o->trials_per_cell = 0;
    o->hist_bins = 50;
    o->hist_dr = 1e-3;
    o->cell_min = 2.0;
    o->block_threads = 128;
    o->sweep_kernel = HD_SWEEP_SPLIT;
    o->threads_per_cell = 1;
    o->cell_min_per_replica = nullptr;
    o->strips = 0;
    o->replica_branches = 0;
}

const char* hd_status_string(hd_status s) {
    switch (s) {
        case HD_OK: return "ok";
        case HD_ERR_ARG: return "invalid argument";
        case HD_ERR_CUDA: return "CUDA runtime error";
        case HD_ERR_OVERFLOW: return "cell capacity overflow";
        case HD_ERR_TIMEOUT: return "bounded device wait timed out";
        case HD_ERR_REACH: return "measurement stencil exceeds the box";
        case HD_ERR_STATE: return "context in sticky error state";
    }
    return "unknown status";
}

hd_status hd_batch_init(hd_ctx** out, int32_t R, const int64_t* N, const double* eta, double sigma,
                        const double* delta, const uint64_t* seed, const hd_opts* opts_in) {
    const Range range("hd_batch_init");
    if (!out) return HD_ERR_ARG;
    *out = nullptr;
    if (R < 1 || R > 65535 || !N || !eta || !delta || !seed) return HD_ERR_ARG;
    hd_opts o;
    hd_default_opts(&o);
    if (opts_in) {
        o.precision = opts_in->precision;
        o.lattice = opts_in->lattice;
        o.trials_per_cell = opts_in->trials_per_cell;
        if (opts_in->hist_bins > 0) o.hist_bins = opts_in->hist_bins;
        if (opts_in->hist_dr > 0.0) o.hist_dr = opts_in->hist_dr;
        if (opts_in->cell_min > 0.0) o.cell_min = opts_in->cell_min;
        if (opts_in->block_threads > 0) o.block_threads = opts_in->block_threads;
        o.sweep_kernel = opts_in->sweep_kernel;
        if (opts_in->threads_per_cell > 0) o.threads_per_cell = opts_in->threads_per_cell;
        o.cell_min_per_replica = opts_in->cell_min_per_replica;
        o.strips = opts_in->strips;
        o.replica_branches = opts_in->replica_branches;
    }
    if (o.precision != HD_FP64 && o.precision != HD_FIXED32) return HD_ERR_ARG;
    if (o.lattice != HD_LATTICE_SQUARE && o.lattice != HD_LATTICE_TRIANGULAR) return HD_ERR_ARG;
    if (!(o.cell_min >= 2.0) || o.hist_bins < 5 || o.hist_bins > kMaxBins || o.trials_per_cell < 0) return HD_ERR_ARG;
    if (o.block_threads < 32 || o.block_threads > 256 || (o.block_threads & 31)) return HD_ERR_ARG;
    if (o.sweep_kernel != HD_SWEEP_FUSED && o.sweep_kernel != HD_SWEEP_SPLIT && o.sweep_kernel != HD_SWEEP_TMA &&
        o.sweep_kernel != HD_SWEEP_PERSISTENT)
        return HD_ERR_ARG;
    {
        const int g = o.threads_per_cell;
        if (g != 1 && g != 2 && g != 4 && g != 8) return HD_ERR_ARG;
        if (g > 1 && (o.sweep_kernel != HD_SWEEP_SPLIT || o.block_threads * g > 512)) return HD_ERR_ARG;
    }
    // graph branches: strips only for one replica on the split one-thread pass
    const bool split1 = o.sweep_kernel == HD_SWEEP_SPLIT && o.threads_per_cell == 1;
    if (o.strips < 0 || o.strips > kMaxStrips || (o.strips >= 2 && (R != 1 || !split1))) return HD_ERR_ARG;
    if (o.replica_branches != 0 && o.replica_branches != 1) return HD_ERR_ARG;

    std::vector<Plan> plans(static_cast<size_t>(R));
    int cap = 4;
    for (int r = 0; r < R; ++r) {
        const double cm = o.cell_min_per_replica ? o.cell_min_per_replica[r] : o.cell_min;
        const hd_status s = plan_replica(N[r], eta[r], sigma, delta[r], seed[r], o, cm, plans[size_t(r)]);
        if (s != HD_OK) return s;
        cap = std::max(cap, plans[size_t(r)].cap);
    }
    cap = cap <= 4 ? 4 : 9;
    if (o.strips > plans[0].rep.hm) return HD_ERR_ARG;  // every strip at least one band

    hd_ctx* ctx = new (std::nothrow) hd_ctx();
    if (!ctx) return HD_ERR_ARG;
    ctx->R = R;
    ctx->fixed = o.precision == HD_FIXED32;
    ctx->cap = cap;
    ctx->K = o.hist_bins;
    ctx->lattice = o.lattice;
    ctx->threads = o.block_threads;
    ctx->tpc = o.threads_per_cell;
    ctx->fused = o.sweep_kernel == HD_SWEEP_FUSED;
    ctx->pass_tma = o.sweep_kernel == HD_SWEEP_TMA;
    ctx->persist = o.sweep_kernel == HD_SWEEP_PERSISTENT;
    ctx->tile = hd::fused_tile(ctx->fixed, cap);
    ctx->sigma = sigma;
    ctx->sweeps.assign(size_t(R), 0);
    const int64_t DR = std::llround(o.hist_dr * kFx);
    if (ctx->fixed && DR < 1) {
        delete ctx;
        return HD_ERR_ARG;
    }
    int64_t cell_off = 0, id_off = 0;
    int blk_cell = 0, blk_act = 0, blk_tile = 0, blk_t32 = 0, blk_seg = 0, band0 = 0;
    for (int r = 0; r < R; ++r) {
        Rep rep = plans[size_t(r)].rep;
        rep.cell_off = cell_off;
        rep.id_off = id_off;
        rep.blk_cell = blk_cell;
        rep.blk_act = blk_act;
        rep.blk_tile = blk_tile;
        rep.blk_t32 = blk_t32;
        rep.tiles_x = (rep.m + 31) / 32;
        rep.tx_mul = 0;
        rep.tx_sh = 0;
        if (rep.tiles_x > 1) {  // invariant divisor tiles_x >= 2: see div_by (tiles_x = 1 needs no division)
            int l = 0;
            while ((int64_t(1) << l) < rep.tiles_x) ++l;
            rep.tx_mul = uint32_t((((uint64_t(1) << l) - uint64_t(rep.tiles_x)) << 32) / uint64_t(rep.tiles_x) + 1u);
            rep.tx_sh = l - 1;
        }
        blk_t32 += int(int64_t(rep.tiles_x) * ((rep.m + ctx->threads / 32 - 1) / (ctx->threads / 32)));
        rep.blk_seg = blk_seg;
        rep.nseg = (rep.hm + ctx->threads - 1) / ctx->threads;
        rep.segw = (rep.hm + rep.nseg - 1) / rep.nseg;
        rep.seg_mul = 0;
        rep.seg_sh = 0;
        rep.band0 = band0;
        band0 += rep.hm;
        if (rep.nseg > 1) {  // invariant divisor nseg >= 2: see div_by
            int l = 0;
            while ((int64_t(1) << l) < rep.nseg) ++l;
            rep.seg_mul = uint32_t((((uint64_t(1) << l) - uint64_t(rep.nseg)) << 32) / uint64_t(rep.nseg) + 1u);
            rep.seg_sh = l - 1;
        }
        blk_seg += rep.hm * rep.nseg;
        const int64_t tx = (rep.m + ctx->tile - 1) / ctx->tile;
        blk_tile += int(tx * tx);
        const int64_t ncell = int64_t(rep.m) * rep.m;
        const int64_t nact = int64_t(rep.hm) * rep.hm;
        cell_off += ncell;
        id_off += rep.N;
        blk_cell += int((ncell + ctx->threads - 1) / ctx->threads);
        blk_act += int((nact + ctx->threads - 1) / ctx->threads);
        if (ctx->fixed) {
            rep.dr = double(DR) / kFx;
            rep.hist_R = int((((int64_t(1) << 25) + int64_t(ctx->K) * DR)) / rep.W) + 1;
        } else {
            rep.dr = o.hist_dr;
            rep.hist_R = int(std::floor((2.0 + double(ctx->K) * o.hist_dr) / rep.w)) + 1;
            const double xK = 2.0 + double(ctx->K) * o.hist_dr;  // as the squared bin edges below
            set_hist_f32_bounds(rep, 4.0, xK * xK);
        }
        ctx->reps.push_back(rep);
        ctx->nlat.push_back(plans[size_t(r)].nlat);
    }
    // cell arrays are padded to a multiple of 16 cells, so that every slot
    // plane starts on a 16-byte boundary (bulk copies need one)
    ctx->Ctot = (cell_off + 15) & ~int64_t(15);
    // Test hook for the bulk-copy pass's error path: with the environment
    // variable HD_TEST_UNALIGNED_SLOT_STRIDE=1 at creation, the slot planes
    // are 8 cells further apart, so every plane after the first starts off
    // the 16-cell boundary.  The cp.async kernels do not need that boundary;
    // the bulk-copy pass rejects its staging plan, issues no copy and reports
    // HD_ERR_TIMEOUT.
    if (const char* t = std::getenv("HD_TEST_UNALIGNED_SLOT_STRIDE"); t && t[0] == '1' && t[1] == '\0')
        ctx->Ctot += 8;
    ctx->Ntot = id_off;
    if (ctx->Ctot * int64_t(cap) >= (int64_t(1) << 31)) {
        delete ctx;
        return HD_ERR_ARG;  // cell and slot indices are 32-bit in the kernels
    }
    for (Rep& rep : ctx->reps) {
        rep.stride = ctx->Ctot;
        rep.coff = uint32_t(rep.cell_off);
        rep.stride32 = uint32_t(ctx->Ctot);
        rep.hh = rep.hm * rep.hm;
    }
    ctx->blocks_cell = blk_cell;
    ctx->blocks_act = blk_act;
    ctx->blocks_tile = blk_tile;
    ctx->blocks_t32 = blk_t32;
    ctx->blocks_seg = blk_seg;

    const size_t slots = size_t(ctx->Ctot) * cap;
    bool ok = dev_alloc(ctx, &ctx->reps_d, size_t(R));
    for (int b = 0; b < 2 && ok; ++b) {
        // occupancy bytes are claimed with 32-bit atomics: pad to whole words
        // occupancy bytes are claimed with 32-bit atomics and bulk copies may
        // read up to 15 bytes past a segment: pad every cell array
        ok = ok && dev_alloc(ctx, &ctx->buf[b].cnt, size_t(ctx->Ctot) + kCellPad);
        ok = ok && dev_alloc(ctx, &ctx->buf[b].pid, slots + kCellPad);
        if (ctx->fixed) {
            int2* p = nullptr;
            ok = ok && dev_alloc(ctx, &p, slots + kCellPad);
            ctx->buf[b].pos = p;
        } else {
            double2* p = nullptr;
            ok = ok && dev_alloc(ctx, &p, slots + kCellPad);
            ctx->buf[b].pos = p;
        }
    }
    ok = ok && dev_alloc(ctx, &ctx->table, size_t(R) * (hd::kMaxChunk + 1));
    ok = ok && dev_alloc(ctx, &ctx->frame, size_t(R));
    ok = ok && dev_alloc(ctx, &ctx->sweep_ctr, size_t(R));
    ok = ok && dev_alloc(ctx, &ctx->counters, size_t(2 * R));
    ok = ok && dev_alloc(ctx, &ctx->err, 1);
    ok = ok && dev_alloc(ctx, &ctx->hist, size_t(R) * ctx->K);
    ok = ok && dev_alloc(ctx, &ctx->edges, size_t(ctx->K + 1));
    ok = ok && dev_alloc(ctx, &ctx->edgesF, size_t(ctx->K + 1));
    ok = ok && dev_alloc(ctx, &ctx->fit, size_t(4 * R));
    ok = ok && dev_alloc(ctx, &ctx->fit_qr, hd::fit_factor_len(ctx->K));
    ok = ok && dev_alloc(ctx, &ctx->psi_local, size_t(ctx->Ntot));
    ok = ok && dev_alloc(ctx, &ctx->psi_part, size_t(ctx->blocks_t32));
    ok = ok && dev_alloc(ctx, &ctx->psi_res, size_t(2 * R));
    ok = ok && dev_alloc(ctx, &ctx->rep_of_act, size_t(ctx->blocks_act));
    ok = ok && dev_alloc(ctx, &ctx->rep_of_cell, size_t(ctx->blocks_cell));
    ok = ok && dev_alloc(ctx, &ctx->xy, size_t(2 * ctx->Ntot));
    ok = ok && cudaMallocHost(reinterpret_cast<void**>(&ctx->pinned), 2 * sizeof(int64_t)) == cudaSuccess;
    ctx->bands = band0;
    if (ctx->persist) {
        // Test hook for the persistent sweep's bounded waits: with the
        // environment variable HD_TEST_PERSIST_STALL=1 at creation, the first
        // item of band 0 is never published and the waits give up after 4096
        // polls, so the sweep reports HD_ERR_TIMEOUT.
        if (const char* t = std::getenv("HD_TEST_PERSIST_STALL"); t && t[0] == '1' && t[1] == '\0')
            ctx->persist_stall = true;
        ok = ok && dev_alloc(ctx, &ctx->persist_sync, hd::persist_sync_words(ctx->bands));
        ok = ok && hd::persist_grid(ctx->cfg(), &ctx->persist_blocks) == cudaSuccess && ctx->persist_blocks > 0;
    }
    // Concurrent branches of captured steps.  One replica: K strips when
    // asked, or automatically 16 when its colour pass is 1.5 to 3.5 waves of
    // resident blocks deep and 8 when it is deeper (measured on GB300 from
    // N = 2^16 to 2^24: 10-14% faster from N = 2^20 up, where launch tails
    // and phase boundaries are a large share of a sweep; shallower passes
    // lose more to the extra graph nodes than the overlap gains).  Several
    // replicas: one branch each, up to kMaxBranches.
    if (ok && R == 1 && split1) {
        if (o.strips >= 2) {
            ctx->strips = o.strips;
        } else if (o.strips == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            ok = cudaGetDevice(&dev) == cudaSuccess &&
                 cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                 hd::pass_blocks_per_sm(ctx->cfg(), &per_sm) == cudaSuccess;
            const double waves = (sms > 0 && per_sm > 0) ? double(ctx->blocks_act) / (double(sms) * per_sm) : 0.0;
            const int k = waves < 3.5 ? kAutoStrips : kAutoStripsDeep;
            if (ok && waves >= 1.5 && ctx->reps[0].hm >= 2 * k) ctx->strips = k;
        }
    }
    ctx->branches = R > 1 && R <= kMaxBranches && split1 && o.replica_branches == 0;
    // the branches' streams and events exist before any step is captured
    // (one side stream at least: the measurement's psi_6 branch)
    ok = ok && ensure_side(ctx, std::max(1, ctx->strips > 1 ? ctx->strips : (ctx->branches ? R : 1)),
                           ctx->strips > 1) == cudaSuccess;
    if (!ok) {
        free_ctx(ctx);
        return HD_ERR_CUDA;
    }
    // squared bin edges: FP64 (2 + k dr)^2, fixed (2^25 + k DR)^2
    std::vector<double> e(size_t(ctx->K + 1));
    std::vector<long long> ef(size_t(ctx->K + 1));
    for (int k = 0; k <= ctx->K; ++k) {
        const double x = 2.0 + double(k) * o.hist_dr;
        e[size_t(k)] = x * x;
        const long long xf = (1LL << 25) + (long long)k * DR;
        ef[size_t(k)] = xf * xf;
    }
    // block -> replica tables of the two cell grids (R <= 65535 replicas)
    std::vector<uint16_t> ra(size_t(ctx->blocks_act)), rc(size_t(ctx->blocks_cell));
    for (int r = 0; r < R; ++r) {
        const Rep& rep = ctx->reps[size_t(r)];
        const int ea = r + 1 < R ? ctx->reps[size_t(r + 1)].blk_act : ctx->blocks_act;
        const int ec = r + 1 < R ? ctx->reps[size_t(r + 1)].blk_cell : ctx->blocks_cell;
        for (int b = rep.blk_act; b < ea; ++b) ra[size_t(b)] = uint16_t(r);
        for (int b = rep.blk_cell; b < ec; ++b) rc[size_t(b)] = uint16_t(r);
    }
    bool cu = cudaMemcpy(ctx->reps_d, ctx->reps.data(), sizeof(Rep) * size_t(R), cudaMemcpyHostToDevice) == cudaSuccess;
    cu = cu && cudaMemcpy(ctx->edges, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    cu = cu && cudaMemcpy(ctx->rep_of_act, ra.data(), ra.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) == cudaSuccess;
    cu = cu && cudaMemcpy(ctx->rep_of_cell, rc.data(), rc.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) == cudaSuccess;
    cu = cu && cudaMemcpy(ctx->edgesF, ef.data(), ef.size() * sizeof(long long), cudaMemcpyHostToDevice) == cudaSuccess;
    cu = cu && cudaMemset(ctx->sweep_ctr, 0, sizeof(uint64_t) * size_t(R)) == cudaSuccess;
    cu = cu && cudaMemset(ctx->counters, 0, sizeof(unsigned long long) * size_t(2 * R)) == cudaSuccess;
    cu = cu && cudaMemset(ctx->err, 0, sizeof(int)) == cudaSuccess;
    cu = cu && cudaMemset(ctx->buf[0].cnt, 0, size_t(ctx->Ctot) + kCellPad) == cudaSuccess;
    cu = cu && cudaMemset(ctx->buf[1].cnt, 0, size_t(ctx->Ctot) + kCellPad) == cudaSuccess;
    cu = cu && hd::launch_fit_factor(nullptr, ctx->K, ctx->fit_qr) == cudaSuccess;
    cu = cu && cudaStreamSynchronize(nullptr) == cudaSuccess;  // before any work on the context's own stream
    if (!cu) {
        free_ctx(ctx);
        return HD_ERR_CUDA;
    }

    // initial lattice (square, or odd rows shifted by half a spacing)
    HostCells h;
    host_cells_init(ctx, h);
    for (int r = 0; r < R; ++r) {
        const Rep& rep = ctx->reps[size_t(r)];
        const int64_t n = ctx->nlat[size_t(r)];
        for (int64_t k = 0; k < rep.N; ++k) {
            const int64_t row = k / n, col = k % n;
            int64_t numx = 2 * col + 1 + ((ctx->lattice == HD_LATTICE_TRIANGULAR && (row & 1)) ? 1 : 0);
            if (numx >= 2 * n) numx -= 2 * n;
            const int64_t numy = 2 * row + 1;
            double x = 0.0, y = 0.0;
            int64_t X = 0, Y = 0;
            if (ctx->fixed) {
                X = (numx * rep.LF) / (2 * n);
                Y = (numy * rep.LF) / (2 * n);
            } else {
                x = (double(numx) * rep.L) / double(2 * n);
                y = (double(numy) * rep.L) / double(2 * n);
            }
            if (!bin_disk(ctx, rep, h, k, x, y, X, Y)) {
                free_ctx(ctx);
                return HD_ERR_OVERFLOW;
            }
        }
    }
    if (upload_cells(ctx, h) != HD_OK) {
        free_ctx(ctx);
        return HD_ERR_CUDA;
    }
    *out = ctx;
    return HD_OK;
}

hd_status hd_init(hd_ctx** out, int64_t N, double eta, double sigma, double delta, uint64_t seed,
                  const hd_opts* opts) {
    return hd_batch_init(out, 1, &N, &eta, sigma, &delta, &seed, opts);
}

hd_status hd_destroy(hd_ctx* ctx) {
    if (!ctx) return HD_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return HD_OK;
}

hd_status hd_set_stream(hd_ctx* ctx, void* stream) {
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return HD_OK;
}

hd_status hd_sweep(hd_ctx* ctx, int64_t n) {
    const Range range("hd_sweep");
    if (!ctx || n < 0) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, enqueue_sweeps(ctx, ctx->stream, n, false));
    for (auto& s : ctx->sweeps) s += n;
    return HD_OK;
}

hd_status hd_pressure(hd_ctx* ctx, double* betaP_over_rho, double* g_contact, uint64_t* hist) {
    const Range range("hd_pressure");
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    for (const Rep& r : ctx->reps)
        if (2 * r.hist_R + 1 > r.m) return HD_ERR_REACH;
    HD_CK(ctx, enqueue_pressure(ctx, ctx->stream, false));
    std::vector<double> res(size_t(4 * ctx->R));
    HD_CK(ctx, cudaMemcpyAsync(res.data(), ctx->fit, res.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (hist)
        HD_CK(ctx, cudaMemcpyAsync(hist, ctx->hist, sizeof(unsigned long long) * size_t(ctx->R) * ctx->K,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const hd_status f = check_flags(ctx);
    if (f != HD_OK) return f;
    for (int r = 0; r < ctx->R; ++r) {
        if (betaP_over_rho) betaP_over_rho[r] = res[size_t(4 * r)];
        if (g_contact) g_contact[r] = res[size_t(4 * r + 1)];
    }
    return HD_OK;
}

hd_status hd_psi6(hd_ctx* ctx, double* re, double* im, double* local) {
    const Range range("hd_psi6");
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, enqueue_psi6(ctx, ctx->stream, local != nullptr, false));
    std::vector<double> res(size_t(2 * ctx->R));
    HD_CK(ctx, cudaMemcpyAsync(res.data(), ctx->psi_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
    if (local)
        HD_CK(ctx, cudaMemcpyAsync(local, ctx->psi_local, sizeof(double2) * size_t(ctx->Ntot), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const hd_status f = check_flags(ctx);
    if (f != HD_OK) return f;
    for (int r = 0; r < ctx->R; ++r) {
        if (re) re[r] = res[size_t(2 * r)];
        if (im) im[r] = res[size_t(2 * r + 1)];
    }
    return HD_OK;
}

hd_status hd_psi6_local_device(hd_ctx* ctx, double* local_device) {
    if (!ctx || !local_device) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, cudaMemcpyAsync(local_device, ctx->psi_local, sizeof(double2) * size_t(ctx->Ntot),
                               cudaMemcpyDeviceToDevice, ctx->stream));
    return HD_OK;
}

hd_status hd_positions_device(hd_ctx* ctx, double* xy_device) {
    if (!ctx || !xy_device) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] {
        return hd::launch_positions(ctx->cfg(), ctx->frame, ctx->buf[ctx->cur], xy_device);
    }));
    return HD_OK;
}

hd_status hd_positions(hd_ctx* ctx, double* xy) {
    const Range range("hd_positions");
    if (!ctx || !xy) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] { return hd::launch_positions(ctx->cfg(), ctx->frame, ctx->buf[ctx->cur], ctx->xy); }));
    HD_CK(ctx, cudaMemcpyAsync(xy, ctx->xy, sizeof(double) * 2 * size_t(ctx->Ntot), cudaMemcpyDeviceToHost,
                               ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx);
}

hd_status hd_set_positions(hd_ctx* ctx, const double* xy) {
    const Range range("hd_set_positions");
    if (!ctx || !xy) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    // upload, then bin on the device into the other generation; switch to it
    // only when every disk found a slot, so a rejected input changes nothing
    const hd::LaunchCfg c = ctx->cfg();
    const size_t cnt_bytes = size_t(ctx->Ctot) + kCellPad;
    CellBufs& to = ctx->buf[ctx->cur ^ 1];
    HD_CK(ctx, cudaMemcpyAsync(ctx->xy, xy, sizeof(double) * 2 * size_t(ctx->Ntot), cudaMemcpyHostToDevice,
                               ctx->stream));
    HD_CK(ctx, cudaMemsetAsync(to.cnt, 0, cnt_bytes, ctx->stream));
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] { return hd::launch_bin(c, ctx->Ntot, ctx->sigma, ctx->xy, to, ctx->err); }));
    int flag = 0;
    HD_CK(ctx, cudaMemcpyAsync(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const int bad = flag & (hd::kErrBinOverflow | hd::kErrBinInput);
    if (bad) {
        HD_CK(ctx, cudaMemsetAsync(to.cnt, 0, cnt_bytes, ctx->stream));  // the rebuild expects it cleared
        const int keep = flag & ~bad;
        HD_CK(ctx, cudaMemcpyAsync(ctx->err, &keep, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
        return (bad & hd::kErrBinInput) ? HD_ERR_ARG : HD_ERR_OVERFLOW;
    }
    ctx->cur ^= 1;
    // the generation left behind must be cleared for the next rebuild; the
    // frame is unshifted (stream-ordered before any later work: no wait)
    HD_CK(ctx, cudaMemsetAsync(ctx->buf[ctx->cur ^ 1].cnt, 0, cnt_bytes, ctx->stream));
    HD_CK(ctx, cudaMemsetAsync(ctx->frame, 0, sizeof(Frame) * size_t(ctx->R), ctx->stream));
    return flags_status(ctx, flag);  // the word as read after the binning, which follows all earlier work
}

hd_status hd_stats(hd_ctx* ctx, uint64_t* attempts, uint64_t* accepts) {
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    std::vector<unsigned long long> c(size_t(2 * ctx->R));
    HD_CK(ctx, cudaMemcpyAsync(c.data(), ctx->counters, c.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < ctx->R; ++r) {
        if (attempts) attempts[r] = c[size_t(2 * r)];
        if (accepts) accepts[r] = c[size_t(2 * r + 1)];
    }
    return check_flags(ctx);
}

hd_status hd_get_geometry(hd_ctx* ctx, int32_t r, hd_geometry* g) {
    if (!ctx || !g || r < 0 || r >= ctx->R) return HD_ERR_ARG;
    const Rep& rep = ctx->reps[size_t(r)];
    g->N = rep.N;
    g->m = rep.m;
    g->capacity = ctx->cap;
    g->trials_per_cell = rep.nt;
    g->precision = ctx->fixed ? HD_FIXED32 : HD_FP64;
    g->hist_bins = ctx->K;
    g->graph_branches = ctx->strips > 1 ? ctx->strips : (ctx->branches ? ctx->R : 1);
    g->L = ctx->fixed ? double(rep.LF) / kFx : rep.L;
    g->w = ctx->fixed ? double(rep.W) / kFx : rep.w;
    g->delta = ctx->fixed ? double(rep.D) / kFx : rep.delta;
    g->eta = double(rep.N) * kPi / (g->L * g->L);
    g->hist_dr = rep.dr;
    g->sweeps = ctx->sweeps[size_t(r)];
    return HD_OK;
}

int32_t hd_replicas(const hd_ctx* ctx) { return ctx ? ctx->R : 0; }

hd_status hd_series_reserve(hd_ctx* ctx, int64_t steps) {
    if (!ctx || steps < 1) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);  // they hold the old series pointers
    if (ctx->series) cudaFree(ctx->series);
    ctx->series = nullptr;
    ctx->series_cap = 0;
    if (!ctx->series_len) HD_CK(ctx, cudaMalloc(&ctx->series_len, sizeof(int64_t)));
    HD_CK(ctx, cudaMalloc(&ctx->series, sizeof(double) * 4 * size_t(ctx->R) * size_t(steps)));
    HD_CK(ctx, cudaMemset(ctx->series_len, 0, sizeof(int64_t)));
    ctx->series_cap = steps;
    return HD_OK;
}

hd_status hd_run(hd_ctx* ctx, int64_t steps, int32_t sweeps_per_step, int32_t measure) {
    const Range range("hd_run");
    if (!ctx || steps < 0 || sweeps_per_step < 0 || (sweeps_per_step == 0 && !measure) || ctx->R > 1024 ||
        measure < 0 || measure > 2)
        return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    if (measure)
        for (const Rep& r : ctx->reps)
            if (2 * r.hist_R + 1 > r.m) return HD_ERR_REACH;
    if (measure && !ctx->series) {
        const hd_status s = hd_series_reserve(ctx, 4096);
        if (s != HD_OK) return s;
    }
    const bool meas = measure != 0;
    const bool local = measure == 2;
    const bool prof = ctx->profiling;
    if (prof && !prof_flush(ctx)) return fail_cuda(ctx);
    if (!ctx->capture_stream) HD_CK(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    for (int64_t k = 0; k < steps; ++k) {
        const int parity = ctx->cur;
        hd_ctx::StepGraph* g = nullptr;
        for (auto& x : ctx->graphs)
            if (x.sweeps == sweeps_per_step && x.measure == meas && x.parity == parity && x.profiled == prof &&
                x.local == local)
                g = &x;
        if (!g) {
            hd_ctx::StepGraph ng;
            ng.sweeps = sweeps_per_step;
            ng.measure = meas;
            ng.local = local;
            ng.parity = parity;
            ng.profiled = prof;
            ng.ev0 = ctx->gev_used;
            if (prof) {  // two events per launch: draws, 5 per sweep, the measurement
                const size_t bound = 2 * (size_t(sweeps_per_step) * 5 + size_t(sweeps_per_step) / hd::kMaxChunk + 16);
                while (ctx->gev.size() < ng.ev0 + bound) {
                    cudaEvent_t e;
                    HD_CK(ctx, cudaEventCreate(&e));
                    ctx->gev.push_back(e);
                }
                ctx->prof_capture = &ng;
                hd::g_no_pdl = true;
            }
            int64_t before[HD_KERNEL_CLASSES];
            std::memcpy(before, ctx->launches, sizeof(before));
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                ce = enqueue_step(ctx, ctx->capture_stream, sweeps_per_step, meas, local, true);
                const cudaError_t ee = cudaStreamEndCapture(ctx->capture_stream, &graph);
                if (ce == cudaSuccess) ce = ee;
            }
            ctx->prof_capture = nullptr;
            hd::g_no_pdl = false;
            ctx->cur = parity;  // capture only recorded the launches
            for (int c = 0; c < HD_KERNEL_CLASSES; ++c) {
                ng.launches[c] = ctx->launches[c] - before[c];
                ctx->launches[c] = before[c];
            }
            if (ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return fail_cuda(ctx);
            }
            const cudaError_t ie = cudaGraphInstantiate(&ng.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return fail_cuda(ctx);
            ctx->gev_used = ng.ev0 + 2 * ng.ev_cls.size();
            ctx->graphs.push_back(std::move(ng));
            g = &ctx->graphs.back();
        }
        HD_CK(ctx, cudaGraphLaunch(g->exec, ctx->stream));
        for (int c = 0; c < HD_KERNEL_CLASSES; ++c) ctx->launches[c] += g->launches[c];
        if (sweeps_per_step & 1) ctx->cur ^= 1;
        if (prof) {  // read this replay's kernel times before the next one
            HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
            for (size_t i = 0; i < g->ev_cls.size(); ++i) {
                float ms = 0.f;
                HD_CK(ctx, cudaEventElapsedTime(&ms, ctx->gev[g->ev0 + 2 * i], ctx->gev[g->ev0 + 2 * i + 1]));
                ctx->kernel_ms[g->ev_cls[i]] += double(ms);
            }
        }
    }
    for (auto& s : ctx->sweeps) s += steps * sweeps_per_step;
    return HD_OK;
}

hd_status hd_series(hd_ctx* ctx, int64_t* n_steps, double* out, int64_t max_steps) {
    if (!ctx || !n_steps || max_steps < 0) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    *n_steps = 0;
    if (!ctx->series) return HD_OK;
    // the count and the error word with one wait
    HD_CK(ctx, cudaMemcpyAsync(&ctx->pinned[0], ctx->series_len, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaMemcpyAsync(&ctx->pinned[1], ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t len = ctx->pinned[0];
    const hd_status f = flags_status(ctx, int(ctx->pinned[1] & 0xffffffff));
    if (f != HD_OK) return f;
    const int64_t n = std::min(len, max_steps);
    if (out && n > 0)
        HD_CK(ctx, cudaMemcpy(out, ctx->series, sizeof(double) * 4 * size_t(ctx->R) * size_t(n), cudaMemcpyDeviceToHost));
    *n_steps = n;
    return HD_OK;
}

hd_status hd_series_clear(hd_ctx* ctx) {
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    if (ctx->series_len) HD_CK(ctx, cudaMemsetAsync(ctx->series_len, 0, sizeof(int64_t), ctx->stream));
    return HD_OK;
}

// Checkpoint layout: header, per-replica geometry keys, then the current cell
// generation (occupancy, slot planes of offsets, slot planes of ids), frames,
// sweep counters, trial counters and host sweep tallies.
namespace {
struct CkHeader {
    char magic[8];
    int32_t version, R, fixed, cap;
    int64_t Ctot, Ntot;
    int32_t K, sweep_kernel;
};
struct CkRep {
    int64_t N;
    int32_t m, W, D, nt;
    uint32_t key0, key1;
    double w, delta, dr;
};
constexpr char kCkMagic[8] = {'H', 'D', 'C', 'K', 'P', 'T', '0', '1'};

size_t pos_bytes(const hd_ctx* ctx) { return ctx->fixed ? sizeof(int2) : sizeof(double2); }

size_t checkpoint_bytes(const hd_ctx* ctx) {
    const size_t slots = size_t(ctx->Ctot) * ctx->cap;
    return sizeof(CkHeader) + sizeof(CkRep) * size_t(ctx->R) + size_t(ctx->Ctot) + slots * pos_bytes(ctx) +
           slots * sizeof(int32_t) + sizeof(Frame) * size_t(ctx->R) + sizeof(uint64_t) * size_t(ctx->R) +
           sizeof(unsigned long long) * 2 * size_t(ctx->R) + sizeof(int64_t) * size_t(ctx->R);
}

void fill_header(const hd_ctx* ctx, CkHeader& h, std::vector<CkRep>& reps) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkMagic, sizeof(kCkMagic));
    h.version = 1;
    h.R = ctx->R;
    h.fixed = ctx->fixed ? 1 : 0;
    h.cap = ctx->cap;
    h.Ctot = ctx->Ctot;
    h.Ntot = ctx->Ntot;
    h.K = ctx->K;
    h.sweep_kernel = 0;  // reserved: every sweep kernel runs the same chain on the same cell state
    reps.assign(size_t(ctx->R), CkRep{});
    for (int r = 0; r < ctx->R; ++r) {
        const Rep& s = ctx->reps[size_t(r)];
        CkRep& c = reps[size_t(r)];
        std::memset(&c, 0, sizeof(c));
        c.N = s.N;
        c.m = s.m;
        c.W = s.W;
        c.D = s.D;
        c.nt = s.nt;
        c.key0 = s.key0;
        c.key1 = s.key1;
        c.w = s.w;
        c.delta = s.delta;
        c.dr = s.dr;
    }
}
}  // namespace

namespace {
// Set replica r's step to delta (sigma units) in the host copy; false if the
// value is out of range for the cell.
bool set_rep_delta(hd_ctx* ctx, int r, double delta) {
    Rep& rep = ctx->reps[size_t(r)];
    if (!(delta >= 0x1p-900)) return false;  // positive, and see scale_2m53
    if (ctx->fixed) {
        const int64_t D = std::llround(delta * kFx);
        if (D < 1 || D >= rep.W) return false;
        rep.D = int32_t(D);
        rep.delta = delta;
    } else {
        if (!(delta < rep.w)) return false;
        rep.delta = delta;
        set_f32_bounds(rep);
    }
    return true;
}

hd_status upload_reps(hd_ctx* ctx) {
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    HD_CK(ctx, cudaMemcpy(ctx->reps_d, ctx->reps.data(), sizeof(Rep) * size_t(ctx->R), cudaMemcpyHostToDevice));
    drop_graphs(ctx);  // captured launches may hold the replica constants by value
    return HD_OK;
}
}  // namespace

hd_status hd_set_delta(hd_ctx* ctx, const double* delta) {
    if (!ctx || !delta) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    const std::vector<Rep> saved = ctx->reps;
    for (int r = 0; r < ctx->R; ++r) {
        if (!set_rep_delta(ctx, r, delta[r] / ctx->sigma)) {
            ctx->reps = saved;
            return HD_ERR_ARG;
        }
    }
    return upload_reps(ctx);
}

hd_status hd_tune_delta(hd_ctx* ctx, double target, int32_t sweeps_per_probe, int32_t probes, double* delta_out) {
    const Range range("hd_tune_delta");
    if (!ctx || !(target > 0.0 && target < 1.0) || sweeps_per_probe < 1 || probes < 1) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    const int R = ctx->R;
    std::vector<double> lo(size_t(R), 0.0), hi(size_t(R), 0.0);
    std::vector<unsigned long long> c0(size_t(2 * R)), c1(size_t(2 * R));
    for (int r = 0; r < R; ++r) {
        const Rep& rep = ctx->reps[size_t(r)];
        lo[size_t(r)] = ctx->fixed ? 1.0 / kFx : 1e-6;
        hi[size_t(r)] = ctx->fixed ? double(rep.W - 1) / kFx : rep.w_below;
    }
    // Damped multiplicative update on log(delta): the acceptance falls
    // smoothly with delta, so log(delta) <- log(delta) + g*log(acc/target)
    // converges for any local log-log slope below 2/g, and it keeps tracking
    // a chain whose acceptance still drifts (e.g. relaxing from a lattice),
    // which an interval bisection cannot.
    const double g = 0.7;
    for (int it = 0; it < probes; ++it) {
        HD_CK(ctx, cudaMemcpy(c0.data(), ctx->counters, sizeof(unsigned long long) * c0.size(), cudaMemcpyDeviceToHost));
        const hd_status s = hd_sweep(ctx, sweeps_per_probe);
        if (s != HD_OK) return s;
        HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
        HD_CK(ctx, cudaMemcpy(c1.data(), ctx->counters, sizeof(unsigned long long) * c1.size(), cudaMemcpyDeviceToHost));
        for (int r = 0; r < R; ++r) {
            const double att = double(c1[size_t(2 * r)] - c0[size_t(2 * r)]);
            const double acc = double(c1[size_t(2 * r + 1)] - c0[size_t(2 * r + 1)]);
            if (att <= 0.0) continue;
            const double d = ctx->reps[size_t(r)].delta;
            const double f = acc > 0.0 ? std::pow(acc / att / target, g) : 0.25;
            const double next = std::min(hi[size_t(r)], std::max(lo[size_t(r)], d * std::min(4.0, std::max(0.25, f))));
            set_rep_delta(ctx, r, next);
        }
        const hd_status u = upload_reps(ctx);
        if (u != HD_OK) return u;
    }
    if (delta_out)
        for (int r = 0; r < R; ++r) delta_out[r] = ctx->reps[size_t(r)].delta * ctx->sigma;
    return check_flags(ctx);
}

hd_status hd_checkpoint_size(hd_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return HD_ERR_ARG;
    *bytes = checkpoint_bytes(ctx);
    return HD_OK;
}

hd_status hd_checkpoint(hd_ctx* ctx, void* buf, size_t bytes) {
    const Range range("hd_checkpoint");
    if (!ctx || !buf || bytes < checkpoint_bytes(ctx)) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const hd_status f = check_flags(ctx);
    if (f != HD_OK) return f;
    CkHeader h;
    std::vector<CkRep> reps;
    fill_header(ctx, h, reps);
    unsigned char* p = static_cast<unsigned char*>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    std::memcpy(p, reps.data(), sizeof(CkRep) * reps.size());
    p += sizeof(CkRep) * reps.size();
    const size_t slots = size_t(ctx->Ctot) * ctx->cap;
    const CellBufs& b = ctx->buf[ctx->cur];
    HD_CK(ctx, cudaMemcpy(p, b.cnt, size_t(ctx->Ctot), cudaMemcpyDeviceToHost));
    p += size_t(ctx->Ctot);
    HD_CK(ctx, cudaMemcpy(p, b.pos, slots * pos_bytes(ctx), cudaMemcpyDeviceToHost));
    p += slots * pos_bytes(ctx);
    HD_CK(ctx, cudaMemcpy(p, b.pid, slots * sizeof(int32_t), cudaMemcpyDeviceToHost));
    p += slots * sizeof(int32_t);
    HD_CK(ctx, cudaMemcpy(p, ctx->frame, sizeof(Frame) * size_t(ctx->R), cudaMemcpyDeviceToHost));
    p += sizeof(Frame) * size_t(ctx->R);
    HD_CK(ctx, cudaMemcpy(p, ctx->sweep_ctr, sizeof(uint64_t) * size_t(ctx->R), cudaMemcpyDeviceToHost));
    p += sizeof(uint64_t) * size_t(ctx->R);
    HD_CK(ctx, cudaMemcpy(p, ctx->counters, sizeof(unsigned long long) * 2 * size_t(ctx->R), cudaMemcpyDeviceToHost));
    p += sizeof(unsigned long long) * 2 * size_t(ctx->R);
    std::memcpy(p, ctx->sweeps.data(), sizeof(int64_t) * size_t(ctx->R));
    return HD_OK;
}

hd_status hd_restore(hd_ctx* ctx, const void* buf, size_t bytes) {
    const Range range("hd_restore");
    if (!ctx || !buf || bytes < checkpoint_bytes(ctx)) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    CkHeader want, got;
    std::vector<CkRep> want_reps;
    fill_header(ctx, want, want_reps);
    const unsigned char* p = static_cast<const unsigned char*>(buf);
    std::memcpy(&got, p, sizeof(got));
    p += sizeof(got);
    if (std::memcmp(&got, &want, sizeof(got)) != 0) return HD_ERR_ARG;
    if (std::memcmp(p, want_reps.data(), sizeof(CkRep) * want_reps.size()) != 0) return HD_ERR_ARG;
    p += sizeof(CkRep) * want_reps.size();
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const size_t slots = size_t(ctx->Ctot) * ctx->cap;
    const CellBufs& b = ctx->buf[ctx->cur];
    HD_CK(ctx, cudaMemcpy(b.cnt, p, size_t(ctx->Ctot), cudaMemcpyHostToDevice));
    p += size_t(ctx->Ctot);
    HD_CK(ctx, cudaMemcpy(b.pos, p, slots * pos_bytes(ctx), cudaMemcpyHostToDevice));
    p += slots * pos_bytes(ctx);
    HD_CK(ctx, cudaMemcpy(b.pid, p, slots * sizeof(int32_t), cudaMemcpyHostToDevice));
    p += slots * sizeof(int32_t);
    // the other generation's occupancy must be zero for the next scatter rebuild
    HD_CK(ctx, cudaMemset(ctx->buf[ctx->cur ^ 1].cnt, 0, size_t(ctx->Ctot) + kCellPad));
    HD_CK(ctx, cudaMemcpy(ctx->frame, p, sizeof(Frame) * size_t(ctx->R), cudaMemcpyHostToDevice));
    p += sizeof(Frame) * size_t(ctx->R);
    HD_CK(ctx, cudaMemcpy(ctx->sweep_ctr, p, sizeof(uint64_t) * size_t(ctx->R), cudaMemcpyHostToDevice));
    p += sizeof(uint64_t) * size_t(ctx->R);
    HD_CK(ctx, cudaMemcpy(ctx->counters, p, sizeof(unsigned long long) * 2 * size_t(ctx->R), cudaMemcpyHostToDevice));
    p += sizeof(unsigned long long) * 2 * size_t(ctx->R);
    std::memcpy(ctx->sweeps.data(), p, sizeof(int64_t) * size_t(ctx->R));
    return HD_OK;
}

hd_status hd_profile(hd_ctx* ctx, int32_t enable) {
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    if (!prof_flush(ctx)) return fail_cuda(ctx);
    if (enable) {
        if (ctx->ev.empty()) {
            ctx->ev.resize(8192);
            for (auto& e : ctx->ev)
                if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda(ctx);
        }
        for (int k = 0; k < HD_KERNEL_CLASSES; ++k) {
            ctx->kernel_ms[k] = 0.0;
            ctx->launches[k] = 0;
        }
    }
    ctx->profiling = enable != 0;
    return HD_OK;
}

hd_status hd_kernel_times(hd_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    if (!prof_flush(ctx)) return fail_cuda(ctx);
    for (int k = 0; k < HD_KERNEL_CLASSES; ++k) {
        if (ms) ms[k] = ctx->kernel_ms[k];
        if (launches) launches[k] = ctx->launches[k];
    }
    return HD_OK;
}

}  // extern "C"

namespace {

// The recorded series length (synchronises).
hd_status series_length(hd_ctx* ctx, int64_t& T) {
    T = 0;
    if (!ctx->series) return HD_OK;
    HD_CK(ctx, cudaMemcpyAsync(&T, ctx->series_len, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

// C[R][max_lag + 1] of the current series into ctx->acf.
hd_status enqueue_acf(hd_ctx* ctx, int64_t T, int64_t max_lag) {
    const size_t need = size_t(ctx->R) * size_t(max_lag + 1);
    if (need > ctx->acf_cap) {
        if (ctx->acf) cudaFree(ctx->acf);
        ctx->acf = nullptr;
        ctx->acf_cap = 0;
        HD_CK(ctx, cudaMalloc(&ctx->acf, need * sizeof(double2)));
        ctx->acf_cap = need;
    }
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] { return hd::launch_acf(ctx->cfg(), ctx->series, T, max_lag, ctx->acf); }));
    return HD_OK;
}

}  // namespace

hd_status hd_psi6_acf(hd_ctx* ctx, int64_t max_lag, double* acf) {
    if (!ctx || !acf || max_lag < 0) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    int64_t T = 0;
    hd_status st = series_length(ctx, T);
    if (st != HD_OK) return st;
    if (max_lag >= T) return HD_ERR_ARG;
    st = enqueue_acf(ctx, T, max_lag);
    if (st != HD_OK) return st;
    HD_CK(ctx, cudaMemcpyAsync(acf, ctx->acf, sizeof(double2) * size_t(ctx->R) * size_t(max_lag + 1),
                               cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

hd_status hd_psi6_tau(hd_ctx* ctx, int64_t lag_lo, int64_t lag_hi, double* tau) {
    if (!ctx || !tau || lag_lo < 0 || lag_hi < lag_lo) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    int64_t T = 0;
    hd_status st = series_length(ctx, T);
    if (st != HD_OK) return st;
    if (lag_hi >= T) return HD_ERR_ARG;
    st = enqueue_acf(ctx, T, lag_hi);
    if (st != HD_OK) return st;
    if (!ctx->tau) HD_CK(ctx, cudaMalloc(&ctx->tau, sizeof(double) * size_t(ctx->R)));
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS,
                      [&] { return hd::launch_acf_tau(ctx->cfg(), lag_hi, lag_lo, lag_hi, ctx->acf, ctx->tau); }));
    HD_CK(ctx, cudaMemcpyAsync(tau, ctx->tau, sizeof(double) * size_t(ctx->R), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

hd_status hd_psi6_field(hd_ctx* ctx, int32_t bins, double* field) {
    const Range range("hd_psi6_field");
    if (!ctx || !field || bins < 1 || bins > 65536) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    const size_t need = size_t(ctx->R) * size_t(bins) * size_t(bins);
    if (need > (size_t(1) << 28)) return HD_ERR_ARG;
    if (need > ctx->field_cap) {
        if (ctx->field_acc) cudaFree(ctx->field_acc);
        if (ctx->field) cudaFree(ctx->field);
        ctx->field_acc = nullptr;
        ctx->field = nullptr;
        ctx->field_cap = 0;
        HD_CK(ctx, cudaMalloc(&ctx->field_acc, need * 3 * sizeof(double)));
        HD_CK(ctx, cudaMalloc(&ctx->field, need * sizeof(double2)));
        ctx->field_cap = need;
    }
    // global positions and local psi_6 of the current state, then the area means
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] {
        return hd::launch_positions(ctx->cfg(), ctx->frame, ctx->buf[ctx->cur], ctx->xy);
    }));
    HD_CK(ctx, enqueue_psi6(ctx, ctx->stream, true, false));
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] {
        return hd::launch_field(ctx->cfg(), ctx->Ntot, bins, ctx->xy, ctx->psi_local, ctx->field_acc, ctx->field);
    }));
    HD_CK(ctx, cudaMemcpyAsync(field, ctx->field, need * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx);
}

namespace {

template <class T>
hd_status grow(hd_ctx* ctx, T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return HD_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    HD_CK(ctx, cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T)));
    cap = need;
    return HD_OK;
}

// S at the wave vectors already in ctx->sq_hk ([R][nq]); positions refreshed first.
hd_status enqueue_sq(hd_ctx* ctx, int nq) {
    std::vector<int64_t> Ns;
    for (const Rep& r : ctx->reps) Ns.push_back(r.N);
    const int nbx = hd::sq_disk_blocks(Ns);
    const size_t need = size_t(ctx->R) * size_t(nbx) * size_t(nq);
    if (need > (size_t(1) << 27)) return HD_ERR_ARG;
    hd_status st = grow(ctx, ctx->sq_part, ctx->sq_part_cap, need);
    if (st != HD_OK) return st;
    st = grow(ctx, ctx->sq_S, ctx->sq_S_cap, size_t(ctx->R) * nq);
    if (st != HD_OK) return st;
    if (!ctx->sq_best) HD_CK(ctx, cudaMalloc(&ctx->sq_best, sizeof(int) * size_t(ctx->R)));
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] {
        return hd::launch_positions(ctx->cfg(), ctx->frame, ctx->buf[ctx->cur], ctx->xy);
    }));
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] {
        return hd::launch_sq(ctx->cfg(), nq, ctx->sq_hk, ctx->xy, nbx, ctx->sq_part, ctx->sq_S, ctx->sq_best);
    }));
    return HD_OK;
}

}  // namespace

hd_status hd_structure_factor(hd_ctx* ctx, int32_t nq, const int32_t* hk, double* S) {
    const Range range("hd_structure_factor");
    if (!ctx || !hk || !S || nq < 1 || nq > 65536) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    hd_status st = grow(ctx, ctx->sq_hk, ctx->sq_cap, size_t(ctx->R) * nq);
    if (st != HD_OK) return st;
    HD_CK(ctx, cudaMemcpyAsync(ctx->sq_hk, hk, sizeof(int2) * size_t(ctx->R) * nq, cudaMemcpyHostToDevice, ctx->stream));
    st = enqueue_sq(ctx, nq);
    if (st != HD_OK) return st;
    HD_CK(ctx, cudaMemcpyAsync(S, ctx->sq_S, sizeof(double) * size_t(ctx->R) * nq, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

hd_status hd_positional_q0(hd_ctx* ctx, int32_t half_width, int32_t* hk0, double* S0) {
    const Range range("hd_positional_q0");
    if (!ctx || !hk0 || half_width < 0 || half_width > 64) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    const int w = 2 * half_width + 1, nq = w * w;
    hd_status st = grow(ctx, ctx->sq_hk, ctx->sq_cap, size_t(ctx->R) * nq);
    if (st != HD_OK) return st;
    HD_CK(ctx, enqueue_psi6(ctx, ctx->stream, false, false));  // Psi_6 orients the window
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] { return hd::launch_q0_window(ctx->cfg(), half_width, ctx->psi_res, ctx->sq_hk); }));
    st = enqueue_sq(ctx, nq);
    if (st != HD_OK) return st;
    std::vector<int2> win(size_t(ctx->R) * nq);
    std::vector<int> best(size_t(ctx->R));
    std::vector<double> Sv(size_t(ctx->R) * nq);
    HD_CK(ctx, cudaMemcpyAsync(win.data(), ctx->sq_hk, sizeof(int2) * win.size(), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaMemcpyAsync(best.data(), ctx->sq_best, sizeof(int) * best.size(), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaMemcpyAsync(Sv.data(), ctx->sq_S, sizeof(double) * Sv.size(), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const hd_status f = check_flags(ctx);
    if (f != HD_OK) return f;
    for (int r = 0; r < ctx->R; ++r) {
        const size_t i = size_t(r) * nq + size_t(best[size_t(r)]);
        hk0[2 * r] = win[i].x;
        hk0[2 * r + 1] = win[i].y;
        if (S0) S0[r] = Sv[i];
    }
    return HD_OK;
}

namespace {

// chi_j of the current state for hk0[R][2] into ctx->chi (positions refreshed first).
hd_status enqueue_chi(hd_ctx* ctx, const int32_t* hk0) {
    if (!ctx->chi) HD_CK(ctx, cudaMalloc(&ctx->chi, sizeof(double2) * size_t(std::max<int64_t>(ctx->Ntot, 1))));
    hd_status st = grow(ctx, ctx->sq_hk, ctx->sq_cap, size_t(ctx->R));
    if (st != HD_OK) return st;
    HD_CK(ctx, cudaMemcpyAsync(ctx->sq_hk, hk0, sizeof(int2) * size_t(ctx->R), cudaMemcpyHostToDevice, ctx->stream));
    HD_CK(ctx, launch(ctx, HD_K_POSITIONS, [&] {
        return hd::launch_positions(ctx->cfg(), ctx->frame, ctx->buf[ctx->cur], ctx->xy);
    }));
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] { return hd::launch_chi(ctx->cfg(), ctx->Ntot, ctx->sq_hk, ctx->xy, ctx->chi); }));
    return HD_OK;
}

}  // namespace

hd_status hd_positional_field(hd_ctx* ctx, const int32_t* hk0, int32_t bins, double* field) {
    const Range range("hd_positional_field");
    if (!ctx || !hk0 || !field || bins < 1 || bins > 65536) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    const size_t need = size_t(ctx->R) * size_t(bins) * size_t(bins);
    if (need > (size_t(1) << 28)) return HD_ERR_ARG;
    hd_status st = enqueue_chi(ctx, hk0);
    if (st != HD_OK) return st;
    if (need > ctx->field_cap) {
        if (ctx->field_acc) cudaFree(ctx->field_acc);
        if (ctx->field) cudaFree(ctx->field);
        ctx->field_acc = nullptr;
        ctx->field = nullptr;
        ctx->field_cap = 0;
        HD_CK(ctx, cudaMalloc(&ctx->field_acc, need * 3 * sizeof(double)));
        HD_CK(ctx, cudaMalloc(&ctx->field, need * sizeof(double2)));
        ctx->field_cap = need;
    }
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] {
        return hd::launch_field(ctx->cfg(), ctx->Ntot, bins, ctx->xy, ctx->chi, ctx->field_acc, ctx->field);
    }));
    HD_CK(ctx, cudaMemcpyAsync(field, ctx->field, need * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

hd_status hd_positional_corr(hd_ctx* ctx, const int32_t* hk0, int32_t nr, double dr, double* C) {
    const Range range("hd_positional_corr");
    if (!ctx || !hk0 || !C || nr < 1 || nr > 1024 || !(dr > 0.0)) return HD_ERR_ARG;
    if (ctx->sticky != HD_OK) return HD_ERR_STATE;
    // cell reach that holds every pair within the largest window, r_nr + 1 (sigma units)
    const double rmax = double(nr) * dr + 1.0;
    int reach = 0;
    for (const Rep& r : ctx->reps) reach = std::max(reach, int(std::ceil(rmax / r.w)) + 1);
    for (const Rep& r : ctx->reps)
        if (2 * reach + 1 > r.m) return HD_ERR_REACH;
    hd_status st = enqueue_chi(ctx, hk0);
    if (st != HD_OK) return st;
    const size_t need = size_t(ctx->R) * size_t(nr);
    if (need > ctx->corr_cap) {
        if (ctx->corr_acc) cudaFree(ctx->corr_acc);
        if (ctx->corr) cudaFree(ctx->corr);
        ctx->corr_acc = nullptr;
        ctx->corr = nullptr;
        ctx->corr_cap = 0;
        HD_CK(ctx, cudaMalloc(&ctx->corr_acc, need * 3 * sizeof(double)));
        HD_CK(ctx, cudaMalloc(&ctx->corr, need * sizeof(double2)));
        ctx->corr_cap = need;
    }
    HD_CK(ctx, launch(ctx, HD_K_ANALYSIS, [&] {
        return hd::launch_poscorr(ctx->cfg(), ctx->buf[ctx->cur], ctx->xy, ctx->chi, nr, dr / ctx->sigma, reach,
                                  ctx->corr_acc, ctx->corr);
    }));
    HD_CK(ctx, cudaMemcpyAsync(C, ctx->corr, need * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}
