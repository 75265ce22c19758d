// hd_kernels.h -- host-side launch interface of the MPMC kernels.  Each
// launcher enqueues one kernel on `stream` and returns the launch status.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

#include "hd_device.cuh"
#include "hd_exact.cuh"

namespace hd {

// Device buffers of one cell-list generation (ping-pong pair in the context).
struct CellBufs {
    uint8_t* cnt;   // [cells] occupancy
    void* pos;      // [cells * cap] double2 (FP64) or int2 (fixed) cell offsets
    int32_t* pid;   // [cells * cap] disk id within the replica
};

struct LaunchCfg {
    const Rep* reps;   // device array [R]
    const Rep* rep0;   // host copy of replica 0 (passed by value to the hot kernels when R == 1)
    const uint16_t* rep_of_act;   // replica of each block of the active-cell grid (R > 1)
    const uint16_t* rep_of_cell;  // replica of each block of the whole-cell grid (R > 1)
    int R;
    int cap;           // 4 or 9
    bool fixed;        // fixed-point form
    int threads;       // threads per block (cells per block of the active-cell grid)
    int tpc;           // threads per active cell of the split colour pass (1, 2, 4 or 8)
    int ntc;           // trials per occupied cell and pass when every replica has the same 1 or 2, else 0
    int blocks_cell;   // whole-cell grid size (all replicas)
    int blocks_act;    // active-cell grid size (all replicas)
    int blocks_tile;   // fused-sweep tile grid size (all replicas)
    int blocks_t32;    // 32 x (threads / 32) cell-tile grid size (all replicas)
    int blocks_seg;    // half-row segment grid size of one colour pass (all replicas)
    int persist_blocks;  // grid of the persistent sweep (resident blocks), from persist_grid
    bool persist_stall;  // test hook: the persistent sweep withholds one item and gives up waiting early
    // One strip of a one-replica sweep (graph wavefront): a colour pass over
    // the active cells [act_lo, act_hi) of its plane, a rebuild over the
    // entries band_lo .. band_lo + band_span - 1 of each colour plane.  The
    // defaults (0, ~0u, 0, 0) cover every cell.
    uint32_t act_lo = 0u, act_hi = ~0u;
    uint32_t band_lo = 0u, band_span = 0u;
    cudaStream_t stream;
};

// Set on a host thread while it captures a step graph with timing events
// between the kernels: programmatic dependent launch is then left off, since
// an event node separates every pair of kernels.
inline thread_local bool g_no_pdl = false;

// Launch `kernel` on stream s; on a created stream the launch opts into
// programmatic dependent launch, so the kernel's blocks may be scheduled while
// the previous kernel drains (every kernel starts with pdl_begin()).
template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = (s != nullptr && !g_no_pdl) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

cudaError_t launch_draws(const LaunchCfg& c, Frame* table, Frame* cur, uint64_t* sweep_ctr, int nchunk);
cudaError_t launch_rebuild(const LaunchCfg& c, const Frame* table, int j, CellBufs from, CellBufs to,
                           int* err);
// Resident blocks per SM of the split colour pass of one replica (the
// occupancy the pass runs at, for sizing the graph wavefront's strips).
cudaError_t pass_blocks_per_sm(const LaunchCfg& c, int* blocks);
cudaError_t launch_pass(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                        unsigned long long* counters);
// The colour pass with tpc > 1 threads per active cell (blocks of threads x tpc).
cudaError_t launch_pass_group(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                              unsigned long long* counters);
// The colour pass with each block's neighbourhood staged by bulk copies (TMA).
cudaError_t launch_pass_tma(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                            unsigned long long* counters, int* err);
// One whole sweep (rebuild + four colour passes) per launch, staged in shared
// memory by tiles of fused_tile(fixed, cap) cells per side.
int fused_tile(bool fixed, int cap);
cudaError_t launch_sweep_fused(const LaunchCfg& c, const Frame* table, int j, CellBufs from, CellBufs to,
                               unsigned long long* counters, int* err);
// nsweeps <= kMaxChunk sweeps of the draw table in one launch (rebuild and
// four colour passes per sweep, scheduled as a wavefront over bands of two
// cell rows), from `from` into `to` for the first sweep and alternating
// after; sync: persist_sync_words(total_bands) words of device scratch,
// cleared by the launcher.
size_t persist_sync_words(int total_bands);
cudaError_t persist_grid(const LaunchCfg& c, int* blocks);
cudaError_t launch_sweeps_persist(const LaunchCfg& c, const Frame* table, int nsweeps, CellBufs from, CellBufs to,
                                  unsigned long long* counters, int* err, uint32_t* sync, int total_bands);
cudaError_t launch_positions(const LaunchCfg& c, const Frame* cur, CellBufs cells, double* xy);
// Psi_6 autocorrelation of the measurement series (series[T][R][4]) for lags
// 0..max_lag into C[R][max_lag + 1], and the correlation time from it.
cudaError_t launch_acf(const LaunchCfg& c, const double* series, int64_t T, int64_t max_lag, double2* C);
cudaError_t launch_acf_tau(const LaunchCfg& c, int64_t max_lag, int64_t lag_lo, int64_t lag_hi, const double2* C,
                           double* tau);
// Coarse psi_6 field over bins x bins sampling areas per replica (acc: R bins^2 x 3 doubles of scratch).
cudaError_t launch_field(const LaunchCfg& c, int64_t Ntot, int bins, const double* xy, const double2* psi,
                         double* acc, double2* out);

// Measurement.
struct HistCfg {
    int K;
    const double* edges;      // [K + 1] FP64 squared bin edges
    const long long* edgesF;  // [K + 1] fixed-point squared bin edges
    int halo;                 // largest histogram reach (cells) over the replicas
};
cudaError_t launch_hist(const LaunchCfg& c, const HistCfg& h, CellBufs cells, unsigned long long* hist);
// The quartic fit's design matrix depends on K alone: launch_fit_factor
// writes its Householder factor (fit_factor_len(K) doubles) once per context,
// launch_fit applies it to each measurement.
size_t fit_factor_len(int K);
cudaError_t launch_fit_factor(cudaStream_t s, int K, double* qr);
cudaError_t launch_fit(const LaunchCfg& c, int K, const double* qr, const unsigned long long* hist, double* res);
// Local psi_6 into local (nullable) and each block's exact sum into partial
// [blocks_t32]; the reduction rounds each replica's total once and divides by N.
cudaError_t launch_psi6(const LaunchCfg& c, CellBufs cells, double2* local, ExactPair* partial, int* err);
cudaError_t launch_psi6_reduce(const LaunchCfg& c, const ExactPair* partial, double* res);
// Append (beta P / rho, g(2 sigma+), Re Psi_6, Im Psi_6) of every replica to
// series[len] and advance len (bounded by cap; a full series sets err bit 4).
cudaError_t launch_record(const LaunchCfg& c, const double* fit, const double* psi, double* series,
                          int64_t* len, int64_t cap, int* err);

}  // namespace hd
