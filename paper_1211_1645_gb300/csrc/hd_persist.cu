// hd_persist.cu -- many checkerboard sweeps in one launch (Engel et al.,
// arXiv:1211.1645, Sec. II.B), with the work of successive rebuilds and
// colour passes overlapping as a wavefront instead of being separated by
// launch boundaries.
//
// Work items.  A sweep is five phases: the rebuild into the sweep's shifted
// frame, then the four colour passes in the sweep's order.  A band b of a
// replica is cell rows 2b and 2b + 1, i.e. half-row b of each colour plane,
// split into nseg segments of segw half-columns (the segment grid of the
// replica).  Item (phase k, band b, segment s) is: for a pass, the active
// cells of that segment; for a rebuild, the old cells of that segment in all
// four planes.  Item t of the launch is phase k = t / NI, entry t mod NI of
// the segment grid over all replicas (NI entries), whose band position p is
// band b = (p + k) mod hm: each phase starts one band further on, so that the
// first items of phase k + 1 depend on the first items of phase k (with the
// same order in every phase, band 0 of phase k + 1 would wait for band
// hm - 1, the last item of phase k, and the phases would not overlap).
//
// Dependencies.  An item of band b reads and writes only cell rows 2b - 1 ..
// 2b + 2 (a pass reads the eight neighbours of its cells, a rebuild moves a
// disk by at most one cell), and items of one phase never conflict (cells of
// one colour are not neighbours; rebuild slots are claimed atomically).  So
// item (k, b, s) may start once phase k - 1 is complete in bands b - 1, b and
// b + 1 (periodically), which is the same as the sequential order of phases
// for every cell it touches: the chain is bit-identical to the split kernels'.
// progress[band] counts the band's completed items; phase k - 1 is complete
// when it reaches k * nseg.  A block publishes its item with a release add
// after all its threads are done, and waits with acquire loads.
//
// Scheduling.  Blocks take items in ticket order from one counter, so an
// item only ever waits on items with lower tickets, which blocks that are
// already running hold: no block waits on a block that has not started, and
// the launch needs no co-residency guarantee.  A block fetches its next ticket
// while it waits on the current item's dependencies.
//
// Bounded waits.  Every wait gives up after `polls` polls (kPersistPolls,
// seconds): the block then sets error bit 16 (reported as HD_ERR_TIMEOUT) and
// the abort word, and every block stops at its next wait or item.  A test
// hook (stall_band >= 0) withholds the publication of the first item of that
// band, with a short poll bound, so that the waits on it give up.
//
// Loads.  Cells are read with coherent loads (ld_cell<true>: cached in L2
// only) and the fixed form's neighbour slots are staged with cp.async (a weak
// load in the memory model), all after the acquire that orders them behind
// the items they depend on.
#include <mutex>

#include "hd_kernels.h"
#include "hd_sweep_cell.cuh"

namespace hd {

namespace {

constexpr uint32_t kPersistPolls = 1u << 24;
constexpr int kErrPersist = 16;

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_gpu(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Wait until progress[b0 + (b - 1, b, b + 1 mod hm)] >= need; false when the
// wait gives up (bit 16 of err and the abort word set) or another block
// aborted.  Called by one thread.
__device__ bool wait_bands(uint32_t* sync, int band0, int hm, int b, uint32_t need, uint32_t polls, int* err) {
    const uint32_t* prog = sync + 2 + band0;
    const int bl = b == 0 ? hm - 1 : b - 1, br = b + 1 == hm ? 0 : b + 1;
    bool okl = false, okc = false, okr = false;
    for (uint32_t i = 0; i < polls; ++i) {
        okl = okl || ld_acquire_gpu(prog + bl) >= need;
        okc = okc || ld_acquire_gpu(prog + b) >= need;
        okr = okr || ld_acquire_gpu(prog + br) >= need;
        if (okl && okc && okr) return true;
        if (ld_acquire_gpu(sync + 1) != 0u) return false;
        __nanosleep(64);
    }
    atomicOr(err, kErrPersist);
    atomicExch(sync + 1, 1u);
    return false;
}

}  // namespace

// Registers are capped at 64 (four blocks of 256 threads, eight of 128, per
// SM): the per-item synchronisation is latency that only more resident warps
// hide.  Measured at N = 1M, 100 sweeps per launch: 9.6 ms uncapped (122
// registers), 7.2 ms at 80, 6.6 ms at 64 (some spills), against 4.4 ms for
// the split kernels.
template <bool FIX, int CAP, int NTC, bool ONE>
__global__ void __launch_bounds__(256, 4)
k_sweep_persist(const Rep* __restrict__ reps, int R, const Rep rep1, const Frame* __restrict__ table, int nsweeps,
                uint32_t NI, CellBufs g0, CellBufs g1, unsigned long long* __restrict__ counters,
                int* __restrict__ err, uint32_t* sync, uint32_t polls, int stall_band) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned char s_raw[];
    P2<FIX>* s_crowd = reinterpret_cast<P2<FIX>*>(s_raw + size_t(blockDim.x) * nbr_bytes_per_thread<FIX>());
    int32_t* s_crowd_id = reinterpret_cast<int32_t*>(s_crowd + size_t(blockDim.x) * CAP);
    int2* mine = nbr_area<FIX>(s_raw);
    P2<FIX>* sp = s_crowd + threadIdx.x * CAP;
    int32_t* si = s_crowd_id + threadIdx.x * CAP;
    __shared__ uint32_t s_first, s_next;
    __shared__ int s_go;

    const uint32_t total = 5u * uint32_t(nsweeps) * NI;
    if (threadIdx.x == 0) s_first = atomicAdd(sync, 1u);
    __syncthreads();
    uint32_t t = s_first;
    uint32_t att = 0, acc = 0;
    int cur_r = -1;
    bool over = false;
    while (t < total) {
        const uint32_t k = t / NI, idx = t - k * NI;
        const int r = ONE ? 0 : find_rep<kGridSeg>(reps, R, int(idx));
        const Rep rep = ONE ? rep1 : reps[r];
        const uint32_t loc = idx - uint32_t(rep.blk_seg);
        const uint32_t nseg = uint32_t(rep.nseg);
        const uint32_t bp = nseg > 1 ? div_by(loc, rep.seg_mul, rep.seg_sh) : loc;
        const int X0 = int(loc - bp * nseg) * rep.segw;
        const uint32_t b = (bp + k) % uint32_t(rep.hm);
        const int Bv = min(rep.segw, rep.hm - X0);
        if (!ONE && r != cur_r) {  // the trial counts go to the replica of the items that made them
            if (cur_r >= 0) block_count(att, acc, counters, cur_r);
            att = acc = 0;
            cur_r = r;
        }
        if (threadIdx.x == 0) {
            s_next = atomicAdd(sync, 1u);  // in flight while the dependencies are polled
            s_go = wait_bands(sync, rep.band0, rep.hm, int(b), k * nseg, polls, err) ? 1 : 0;
        }
        __syncthreads();
        const bool go = s_go != 0;
        const uint32_t next = s_next;
        if (!go) break;
        const uint32_t i = k / 5u, ph = k - 5u * i;
        const int j = int(i) + 1;  // sweep i of the launch uses table entries j - 1 and j
        const CellBufs from = ((i & 1u) == 0u) ? g0 : g1;
        const CellBufs to = ((i & 1u) == 0u) ? g1 : g0;
        const Frame* tab = table + size_t(ONE ? 0 : r) * (kMaxChunk + 1);
        const int x = X0 + int(threadIdx.x);
        if (ph == 0u) {
            if (x < X0 + Bv) {
                const uint32_t base = b * uint32_t(rep.hm) + uint32_t(x);
                const bool live[2] = {true, true};
#pragma unroll 1
                for (uint32_t pp = 0; pp < 4u; pp += 2u) {
                    const uint32_t a[2] = {pp * uint32_t(rep.hh) + base, (pp + 1u) * uint32_t(rep.hh) + base};
                    over |= rebuild_pair<FIX, CAP, true>(rep, tab, j, a, live, from.cnt, (const P2<FIX>*)from.pos,
                                                         from.pid, to.cnt, (P2<FIX>*)to.pos, to.pid);
                }
            }
        } else {
            const Frame f = tab[j];
            const int col = int(f.perm >> (2u * (ph - 1u))) & 3;
            if (x < X0 + Bv)
                pass_cell<FIX, CAP, NTC, true>(rep, f, col, b * uint32_t(rep.hm) + uint32_t(x), to.cnt,
                                               (P2<FIX>*)to.pos, to.pid, mine, sp, si, att, acc);
        }
        __syncthreads();  // every thread's writes of the item precede the release below
        if (threadIdx.x == 0 && !(k == 0u && int(rep.band0 + b) == stall_band && X0 == 0))
            red_release_add_gpu(sync + 2 + rep.band0 + b, 1u);  // orders the block's writes (cumulative via the barrier)
        t = next;
    }
    if (over) atomicOr(err, 1);
    if (ONE) block_count(att, acc, counters, 0);
    else if (cur_r >= 0) block_count(att, acc, counters, cur_r);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

namespace {

template <bool FIX, int CAP, int NTC>
auto persist_kernel(const LaunchCfg& c) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_sweep_persist<FIX, CAP, NTC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(pass_smem<FIX, CAP>(256)));
        cudaFuncSetAttribute(k_sweep_persist<FIX, CAP, NTC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(pass_smem<FIX, CAP>(256)));
    });
    return c.R == 1 ? k_sweep_persist<FIX, CAP, NTC, true> : k_sweep_persist<FIX, CAP, NTC, false>;
}

template <bool FIX, int CAP, int NTC>
cudaError_t persist_t(const LaunchCfg& c, const Frame* table, int nsweeps, CellBufs a, CellBufs b,
                      unsigned long long* counters, int* err, uint32_t* sync) {
    if (c.persist_blocks < 1) return cudaErrorInvalidConfiguration;
    const uint32_t NI = uint32_t(c.blocks_seg);
    const int blocks = int(std::min<uint64_t>(uint64_t(c.persist_blocks), 5ull * uint64_t(nsweeps) * NI));
    return launch_k(persist_kernel<FIX, CAP, NTC>(c), dim3(blocks), dim3(c.threads), pass_smem<FIX, CAP>(c.threads),
                    c.stream, c.reps, c.R, c.R == 1 ? *c.rep0 : Rep{}, table, nsweeps, NI, a, b, counters, err, sync,
                    c.persist_stall ? 1u << 12 : kPersistPolls, c.persist_stall ? 0 : -1);
}

template <bool FIX, int CAP>
cudaError_t persist_nt(const LaunchCfg& c, const Frame* table, int nsweeps, CellBufs a, CellBufs b,
                       unsigned long long* counters, int* err, uint32_t* sync) {
    if (c.ntc == 1) return persist_t<FIX, CAP, 1>(c, table, nsweeps, a, b, counters, err, sync);
    return persist_t<FIX, CAP, 0>(c, table, nsweeps, a, b, counters, err, sync);
}

template <bool FIX, int CAP, int NTC>
cudaError_t persist_grid_t(const LaunchCfg& c, int* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel<FIX, CAP, NTC>(c), c.threads,
                                                          pass_smem<FIX, CAP>(c.threads));
    *blocks = sms * std::max(per_sm, 1);
    return e;
}

}  // namespace

size_t persist_sync_words(int total_bands) { return size_t(2 + total_bands); }

// As many blocks as are resident at once: more would only wait for a free
// slot and then find every ticket taken.
cudaError_t persist_grid(const LaunchCfg& c, int* blocks) {
    if (c.fixed) {
        if (c.cap == 4) return c.ntc == 1 ? persist_grid_t<true, 4, 1>(c, blocks) : persist_grid_t<true, 4, 0>(c, blocks);
        return c.ntc == 1 ? persist_grid_t<true, 9, 1>(c, blocks) : persist_grid_t<true, 9, 0>(c, blocks);
    }
    if (c.cap == 4) return c.ntc == 1 ? persist_grid_t<false, 4, 1>(c, blocks) : persist_grid_t<false, 4, 0>(c, blocks);
    return c.ntc == 1 ? persist_grid_t<false, 9, 1>(c, blocks) : persist_grid_t<false, 9, 0>(c, blocks);
}

cudaError_t launch_sweeps_persist(const LaunchCfg& c, const Frame* table, int nsweeps, CellBufs from, CellBufs to,
                                  unsigned long long* counters, int* err, uint32_t* sync, int total_bands) {
    if (nsweeps < 1 || nsweeps > kMaxChunk) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sync, 0, persist_sync_words(total_bands) * sizeof(uint32_t), c.stream);
    if (e != cudaSuccess) return e;
    if (c.fixed)
        return c.cap == 4 ? persist_nt<true, 4>(c, table, nsweeps, from, to, counters, err, sync)
                          : persist_nt<true, 9>(c, table, nsweeps, from, to, counters, err, sync);
    return c.cap == 4 ? persist_nt<false, 4>(c, table, nsweeps, from, to, counters, err, sync)
                      : persist_nt<false, 9>(c, table, nsweeps, from, to, counters, err, sync);
}

}  // namespace hd
