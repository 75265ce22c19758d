// hd_sweep.cu -- the checkerboard sweep of massively parallel local Monte
// Carlo for hard disks (Engel et al., arXiv:1211.1645, Sec. II.B), split into
// one launch per rebuild and one per colour pass.
//
// Layout (per replica, concatenated over replicas): an m x m grid of cells in
// the current shifted frame, stored colour-planar (see cell_index).  Cell c
// holds cnt[c] <= CAP disks; occupant k has its offset inside the cell in
// pos[k * stride + c] (double2 in [0,w)^2, or int2 in [0,W)^2 in units of
// 2^-24 sigma) and its id in pid[k * stride + c].  Cell-local coordinates are
// the paper's remedy for cancellation at large L (Sec. II.B).  Slots at or
// beyond the occupancy hold stale data.
//
// One sweep = k_rebuild (move every disk into the new shifted frame; each old
// cell scatters its disks) followed by four k_pass launches, one per colour
// in the sweep's random order.  Cells of one colour are never neighbours, so
// every thread of a pass owns its cell outright and only reads the
// (unchanging) cells of the other colours.
#include <mutex>

#include "hd_kernels.h"
#include "hd_sweep_cell.cuh"

namespace hd {

__global__ void k_draws(const Rep* __restrict__ reps, int R, Frame* __restrict__ table,
                        Frame* __restrict__ cur, uint64_t* __restrict__ sweep_ctr, int nchunk) {
    pdl_begin();
    // one block per replica, one thread per sweep of the chunk: every sweep's
    // draws come from its own generator block
    const int r = blockIdx.x;
    const Rep& rep = reps[r];
    Frame* t = table + size_t(r) * (kMaxChunk + 1);
    const uint64_t s0 = sweep_ctr[r];
    if (threadIdx.x == 0) t[0] = cur[r];
    for (int j = 1 + int(threadIdx.x); j <= nchunk; j += int(blockDim.x)) {
        Frame f;
        const uint32_t s = uint32_t(s0 + uint64_t(j - 1));
        const uint4 a = philox(s, 0u, 0u, kTagSweep, rep.key0, rep.key1);
        f.sx = __dmul_rn(double(a.x) * 0x1p-32, rep.w);
        f.sy = __dmul_rn(double(a.y) * 0x1p-32, rep.w);
        f.Sx = int32_t(__umulhi(a.x, uint32_t(rep.W)));
        f.Sy = int32_t(__umulhi(a.y, uint32_t(rep.W)));
        f.sweep = s;
        // rank in [0, 24) -> permutation of the four colours in lexicographic order
        uint32_t rank = bounded(a.z, 24u);
        uint32_t avail = 0x3210u;  // remaining colours, one nibble each, ascending
        uint32_t perm = 0;
        const uint32_t radix[3] = {6u, 2u, 1u};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const uint32_t d = rank / radix[p];
            rank %= radix[p];
            perm |= ((avail >> (4 * d)) & 0xFu) << (2 * p);
            const uint32_t low = avail & ((1u << (4 * d)) - 1u);
            const uint32_t high = avail >> (4 * (d + 1));
            avail = low | (high << (4 * d));
        }
        perm |= (avail & 0xFu) << 6;
        f.perm = perm;
        t[j] = f;
    }
    // every thread has read sweep_ctr[r], thread 0 has read cur[r], and the
    // chunk's last frame is visible to the block
    __syncthreads();
    if (threadIdx.x == 0) {
        cur[r] = t[nchunk];
        sweep_ctr[r] = s0 + uint64_t(nchunk);
    }
}

// ---------------------------------------------------------------------------
// Rebuild by scatter: one thread per old cell moves each of its disks into
// the new shifted frame once (the per-disk frame change of the paper's random
// grid shift) and claims a slot in the destination cell with a byte-lane
// atomic.  Slot order inside a new cell is therefore arbitrary; the colour
// pass orders a cell's occupants by id before its shuffle, so the chain is
// unaffected.  Each thread also clears the occupancy of its old cell, which
// leaves that buffer zeroed for the rebuild after next (the two cell buffers
// alternate), so no separate clearing launch is needed.
// With d = old shift - new shift in (-w, w), a coordinate u + d lies in
// (-w, 2w), so a disk changes cell by at most one per axis.
// ---------------------------------------------------------------------------
// A thread handles two old cells, blockDim apart, and issues the loads of
// both and then the slot claims of both before it waits on any, so the two
// latency chains (loads, then claims, then stores) overlap.
// ONE: a single replica, whose constants come by value in rep1 (kernel
// parameters, read as constant operands) instead of from reps; otherwise the
// block's replica comes from rep_of (one entry per block).
template <bool FIX, int CAP, bool ONE>
__global__ void __launch_bounds__(256)
k_rebuild(const Rep* __restrict__ reps, const uint16_t* __restrict__ rep_of, const Rep rep1,
          const Frame* __restrict__ table, int j, uint32_t x_lo, uint32_t x_span,
          uint8_t* __restrict__ cnt_o, const P2<FIX>* __restrict__ pos_o, const int32_t* __restrict__ pid_o,
          uint8_t* __restrict__ cnt_n, P2<FIX>* __restrict__ pos_n, int32_t* __restrict__ pid_n,
          int* __restrict__ err) {
    pdl_begin();
    const int r = ONE ? 0 : int(rep_of[blockIdx.x]);
    const Rep rep = ONE ? rep1 : reps[r];
    uint32_t a[2];
    bool live[2];
    if (ONE && x_span != 0u) {
        // one strip: entries x_lo + x of colour planes 2y and 2y + 1
        const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
        a[0] = 2u * blockIdx.y * uint32_t(rep.hh) + x_lo + x;
        a[1] = a[0] + uint32_t(rep.hh);
        live[0] = live[1] = x < x_span;
    } else {
        const uint32_t mm = uint32_t(rep.m) * uint32_t(rep.m);
        const uint32_t a0 = uint32_t(blockIdx.x - rep.blk_cell) * (2u * blockDim.x) + threadIdx.x;
        a[0] = a0;
        a[1] = a0 + blockDim.x;
        live[0] = a[0] < mm;
        live[1] = a[1] < mm;
    }
    if (rebuild_pair<FIX, CAP, false>(rep, table + size_t(r) * (kMaxChunk + 1), j, a, live, cnt_o, pos_o, pid_o,
                                      cnt_n, pos_n, pid_n))
        atomicOr(err, 1);
}

// ---------------------------------------------------------------------------
// One colour pass: every active cell shuffles its occupants and makes nt
// serial trial moves (try_cell).  The loads of the cell and its eight
// neighbours are issued before the draws are made, so the generator's
// arithmetic overlaps their latency.  In the fixed-point form the first two
// slots of each neighbour are copied into the thread's own shared-memory
// area with cp.async, which holds no register while the copy is in flight;
// that halves the registers of the kernel and doubles the resident warps
// that hide the latency.  (The FP64 form, whose slots are twice as wide,
// loads one neighbour at a time inside the test.)
// ---------------------------------------------------------------------------
template <bool FIX, int CAP, int NTC, bool ONE>
__global__ void __launch_bounds__(256)
k_pass(const Rep* __restrict__ reps, const uint16_t* __restrict__ rep_of, const Rep rep1,
       const Frame* __restrict__ table, int j, int p, uint32_t a_lo, uint32_t a_hi,
       const uint8_t* __restrict__ cnt, P2<FIX>* pos, int32_t* pid, unsigned long long* __restrict__ counters) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char s_raw[];
    P2<FIX>* s_crowd = reinterpret_cast<P2<FIX>*>(s_raw + size_t(blockDim.x) * nbr_bytes_per_thread<FIX>());
    int32_t* s_crowd_id = reinterpret_cast<int32_t*>(s_crowd + size_t(blockDim.x) * CAP);
    const int r = ONE ? 0 : int(rep_of[blockIdx.x]);
    const Rep rep = ONE ? rep1 : reps[r];
    const uint32_t a = a_lo + uint32_t(blockIdx.x - rep.blk_act) * blockDim.x + threadIdx.x;
    const Frame f = table[size_t(r) * (kMaxChunk + 1) + j];
    const int col = int(f.perm >> (2 * p)) & 3;
    uint32_t att = 0, acc = 0;
    if (a < a_hi && a < uint32_t(rep.hh)) {
        pass_cell<FIX, CAP, NTC, false>(rep, f, col, a, cnt, pos, pid, nbr_area<FIX>(s_raw),
                                        s_crowd + threadIdx.x * CAP, s_crowd_id + threadIdx.x * CAP, att, acc);
    }
    block_count(att, acc, counters, r);
}

// ---------------------------------------------------------------------------
// Global positions from the cell frame: X = (cx w + u) + shift, wrapped once.
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_positions(const Rep* __restrict__ reps, int R, const Frame* __restrict__ cur, const uint8_t* __restrict__ cnt,
            const P2<FIX>* __restrict__ pos, const int32_t* __restrict__ pid, double* __restrict__ xy) {
    pdl_begin();
    const int r = find_rep<kGridCell>(reps, R, blockIdx.x);
    const Rep rep = reps[r];
    const int m = rep.m;
    const uint32_t a = uint32_t(blockIdx.x - rep.blk_cell) * blockDim.x + threadIdx.x;
    if (a >= uint32_t(m) * uint32_t(m)) return;
    int cx, cy;
    cell_coords(rep, a, cx, cy);
    const Frame f = cur[r];
    const uint32_t cell = rep.coff + a;
    const int n = min(int(cnt[cell]), CAP);
    for (int k = 0; k < n; ++k) {
        const P2<FIX> q = pos[size_t(k) * rep.stride32 + cell];
        const int64_t id = rep.id_off + pid[size_t(k) * rep.stride32 + cell];
        double X, Y;
        if constexpr (FIX) {
            int64_t IX = int64_t(cx) * rep.W + q.x + f.Sx;
            int64_t IY = int64_t(cy) * rep.W + q.y + f.Sy;
            if (IX >= rep.LF) IX -= rep.LF;
            if (IY >= rep.LF) IY -= rep.LF;
            X = double(IX) * 0x1p-24;
            Y = double(IY) * 0x1p-24;
        } else {
            X = __dadd_rn(__dadd_rn(__dmul_rn(double(cx), rep.w), q.x), f.sx);
            Y = __dadd_rn(__dadd_rn(__dmul_rn(double(cy), rep.w), q.y), f.sy);
            if (X >= rep.L) X = __dsub_rn(X, rep.L);
            if (Y >= rep.L) Y = __dsub_rn(Y, rep.L);
        }
        xy[2 * id] = __dmul_rn(X, rep.sigma);
        xy[2 * id + 1] = __dmul_rn(Y, rep.sigma);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_draws(const LaunchCfg& c, Frame* table, Frame* cur, uint64_t* sweep_ctr, int nchunk) {
    return launch_k(k_draws, dim3(c.R), dim3(128), 0, c.stream, c.reps, c.R, table, cur, sweep_ctr, nchunk);
}

template <bool FIX, int CAP>
static cudaError_t rebuild_t(const LaunchCfg& c, const Frame* table, int j, CellBufs a, CellBufs b, int* err) {
    // one replica: blocks of `threads` threads over 2 threads cells each (no
    // per-replica block partition to follow; 1% faster than half-size blocks);
    // one strip: a thread per planar entry of the band range, its cells in two
    // colour planes (grid y picks the pair)
    if (c.R == 1) {
        const dim3 grid = c.band_span ? dim3((c.band_span + uint32_t(c.threads) - 1) / uint32_t(c.threads), 2)
                                      : dim3((c.blocks_cell + 1) / 2);
        return launch_k(k_rebuild<FIX, CAP, true>, grid, dim3(c.threads), 0, c.stream, c.reps, c.rep_of_cell, *c.rep0,
                        table, j, c.band_lo, c.band_span, a.cnt, (const P2<FIX>*)a.pos, (const int32_t*)a.pid, b.cnt,
                        (P2<FIX>*)b.pos, b.pid, err);
    }
    return launch_k(k_rebuild<FIX, CAP, false>, dim3(c.blocks_cell), dim3(c.threads / 2), 0, c.stream, c.reps,
                    c.rep_of_cell, Rep{}, table, j, 0u, 0u, a.cnt, (const P2<FIX>*)a.pos, (const int32_t*)a.pid, b.cnt,
                    (P2<FIX>*)b.pos, b.pid, err);
}

cudaError_t launch_rebuild(const LaunchCfg& c, const Frame* table, int j, CellBufs from, CellBufs to, int* err) {
    if (c.fixed) return c.cap == 4 ? rebuild_t<true, 4>(c, table, j, from, to, err) : rebuild_t<true, 9>(c, table, j, from, to, err);
    return c.cap == 4 ? rebuild_t<false, 4>(c, table, j, from, to, err) : rebuild_t<false, 9>(c, table, j, from, to, err);
}

template <bool FIX, int CAP, int NTC>
static cudaError_t pass_t(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                          unsigned long long* counters) {
    const size_t smem = pass_smem<FIX, CAP>(c.threads);
    static std::once_flag attr_once;
    std::call_once(attr_once, [&] {
        cudaFuncSetAttribute(k_pass<FIX, CAP, NTC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(pass_smem<FIX, CAP>(256)));
        cudaFuncSetAttribute(k_pass<FIX, CAP, NTC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(pass_smem<FIX, CAP>(256)));
    });
    if (c.R == 1) {
        // a strip covers its active-cell range; the whole plane otherwise
        const int blocks = c.act_hi != ~0u ? int((c.act_hi - c.act_lo + uint32_t(c.threads) - 1) / uint32_t(c.threads))
                                          : c.blocks_act;
        return launch_k(k_pass<FIX, CAP, NTC, true>, dim3(blocks), dim3(c.threads), smem, c.stream, c.reps,
                        c.rep_of_act, *c.rep0, table, j, p, c.act_lo, c.act_hi, (const uint8_t*)cells.cnt,
                        (P2<FIX>*)cells.pos, cells.pid, counters);
    }
    return launch_k(k_pass<FIX, CAP, NTC, false>, dim3(c.blocks_act), dim3(c.threads), smem, c.stream, c.reps,
                    c.rep_of_act, Rep{}, table, j, p, 0u, ~0u, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos,
                    cells.pid, counters);
}

template <bool FIX, int CAP>
static cudaError_t pass_nt(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                           unsigned long long* counters) {
    // a compile-time count of two measured slower than the run-time loop, so only one is specialised
    if (c.ntc == 1) return pass_t<FIX, CAP, 1>(c, table, j, p, cells, counters);
    return pass_t<FIX, CAP, 0>(c, table, j, p, cells, counters);
}

cudaError_t launch_pass(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                        unsigned long long* counters) {
    if (c.tpc > 1) return launch_pass_group(c, table, j, p, cells, counters);
    if (c.fixed) return c.cap == 4 ? pass_nt<true, 4>(c, table, j, p, cells, counters) : pass_nt<true, 9>(c, table, j, p, cells, counters);
    return c.cap == 4 ? pass_nt<false, 4>(c, table, j, p, cells, counters) : pass_nt<false, 9>(c, table, j, p, cells, counters);
}

// Resident blocks per SM of the one-replica colour pass (split kernel).
template <bool FIX, int CAP, int NTC>
static cudaError_t pass_occupancy_t(const LaunchCfg& c, int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_pass<FIX, CAP, NTC, true>, c.threads,
                                                         pass_smem<FIX, CAP>(c.threads));
}

cudaError_t pass_blocks_per_sm(const LaunchCfg& c, int* blocks) {
    if (c.fixed) {
        if (c.cap == 4) return c.ntc == 1 ? pass_occupancy_t<true, 4, 1>(c, blocks) : pass_occupancy_t<true, 4, 0>(c, blocks);
        return c.ntc == 1 ? pass_occupancy_t<true, 9, 1>(c, blocks) : pass_occupancy_t<true, 9, 0>(c, blocks);
    }
    if (c.cap == 4) return c.ntc == 1 ? pass_occupancy_t<false, 4, 1>(c, blocks) : pass_occupancy_t<false, 4, 0>(c, blocks);
    return c.ntc == 1 ? pass_occupancy_t<false, 9, 1>(c, blocks) : pass_occupancy_t<false, 9, 0>(c, blocks);
}

template <bool FIX, int CAP>
static cudaError_t positions_t(const LaunchCfg& c, const Frame* cur, CellBufs cells, double* xy) {
    return launch_k(k_positions<FIX, CAP>, dim3(c.blocks_cell), dim3(c.threads), 0, c.stream, c.reps, c.R, cur,
                    (const uint8_t*)cells.cnt, (const P2<FIX>*)cells.pos, (const int32_t*)cells.pid, xy);
}

cudaError_t launch_positions(const LaunchCfg& c, const Frame* cur, CellBufs cells, double* xy) {
    if (c.fixed) return c.cap == 4 ? positions_t<true, 4>(c, cur, cells, xy) : positions_t<true, 9>(c, cur, cells, xy);
    return c.cap == 4 ? positions_t<false, 4>(c, cur, cells, xy) : positions_t<false, 9>(c, cur, cells, xy);
}

}  // namespace hd
