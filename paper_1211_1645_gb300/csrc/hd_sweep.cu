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

#include "hd_cell.cuh"
#include "hd_kernels.h"

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
          const Frame* __restrict__ table, int j,
          uint8_t* __restrict__ cnt_o, const P2<FIX>* __restrict__ pos_o, const int32_t* __restrict__ pid_o,
          uint8_t* __restrict__ cnt_n, P2<FIX>* __restrict__ pos_n, int32_t* __restrict__ pid_n,
          int* __restrict__ err) {
    pdl_begin();
    const int r = ONE ? 0 : int(rep_of[blockIdx.x]);
    const Rep rep = ONE ? rep1 : reps[r];
    const int m = rep.m;
    const uint32_t mm = uint32_t(m) * uint32_t(m);
    const uint32_t a0 = uint32_t(blockIdx.x - rep.blk_cell) * (2u * blockDim.x) + threadIdx.x;
    uint32_t c[2];
    int n[2];
    CellRegs<FIX, true> src[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t a = a0 + uint32_t(h) * blockDim.x;
        c[h] = rep.coff + a;
        n[h] = 0;
        if (a < mm) {
            load_cell<FIX, true, CAP>(cnt_o, pos_o, pid_o, rep.stride32, c[h], src[h]);
            n[h] = src[h].n;
        }
    }
    if (n[0] == 0 && n[1] == 0) return;
    const ShiftDelta<FIX> sd(table[size_t(r) * (kMaxChunk + 1) + j - 1], table[size_t(r) * (kMaxChunk + 1) + j]);
    // destination and new offsets of the first kEagerSlots disks of both cells
    uint32_t di[2][kEagerSlots];
    P2<FIX> nq[2][kEagerSlots];
    int cxy[2][2];
    // Fixed point: the shift difference has one sign per axis for the whole
    // sweep, so a coordinate can only leave its cell on that side (the same
    // integers as frame_change_fixed, with the impossible branch dropped).
    auto step_fixed = [&](int32_t d, int c, int32_t u, int& c_out, int32_t& u_out) {
        int32_t t = u + d;
        if (d >= 0) {
            if (t >= rep.W) {
                t -= rep.W;
                c = c + 1 == m ? 0 : c + 1;
            }
        } else if (t < 0) {
            t += rep.W;
            c = c == 0 ? m - 1 : c - 1;
        }
        c_out = c;
        u_out = t;
    };
    auto move = [&](const P2<FIX>& q, int cx, int cy, uint32_t& d, P2<FIX>& out) {
        int tcx, tcy;
        if constexpr (FIX) {
            step_fixed(sd.fx, cx, q.x, tcx, out.x);
            step_fixed(sd.fy, cy, q.y, tcy, out.y);
        } else {
            frame_change_fp64(sd.dx, rep.w, rep.w_below, m, cx, q.x, tcx, out.x);
            frame_change_fp64(sd.dy, rep.w, rep.w_below, m, cy, q.y, tcy, out.y);
        }
        d = rep.coff + row_part(rep, tcy) + col_part(rep, tcx);
    };
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (n[h] == 0) continue;
        cnt_o[c[h]] = 0;  // leaves this buffer zeroed for the rebuild after next
        cell_coords(rep, a0 + uint32_t(h) * blockDim.x, cxy[h][0], cxy[h][1]);
#pragma unroll
        for (int k = 0; k < kEagerSlots; ++k)
            if (k < n[h]) move(src[h].s[k], cxy[h][0], cxy[h][1], di[h][k], nq[h][k]);
    }
    int slot[2][kEagerSlots];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < kEagerSlots; ++k)
            if (k < n[h]) slot[h][k] = claim_slot(cnt_n, di[h][k]);
    bool over = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int k = 0; k < kEagerSlots; ++k) {
            if (k < n[h]) {
                if (slot[h][k] < CAP) {
                    pos_n[size_t(slot[h][k]) * rep.stride32 + di[h][k]] = nq[h][k];
                    pid_n[size_t(slot[h][k]) * rep.stride32 + di[h][k]] = src[h].id[k];
                } else {
                    over = true;
                }
            }
        }
        // crowded old cells (rare): the remaining disks one at a time
        if (n[h] > kEagerSlots)
        for (int k = kEagerSlots; k < n[h]; ++k) {
            uint32_t d;
            P2<FIX> q;
            move(src[h].slot(k, pos_o, rep.stride32), cxy[h][0], cxy[h][1], d, q);
            const int s2 = claim_slot(cnt_n, d);
            if (s2 < CAP) {
                pos_n[size_t(s2) * rep.stride32 + d] = q;
                pid_n[size_t(s2) * rep.stride32 + d] = src[h].slot_id(k, pid_o, rep.stride32);
            } else {
                over = true;
            }
        }
    }
    if (over) atomicOr(err, 1);
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
// Per-thread shared area of the fixed form: 8 neighbours x kEagerSlots slots,
// plus one pad entry so that a warp's 8-byte accesses take the minimum two
// shared-memory wavefronts.
constexpr int kNbrStride = 17;

// ... followed by each thread's area for the occupants of a crowded cell
// (more than kEagerSlots disks): CAP positions and CAP ids.
template <bool FIX, int CAP>
constexpr size_t pass_smem(int threads) {
    return (FIX ? size_t(threads) * kNbrStride * sizeof(int2) : 0) + size_t(threads) * CAP * (sizeof(P2<FIX>) + 4);
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <bool FIX, int CAP, int NTC, bool ONE>
__global__ void __launch_bounds__(256)
k_pass(const Rep* __restrict__ reps, const uint16_t* __restrict__ rep_of, const Rep rep1,
       const Frame* __restrict__ table, int j, int p,
       const uint8_t* __restrict__ cnt, P2<FIX>* pos, int32_t* pid, unsigned long long* __restrict__ counters) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char s_raw[];
    int2* s_nbr = reinterpret_cast<int2*>(s_raw);
    P2<FIX>* s_crowd = reinterpret_cast<P2<FIX>*>(s_raw + (FIX ? size_t(blockDim.x) * kNbrStride * sizeof(int2) : 0));
    int32_t* s_crowd_id = reinterpret_cast<int32_t*>(s_crowd + size_t(blockDim.x) * CAP);
    const int r = ONE ? 0 : int(rep_of[blockIdx.x]);
    const Rep rep = ONE ? rep1 : reps[r];
    const int m = rep.m, hm = rep.hm;
    const uint32_t a = uint32_t(blockIdx.x - rep.blk_act) * blockDim.x + threadIdx.x;
    const Frame f = table[size_t(r) * (kMaxChunk + 1) + j];
    const int col = int(f.perm >> (2 * p)) & 3;
    uint32_t att = 0, acc = 0;
    if (a < uint32_t(rep.hh)) {
        const uint32_t row = div_by(a, rep.hm_mul, rep.hm_sh);
        const int cx = 2 * int(a - row * uint32_t(hm)) + (col & 1);
        const int cy = 2 * int(row) + (col >> 1);
        const uint32_t cl = uint32_t(cy) * uint32_t(m) + uint32_t(cx);  // Philox counter: row-major cell
        const uint32_t cell = rep.coff + uint32_t(col) * uint32_t(rep.hh) + a;
        uint32_t xp[3], yp[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            xp[o] = col_part(rep, wrap_cell(cx + o - 1, m));
            yp[o] = rep.coff + row_part(rep, wrap_cell(cy + o - 1, m));
        }
        // Fixed form: neighbour i (0..8, centre skipped as nbr index q) has its
        // occupancy in bits 4q..4q+3 of nocc and slots 0, 1 in mine[2q], mine[2q + 1].
        int2* mine = s_nbr + threadIdx.x * kNbrStride;
        uint32_t nocc = 0;
        if constexpr (FIX) {
            const uint32_t sm = static_cast<uint32_t>(__cvta_generic_to_shared(mine));
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if (i == 4) continue;
                const int q = i < 4 ? i : i - 1;
                const uint32_t ci = yp[i / 3] + xp[i % 3];
                nocc |= uint32_t(occupancy<CAP>(cnt, ci)) << (4 * q);
                cp_async8(sm + uint32_t(2 * q) * 8u, pos + ci);
                cp_async8(sm + uint32_t(2 * q + 1) * 8u, pos + rep.stride32 + ci);
            }
        }
        CellRegs<FIX, true> own;
        load_cell<FIX, true, CAP>(cnt, pos, pid, rep.stride32, cell, own);
        const int n = own.n;
        if (n > 0) {
            auto neighbours_clear = [&](const P2<FIX>& np) {
                bool ok = true;
                if constexpr (FIX) {
                    cp_async_wait_all();  // a no-op after the first trial
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (i == 4) continue;
                        const int q = i < 4 ? i : i - 1;
                        const int ox = i % 3 - 1, oy = i / 3 - 1;
                        const int ni = int(nocc >> (4 * q)) & 0xF;
                        ok &= pair_clear<FIX>(mine[2 * q], ox, oy, np, rep) | (ni < 1);
                        ok &= pair_clear<FIX>(mine[2 * q + 1], ox, oy, np, rep) | (ni < 2);
                    }
                    // Neighbours holding more than kEagerSlots disks (rare): a
                    // nibble n >= 3 is the one whose n + 5 sets its bit 3.
                    if ((nocc + 0x55555555u) & 0x88888888u) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            if (i == 4) continue;
                            const int q = i < 4 ? i : i - 1;
                            const int ni = int(nocc >> (4 * q)) & 0xF;
                            // the cell index is recomputed here, so that no register keeps it
                            const uint32_t ci = rep.coff + row_part(rep, wrap_cell(cy + i / 3 - 1, m)) +
                                                col_part(rep, wrap_cell(cx + i % 3 - 1, m));
                            for (int k = kEagerSlots; k < ni; ++k)
                                ok &= pair_clear<FIX>(__ldg(pos + size_t(k) * rep.stride32 + ci), i % 3 - 1, i / 3 - 1,
                                                      np, rep);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (i == 4 || !ok) continue;
                        const int ox = i % 3 - 1, oy = i / 3 - 1;
                        CellRegs<FIX, false> c;
                        load_cell<FIX, false, CAP>(cnt, pos, nullptr, rep.stride32, yp[i / 3] + xp[i % 3], c);
                        for (int k = 0; k < c.n && ok; ++k) ok = pair_clear<FIX>(c.slot(k, pos, rep.stride32), ox, oy, np, rep);
                    }
                }
                return ok;
            };
            if (n <= kEagerSlots) {
                // the usual cell: its occupants in registers, in ascending id
                // (the base order of the shuffle)
                P2<FIX> P[kEagerSlots] = {own.s[0], own.s[1]};
                int32_t ids[kEagerSlots] = {own.id[0], own.id[1]};
                if (n > 1) sort_by_id<FIX, kEagerSlots>(P, ids, n);
                acc = try_cell<FIX, kEagerSlots, NTC>(rep, f.sweep, cl, P, n, neighbours_clear);
                // written back in id order (the ids too, since the sort may have permuted them)
                if (acc > 0 || n > 1) {
#pragma unroll
                    for (int q = 0; q < kEagerSlots; ++q)
                        if (q < n) pos[size_t(q) * rep.stride32 + cell] = P[q];
                }
                if (n > 1) {
#pragma unroll
                    for (int q = 0; q < kEagerSlots; ++q)
                        if (q < n) pid[size_t(q) * rep.stride32 + cell] = ids[q];
                }
            } else {
                // a crowded cell (rare): its occupants in this thread's shared
                // area, so that the registers stay sized for two
                P2<FIX>* sp = s_crowd + threadIdx.x * CAP;
                int32_t* si = s_crowd_id + threadIdx.x * CAP;
                for (int q = 0; q < n; ++q) {
                    P2<FIX> v = own.slot(q, pos, rep.stride32);
                    int32_t id = own.slot_id(q, pid, rep.stride32);
                    int k = q;
                    for (; k > 0 && si[k - 1] > id; --k) {
                        sp[k] = sp[k - 1];
                        si[k] = si[k - 1];
                    }
                    sp[k] = v;
                    si[k] = id;
                }
                acc = try_cell_in<FIX, CAP, NTC>(rep, f.sweep, cl, SmemCell<FIX>{sp}, n, neighbours_clear);
                for (int q = 0; q < n; ++q) {
                    pos[size_t(q) * rep.stride32 + cell] = sp[q];
                    pid[size_t(q) * rep.stride32 + cell] = si[q];
                }
            }
            att = uint32_t(rep.nt);
        }
        // no copy may still be landing in shared memory when the thread exits
        if constexpr (FIX) cp_async_wait_all();
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
    // per-replica block partition to follow; 1% faster than half-size blocks)
    if (c.R == 1)
        return launch_k(k_rebuild<FIX, CAP, true>, dim3((c.blocks_cell + 1) / 2), dim3(c.threads), 0, c.stream, c.reps,
                        c.rep_of_cell, *c.rep0, table, j, a.cnt, (const P2<FIX>*)a.pos, (const int32_t*)a.pid, b.cnt,
                        (P2<FIX>*)b.pos, b.pid, err);
    return launch_k(k_rebuild<FIX, CAP, false>, dim3(c.blocks_cell), dim3(c.threads / 2), 0, c.stream, c.reps,
                    c.rep_of_cell, Rep{}, table, j, a.cnt, (const P2<FIX>*)a.pos, (const int32_t*)a.pid, b.cnt,
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
    if (c.R == 1)
        return launch_k(k_pass<FIX, CAP, NTC, true>, dim3(c.blocks_act), dim3(c.threads), smem, c.stream, c.reps,
                        c.rep_of_act, *c.rep0, table, j, p, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos, cells.pid,
                        counters);
    return launch_k(k_pass<FIX, CAP, NTC, false>, dim3(c.blocks_act), dim3(c.threads), smem, c.stream, c.reps,
                    c.rep_of_act, Rep{}, table, j, p, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos, cells.pid,
                    counters);
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
