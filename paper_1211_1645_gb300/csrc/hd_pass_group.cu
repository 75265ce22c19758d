// hd_pass_group.cu -- the colour pass with G threads per active cell
// (Engel et al., arXiv:1211.1645, Sec. II.B).
//
// The G lanes of a group (consecutive lanes of one warp) share one active
// cell.  Every lane draws the same generator blocks, shuffles the same
// occupants and proposes the same moves (identical inputs give identical
// results, so nothing needs broadcasting); the overlap tests against the
// eight neighbouring cells are split between the lanes, lane l taking the
// neighbours q = l, l + G, ... (q = 0..7 over the 3 x 3 stencil without its
// centre), and a trial is accepted when the warp ballot over the group shows
// every lane clear.  A move is accepted exactly when no pair overlaps, so the
// chain is the one-thread pass's, bit for bit.  Lane 0 writes the cell back
// and counts its trials.
//
// Compared with one thread per cell, a group spreads a cell's neighbour
// loads and pair tests over G lanes (shorter per-lane dependency chains,
// more loads in flight per cell) and repeats the cell's common work (the
// generator, the shuffle, the boundary test) on every lane.
#include <mutex>

#include "hd_cell.cuh"
#include "hd_kernels.h"

namespace hd {

namespace {

constexpr int kGroupMaxThreads = 512;  // cells per block x G

__device__ __forceinline__ void cp_async8_g(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_g() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Per-thread shared area of the fixed form: slots 0 and 1 of the lane's
// 8 / G neighbours, plus one pad entry (an odd stride in 8-byte words keeps
// a warp's accesses to the minimum wavefronts).
template <int G>
__host__ __device__ constexpr int group_nbr_stride() { return 2 * (8 / G) + 1; }

template <bool FIX, int CAP, int G>
__host__ __device__ constexpr size_t group_smem(int threads) {
    return (FIX ? size_t(threads) * group_nbr_stride<G>() * sizeof(int2) : 0) +
           size_t(threads) * CAP * (sizeof(P2<FIX>) + 4);
}

}  // namespace

template <bool FIX, int CAP, int NTC, bool ONE, int G>
__global__ void __launch_bounds__(kGroupMaxThreads)
k_pass_group(const Rep* __restrict__ reps, const uint16_t* __restrict__ rep_of, const Rep rep1,
             const Frame* __restrict__ table, int j, int p, const uint8_t* __restrict__ cnt, P2<FIX>* pos,
             int32_t* pid, unsigned long long* __restrict__ counters) {
    static_assert(G == 2 || G == 4 || G == 8, "a group is 2, 4 or 8 lanes of one warp");
    constexpr int NQ = 8 / G;  // neighbours per lane
    pdl_begin();
    extern __shared__ __align__(16) unsigned char s_raw[];
    int2* s_nbr = reinterpret_cast<int2*>(s_raw);
    P2<FIX>* s_crowd = reinterpret_cast<P2<FIX>*>(
        s_raw + (FIX ? size_t(blockDim.x) * group_nbr_stride<G>() * sizeof(int2) : 0));
    int32_t* s_crowd_id = reinterpret_cast<int32_t*>(s_crowd + size_t(blockDim.x) * CAP);
    const int lane = int(threadIdx.x) & (G - 1);
    const uint32_t gmask = ((1u << G) - 1u) << ((threadIdx.x & 31u) & ~uint32_t(G - 1));
    const int r = ONE ? 0 : int(rep_of[blockIdx.x]);
    const Rep rep = ONE ? rep1 : reps[r];
    const int m = rep.m, hm = rep.hm;
    const uint32_t cells_per_block = blockDim.x / G;
    const uint32_t a = uint32_t(blockIdx.x - rep.blk_act) * cells_per_block + threadIdx.x / G;
    const Frame f = table[size_t(r) * (kMaxChunk + 1) + j];
    const int col = int(f.perm >> (2 * p)) & 3;
    uint32_t att = 0, acc = 0;
    if (a < uint32_t(rep.hh)) {  // the same for every lane of a group
        const uint32_t row = div_by(a, rep.hm_mul, rep.hm_sh);
        const int cx = 2 * int(a - row * uint32_t(hm)) + (col & 1);
        const int cy = 2 * int(row) + (col >> 1);
        const uint32_t cl = uint32_t(cy) * uint32_t(m) + uint32_t(cx);  // Philox counter: row-major cell
        const uint32_t cell = rep.coff + uint32_t(col) * uint32_t(rep.hh) + a;
        // this lane's neighbours: stencil index i (0..8, centre 4 skipped) of q = lane + k G
        auto nbr_i = [&](int k) {
            const int q = lane + k * G;
            return q < 4 ? q : q + 1;
        };
        auto nbr_cell = [&](int i) {
            return rep.coff + row_part(rep, wrap_cell(cy + i / 3 - 1, m)) + col_part(rep, wrap_cell(cx + i % 3 - 1, m));
        };
        int2* mine = s_nbr + threadIdx.x * group_nbr_stride<G>();
        uint32_t nocc = 0;  // occupancy of the lane's neighbour k in bits 4k..4k+3
        if constexpr (FIX) {
            const uint32_t sm = static_cast<uint32_t>(__cvta_generic_to_shared(mine));
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const uint32_t ci = nbr_cell(nbr_i(k));
                nocc |= uint32_t(occupancy<CAP>(cnt, ci)) << (4 * k);
                cp_async8_g(sm + uint32_t(2 * k) * 8u, pos + ci);
                cp_async8_g(sm + uint32_t(2 * k + 1) * 8u, pos + rep.stride32 + ci);
            }
        }
        CellRegs<FIX, true> own;
        load_cell<FIX, true, CAP>(cnt, pos, pid, rep.stride32, cell, own);
        const int n = own.n;
        if (n > 0) {
            auto neighbours_clear = [&](const P2<FIX>& np) {
                bool ok = true;
                if constexpr (FIX) {
                    cp_async_wait_all_g();
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        const int i = nbr_i(k);
                        const int ox = i % 3 - 1, oy = i / 3 - 1;
                        const int ni = int(nocc >> (4 * k)) & 0xF;
                        ok &= pair_clear<FIX>(mine[2 * k], ox, oy, np, rep) | (ni < 1);
                        ok &= pair_clear<FIX>(mine[2 * k + 1], ox, oy, np, rep) | (ni < 2);
                        for (int s2 = kEagerSlots; s2 < ni; ++s2)
                            ok &= pair_clear<FIX>(__ldg(pos + size_t(s2) * rep.stride32 + nbr_cell(i)), ox, oy, np,
                                                  rep);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        if (!ok) continue;
                        const int i = nbr_i(k);
                        const int ox = i % 3 - 1, oy = i / 3 - 1;
                        CellRegs<FIX, false> c;
                        load_cell<FIX, false, CAP>(cnt, pos, nullptr, rep.stride32, nbr_cell(i), c);
                        for (int s2 = 0; s2 < c.n && ok; ++s2) ok = pair_clear<FIX>(c.slot(s2, pos, rep.stride32), ox, oy, np, rep);
                    }
                }
                // every lane of the group reaches this ballot together: its
                // inputs (the cell, the draws, the proposal) are the same
                return (__ballot_sync(gmask, ok) & gmask) == gmask;
            };
            if (n <= kEagerSlots) {
                P2<FIX> P[kEagerSlots] = {own.s[0], own.s[1]};
                int32_t ids[kEagerSlots] = {own.id[0], own.id[1]};
                if (n > 1) sort_by_id<FIX, kEagerSlots>(P, ids, n);
                acc = try_cell<FIX, kEagerSlots, NTC>(rep, f.sweep, cl, P, n, neighbours_clear);
                if (lane == 0) {
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
                }
            } else {
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
                // every lane has read the cell (its own copy) before lane 0 writes it
                __syncwarp(gmask);
                if (lane == 0) {
                    for (int q = 0; q < n; ++q) {
                        pos[size_t(q) * rep.stride32 + cell] = sp[q];
                        pid[size_t(q) * rep.stride32 + cell] = si[q];
                    }
                }
            }
            if (lane == 0) att = uint32_t(rep.nt);
            else acc = 0;
        }
        if constexpr (FIX) cp_async_wait_all_g();
    }
    block_count(att, acc, counters, r);
}

template <bool FIX, int CAP, int NTC, int G>
static cudaError_t pass_group_t(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                                unsigned long long* counters) {
    const int threads = c.threads * G;
    if (threads > kGroupMaxThreads) return cudaErrorInvalidConfiguration;
    const size_t smem = group_smem<FIX, CAP, G>(threads);
    static std::once_flag attr_once;
    std::call_once(attr_once, [&] {
        cudaFuncSetAttribute(k_pass_group<FIX, CAP, NTC, true, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(group_smem<FIX, CAP, G>(kGroupMaxThreads)));
        cudaFuncSetAttribute(k_pass_group<FIX, CAP, NTC, false, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(group_smem<FIX, CAP, G>(kGroupMaxThreads)));
    });
    if (c.R == 1)
        return launch_k(k_pass_group<FIX, CAP, NTC, true, G>, dim3(c.blocks_act), dim3(threads), smem, c.stream,
                        c.reps, c.rep_of_act, *c.rep0, table, j, p, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos,
                        cells.pid, counters);
    return launch_k(k_pass_group<FIX, CAP, NTC, false, G>, dim3(c.blocks_act), dim3(threads), smem, c.stream, c.reps,
                    c.rep_of_act, Rep{}, table, j, p, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos, cells.pid,
                    counters);
}

template <bool FIX, int CAP, int NTC>
static cudaError_t pass_group_g(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                                unsigned long long* counters) {
    switch (c.tpc) {
        case 2: return pass_group_t<FIX, CAP, NTC, 2>(c, table, j, p, cells, counters);
        case 4: return pass_group_t<FIX, CAP, NTC, 4>(c, table, j, p, cells, counters);
        case 8: return pass_group_t<FIX, CAP, NTC, 8>(c, table, j, p, cells, counters);
        default: return cudaErrorInvalidValue;
    }
}

template <bool FIX, int CAP>
static cudaError_t pass_group_nt(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                                 unsigned long long* counters) {
    if (c.ntc == 1) return pass_group_g<FIX, CAP, 1>(c, table, j, p, cells, counters);
    return pass_group_g<FIX, CAP, 0>(c, table, j, p, cells, counters);
}

cudaError_t launch_pass_group(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                              unsigned long long* counters) {
    if (c.fixed)
        return c.cap == 4 ? pass_group_nt<true, 4>(c, table, j, p, cells, counters)
                          : pass_group_nt<true, 9>(c, table, j, p, cells, counters);
    return c.cap == 4 ? pass_group_nt<false, 4>(c, table, j, p, cells, counters)
                      : pass_group_nt<false, 9>(c, table, j, p, cells, counters);
}

}  // namespace hd
