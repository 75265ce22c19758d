// hd_pass_tma.cu -- the colour pass with its neighbourhood staged in shared
// memory by bulk copies (Engel et al., arXiv:1211.1645, Sec. II.B).
//
// A block owns a segment of one half-row of the active colour plane: the
// cells (cx, cy) = (2X + px, 2R + py) with X in [X0, X0 + Bv), colour
// col = px + 2 py.  In the colour-planar layout every neighbour those cells
// read lies in one of five row segments of the other planes, each contiguous
// in memory:
//   H        plane col^1, half-row R,      half-columns [X0 - 1 + px, X0 + Bv + px)
//   Va, Vb   plane col^2, half-rows Ra, Rb, half-columns [X0, X0 + Bv)
//   Da, Db   plane col^3, half-rows Ra, Rb, half-columns as H
// with Ra = R - 1 + py and Rb = R + py (mod m/2), plus the block's own
// segment.  One thread stages the occupancies, the first two slots of every
// segment and the own cells' ids with 1-D bulk copies (TMA) on one mbarrier;
// each thread then finds its neighbours at fixed offsets from its own index.
// A half-column outside [0, m/2) (the periodic wrap at a row end) and slots
// beyond the second are read from global memory instead.
#include <mutex>

#include "hd_cell.cuh"
#include "hd_kernels.h"
#include "hd_tma.cuh"

namespace hd {

namespace {

enum { kSegOwn = 0, kSegH = 1, kSegVa = 2, kSegVb = 3, kSegDa = 4, kSegDb = 5, kSegs = 6 };

// Shared-memory capacities for a block of B threads (B a multiple of 32).
__host__ __device__ constexpr int seg_pos_cap(int B) { return B + 4; }  // one more, alignment shift, round-up
__host__ __device__ constexpr int seg_cnt_cap(int B) { return B + 32; }  // one more, shift < 16, round-up

template <bool FIX>
__host__ __device__ constexpr size_t seg_smem_bytes(int B) {
    return size_t(kSegs) * 2 * seg_pos_cap(B) * sizeof(P2<FIX>) + size_t(2) * seg_pos_cap(B) * sizeof(int32_t) +
           size_t(kSegs) * seg_cnt_cap(B) + 16;
}

constexpr uint32_t kWaitPolls = 1u << 22;  // bound of the mbarrier wait (each poll suspends briefly)
constexpr int kErrStage = 8;               // error flag: a staging copy was refused or never completed

}  // namespace

template <bool FIX, int CAP, bool NT1>
__global__ void __launch_bounds__(256)
k_pass_tma(const Rep* __restrict__ reps, int R, const Frame* __restrict__ table, int j, int p,
           const uint8_t* __restrict__ cnt, P2<FIX>* pos, int32_t* pid, unsigned long long* __restrict__ counters,
           int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int B = int(blockDim.x);
    const int pc = seg_pos_cap(B), cc = seg_cnt_cap(B);
    P2<FIX>* s_p0 = reinterpret_cast<P2<FIX>*>(s_raw);  // [kSegs][pc]
    P2<FIX>* s_p1 = s_p0 + kSegs * pc;                  // [kSegs][pc]
    int32_t* s_i0 = reinterpret_cast<int32_t*>(s_p1 + kSegs * pc);
    int32_t* s_i1 = s_i0 + pc;
    uint8_t* s_n = reinterpret_cast<uint8_t*>(s_i1 + pc);  // [kSegs][cc]
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_n + kSegs * cc);
    __shared__ int s_bad;
    __shared__ int s_poff[kSegs], s_coff[kSegs];  // staged index of half-column hc: hc + off
    __shared__ uint32_t s_base[kSegs];             // first cell index of each segment's row

    pdl_begin();
    const int r = find_rep<kGridSeg>(reps, R, blockIdx.x);
    const Rep rep = reps[r];
    const int hm = rep.hm;
    const uint32_t b = uint32_t(blockIdx.x - rep.blk_seg);
    const uint32_t row = rep.nseg > 1 ? div_by(b, rep.seg_mul, rep.seg_sh) : b;
    const int X0 = int(b - row * uint32_t(rep.nseg)) * rep.segw;
    const int Bv = min(rep.segw, hm - X0);
    const Frame f = table[size_t(r) * (kMaxChunk + 1) + j];
    const int col = int(f.perm >> (2 * p)) & 3;
    const int px = col & 1, py = col >> 1;
    const int Ra = (int(row) - 1 + py + hm) % hm, Rb = (int(row) + py) % hm;
    // Segment k: first cell index of its row and its staged half-columns [c0, c1).
    auto seg_base = [&](int k) -> uint32_t {
        const int pl = k == kSegOwn ? col : (k == kSegH ? col ^ 1 : (k == kSegVa || k == kSegVb ? col ^ 2 : col ^ 3));
        const int hr = (k == kSegVa || k == kSegDa) ? Ra : ((k == kSegVb || k == kSegDb) ? Rb : int(row));
        return rep.coff + uint32_t(pl) * uint32_t(rep.hh) + uint32_t(hr) * uint32_t(hm);
    };
    auto seg_c0 = [&](int k) { return (k == kSegOwn || k == kSegVa || k == kSegVb) ? X0 : max(X0 - 1 + px, 0); };
    auto seg_c1 = [&](int k) { return (k == kSegOwn || k == kSegVa || k == kSegVb) ? X0 + Bv : min(X0 + Bv + px, hm); };

    if (threadIdx.x == 0) {
        mbar_init(s_bar, kSegs);
        s_bad = 0;
    }
    __syncthreads();
    // Threads 0..5 each stage one segment: its slots 0 and 1 and occupancies
    // (and the own segment's ids), from 16-byte aligned starts; every slot
    // plane starts on a 16-byte boundary (the plane stride is a multiple of
    // 16 cells), so the start shift is the same for both slot planes.
    if (threadIdx.x < kSegs) {
        const int k = int(threadIdx.x);
        const uint32_t e = seg_base(k) + uint32_t(seg_c0(k));
        const int n = seg_c1(k) - seg_c0(k);
        const int ps = FIX ? int(e & 1u) : 0, cs = int(e & 15u), is = int(e & 3u);
        const uint32_t pb = uint32_t(((n + ps) * int(sizeof(P2<FIX>)) + 15) & ~15);
        const uint32_t cb = uint32_t((n + cs + 15) & ~15);
        const uint32_t ib = k == kSegOwn ? uint32_t(((n + is) * 4 + 15) & ~15) : 0u;
        const bool ok = (reinterpret_cast<uintptr_t>(cnt) & 15u) == 0 && (reinterpret_cast<uintptr_t>(pos) & 15u) == 0 &&
                        (reinterpret_cast<uintptr_t>(pid) & 15u) == 0 && (rep.stride32 & 15u) == 0 && n > 0 &&
                        pb <= uint32_t(pc) * sizeof(P2<FIX>) && cb <= uint32_t(cc) && ib <= uint32_t(pc) * 4u;
        s_poff[k] = ps - seg_c0(k);
        s_coff[k] = cs - seg_c0(k);
        s_base[k] = seg_base(k);
        if (ok) {
            mbar_arrive_expect_tx(s_bar, 2 * pb + cb + 2 * ib);
            bulk_copy_g2s(s_p0 + k * pc, pos + (e - uint32_t(ps)), pb, s_bar);
            bulk_copy_g2s(s_p1 + k * pc, pos + size_t(rep.stride32) + (e - uint32_t(ps)), pb, s_bar);
            bulk_copy_g2s(s_n + k * cc, cnt + (e - uint32_t(cs)), cb, s_bar);
            if (k == kSegOwn) {
                bulk_copy_g2s(s_i0, pid + (e - uint32_t(is)), ib, s_bar);
                bulk_copy_g2s(s_i1, pid + size_t(rep.stride32) + (e - uint32_t(is)), ib, s_bar);
            }
        } else {
            s_bad = 1;
            mbar_arrive_expect_tx(s_bar, 0);
        }
    }

    const int t = int(threadIdx.x);
    const bool live = t < Bv;
    const int X = X0 + t;
    const int cx = 2 * X + px, cy = 2 * int(row) + py;
    const uint32_t cl = uint32_t(cy) * uint32_t(rep.m) + uint32_t(cx);  // Philox counter: row-major cell
    // the generator does not depend on the staged data: draw while the copies fly
    uint4 u0 = make_uint4(0, 0, 0, 0);
    if constexpr (FIX)
        if (live) u0 = philox(f.sweep, 0u, cl, kTagTrial, rep.key0, rep.key1);

    bool staged = mbar_wait_bounded(s_bar, 0, kWaitPolls);
    if (!staged) mbar_wait_bounded(s_bar, 0, kWaitPolls);  // a second bound for copies still in flight
    staged = staged && s_bad == 0;
    if (!staged && threadIdx.x == 0) atomicOr(err, kErrStage);

    uint32_t att = 0, acc = 0;
    if (staged && live) {
        // per-segment offsets and row bases, written by the issuing threads
        // before they arrived on the barrier (read as shared-memory broadcasts)
        const int* poff = s_poff;
        const int* coff = s_coff;
        const uint32_t* sbase = s_base;
        const uint32_t cell = sbase[kSegOwn] + uint32_t(X);
        const int n = min(int(s_n[kSegOwn * cc + X + coff[kSegOwn]]), CAP);
        // neighbour i (dx, dy): segment and unwrapped half-column; occupancy
        // nibble q of nocc, staged slot index lp[q] (-1: wraps around a row
        // end, read from global memory)
        auto nbr_seg = [](int i) {
            const int dx = i % 3 - 1, dy = i / 3 - 1;
            return dy == 0 ? int(kSegH) : (dx == 0 ? (dy < 0 ? int(kSegVa) : int(kSegVb)) : (dy < 0 ? int(kSegDa) : int(kSegDb)));
        };
        auto nbr_hc = [&](int i) {
            const int dx = i % 3 - 1;
            return dx == 0 ? X : (dx < 0 ? X - 1 + px : X + px);
        };
        const bool edge = X == 0 || X == hm - 1;  // only these have a neighbour across a row end
        uint32_t nocc = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) continue;
            const int q = i < 4 ? i : i - 1;
            const int k = nbr_seg(i), hc = nbr_hc(i);
            int nn;
            if (!edge || (hc >= 0 && hc < hm)) nn = s_n[k * cc + hc + coff[k]];
            else nn = __ldg(cnt + sbase[k] + uint32_t(hc < 0 ? hc + hm : hc - hm));
            nocc |= uint32_t(min(nn, CAP)) << (4 * q);
        }
        if (n > 0) {
            P2<FIX> P[CAP];
            int32_t ids[CAP];
            const int op = X + poff[kSegOwn];
            const int oi = X + int((sbase[kSegOwn] + uint32_t(X0)) & 3u) - X0;
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                if (q == 0) {
                    P[q] = s_p0[kSegOwn * pc + op];
                    ids[q] = s_i0[oi];
                } else if (q == 1) {
                    P[q] = s_p1[kSegOwn * pc + op];
                    ids[q] = s_i1[oi];
                } else {
                    P[q] = q < n ? pos[size_t(q) * rep.stride32 + cell] : P2<FIX>{};
                    ids[q] = q < n ? pid[size_t(q) * rep.stride32 + cell] : 0;
                }
            }
            if (n > 1) sort_by_id<FIX, CAP>(P, ids, n);
            auto neighbours_clear = [&](const P2<FIX>& np) {
                bool ok = true;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (i == 4) continue;
                    const int q = i < 4 ? i : i - 1;
                    const int dx = i % 3 - 1, dy = i / 3 - 1;
                    const int k = nbr_seg(i), hc = nbr_hc(i);
                    const int nn = int(nocc >> (4 * q)) & 0xF;
                    P2<FIX> a, c;
                    if (!edge || (hc >= 0 && hc < hm)) {
                        const int lp = hc + poff[k];
                        a = s_p0[k * pc + lp];
                        c = s_p1[k * pc + lp];
                    } else {  // periodic wrap at a row end
                        const uint32_t ci = sbase[k] + uint32_t(hc < 0 ? hc + hm : hc - hm);
                        a = __ldg(pos + ci);
                        c = __ldg(pos + size_t(rep.stride32) + ci);
                    }
                    ok &= pair_clear<FIX>(a, dx, dy, np, rep) | (nn < 1);
                    ok &= pair_clear<FIX>(c, dx, dy, np, rep) | (nn < 2);
                }
                // neighbours holding more than kEagerSlots disks (rare): nibble n >= 3
                if ((nocc + 0x55555555u) & 0x88888888u) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        if (i == 4) continue;
                        const int q = i < 4 ? i : i - 1;
                        const int k = nbr_seg(i), hc = nbr_hc(i);
                        const int nn = int(nocc >> (4 * q)) & 0xF;
                        const uint32_t ci = sbase[k] + uint32_t(hc < 0 ? hc + hm : (hc >= hm ? hc - hm : hc));
                        for (int s2 = kEagerSlots; s2 < nn; ++s2)
                            ok &= pair_clear<FIX>(__ldg(pos + size_t(s2) * rep.stride32 + ci), i % 3 - 1, i / 3 - 1, np,
                                                  rep);
                    }
                }
                return ok;
            };
            acc = try_cell<FIX, CAP, NT1 ? 1 : 0>(rep, f.sweep, cl, P, n, neighbours_clear, FIX ? &u0 : nullptr);
            att = uint32_t(rep.nt);
            // written back in id order (the ids too, since the sort may have permuted them)
            if (acc > 0 || n > 1) {
#pragma unroll
                for (int q = 0; q < CAP; ++q)
                    if (q < n) pos[size_t(q) * rep.stride32 + cell] = P[q];
            }
            if (n > 1) {
#pragma unroll
                for (int q = 0; q < CAP; ++q)
                    if (q < n) pid[size_t(q) * rep.stride32 + cell] = ids[q];
            }
        }
    }
    block_count(att, acc, counters, r);
}

template <bool FIX, int CAP, bool NT1>
static cudaError_t pass_tma_t(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                              unsigned long long* counters, int* err) {
    const size_t smem = seg_smem_bytes<FIX>(c.threads);
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_pass_tma<FIX, CAP, NT1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(seg_smem_bytes<FIX>(256)));
    });
    return launch_k(k_pass_tma<FIX, CAP, NT1>, dim3(c.blocks_seg), dim3(c.threads), smem, c.stream, c.reps, c.R,
                    table, j, p, (const uint8_t*)cells.cnt, (P2<FIX>*)cells.pos, cells.pid, counters, err);
}

template <bool FIX, int CAP>
static cudaError_t pass_tma_nt(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                               unsigned long long* counters, int* err) {
    return c.ntc == 1 ? pass_tma_t<FIX, CAP, true>(c, table, j, p, cells, counters, err)
                 : pass_tma_t<FIX, CAP, false>(c, table, j, p, cells, counters, err);
}

cudaError_t launch_pass_tma(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                            unsigned long long* counters, int* err) {
    if (c.fixed)
        return c.cap == 4 ? pass_tma_nt<true, 4>(c, table, j, p, cells, counters, err)
                          : pass_tma_nt<true, 9>(c, table, j, p, cells, counters, err);
    return c.cap == 4 ? pass_tma_nt<false, 4>(c, table, j, p, cells, counters, err)
                      : pass_tma_nt<false, 9>(c, table, j, p, cells, counters, err);
}

}  // namespace hd
