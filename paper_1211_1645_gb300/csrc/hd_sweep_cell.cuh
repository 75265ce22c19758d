// hd_sweep_cell.cuh -- the per-cell bodies of the checkerboard sweep's
// rebuild and colour pass (Engel et al., arXiv:1211.1645, Sec. II.B), shared
// by the split kernels (one launch per rebuild and per colour pass, loads
// through the read-only path) and the persistent sweep kernel (many sweeps
// per launch, coherent loads; see ld_cell).
#pragma once

#include "hd_cell.cuh"

namespace hd {

// Shared staging of the neighbours' slots.  Fixed form: per thread 8
// neighbours x kEagerSlots slots plus one pad entry (17 int2, thread-major),
// so that a warp's 8-byte accesses take the minimum two shared-memory
// wavefronts.  FP64 form: slot 0 of the 8 neighbours (16 bytes each), stored
// slot-major (entry q of thread t at q * blockDim + t), so that consecutive
// threads' 16-byte entries are consecutive and need no pad.
constexpr int kNbrStride = 17;

template <bool FIX>
__host__ __device__ constexpr size_t nbr_bytes_per_thread() {
    return FIX ? size_t(kNbrStride) * sizeof(int2) : size_t(8) * sizeof(double2);
}

// This thread's staging pointer (FP64: its entry of slot-major row 0).
template <bool FIX>
__device__ __forceinline__ int2* nbr_area(unsigned char* s_raw) {
    if constexpr (FIX) return reinterpret_cast<int2*>(s_raw) + size_t(threadIdx.x) * kNbrStride;
    else return reinterpret_cast<int2*>(reinterpret_cast<double2*>(s_raw) + threadIdx.x);
}

// ... followed by each thread's area for the occupants of a crowded cell
// (more than kEagerSlots disks): CAP positions and CAP ids.
template <bool FIX, int CAP>
constexpr size_t pass_smem(int threads) {
    return size_t(threads) * nbr_bytes_per_thread<FIX>() + size_t(threads) * CAP * (sizeof(P2<FIX>) + 4);
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}


// Rebuild by scatter of two old cells of one replica (replica-local planar
// indices a[0], a[1]; live[h] false skips one): each disk is moved into the
// frame of sweep j (shift difference of tab[j - 1] and tab[j]) and claims a
// slot of its new cell; the old cells' occupancies are cleared.  The loads of
// both cells and then the slot claims of both are issued before either is
// waited on.  Returns true if a new cell overflowed.
template <bool FIX, int CAP, bool COH>
__device__ __forceinline__ bool rebuild_pair(const Rep& rep, const Frame* __restrict__ tab, int j, const uint32_t (&a)[2],
                                             const bool (&live)[2], uint8_t* __restrict__ cnt_o,
                                             const P2<FIX>* __restrict__ pos_o, const int32_t* __restrict__ pid_o,
                                             uint8_t* __restrict__ cnt_n, P2<FIX>* __restrict__ pos_n,
                                             int32_t* __restrict__ pid_n) {
    const int m = rep.m;
    uint32_t c[2];
    int n[2];
    CellRegs<FIX, true> src[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        c[h] = rep.coff + a[h];
        n[h] = 0;
        if (live[h]) {
            load_cell<FIX, true, CAP, COH>(cnt_o, pos_o, pid_o, rep.stride32, c[h], src[h]);
            n[h] = src[h].n;
        }
    }
    if (n[0] == 0 && n[1] == 0) return false;
    const ShiftDelta<FIX> sd(tab[j - 1], tab[j]);
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
        cell_coords(rep, a[h], cxy[h][0], cxy[h][1]);
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
            move(src[h].template slot<COH>(k, pos_o, rep.stride32), cxy[h][0], cxy[h][1], d, q);
            const int s2 = claim_slot(cnt_n, d);
            if (s2 < CAP) {
                pos_n[size_t(s2) * rep.stride32 + d] = q;
                pid_n[size_t(s2) * rep.stride32 + d] = src[h].template slot_id<COH>(k, pid_o, rep.stride32);
            } else {
                over = true;
            }
        }
    }
    return over;
}

// One active cell of a colour pass: planar index a of colour col in the
// replica.  Its eight neighbours' occupancies are loaded and, in the fixed
// form, their first two slots copied into `mine` (this thread's 2 x 8 + 1
// entries of shared memory) with cp.async, all before the cell itself is
// loaded and its draws are made, so the generator's arithmetic overlaps the
// latency.  Then the cell's occupants are shuffled and make rep.nt serial
// trial moves (try_cell); a cell of more than kEagerSlots disks keeps them in
// sp / si (this thread's CAP entries of shared memory).  Adds the trials and
// acceptances to att and acc.  No copy is left in flight on return.
template <bool FIX, int CAP, int NTC, bool COH>
__device__ __forceinline__ void pass_cell(const Rep& rep, const Frame& f, int col, uint32_t a,
                                          const uint8_t* __restrict__ cnt, P2<FIX>* pos, int32_t* pid, int2* mine,
                                          P2<FIX>* sp, int32_t* si, uint32_t& att, uint32_t& acc) {
    const int m = rep.m, hm = rep.hm;
    const uint32_t row = div_by(a, rep.hm_mul, rep.hm_sh);
    const int X = int(a - row * uint32_t(hm));
    const int px = col & 1, py = col >> 1;
    const int cx = 2 * X + px;
    const int cy = 2 * int(row) + py;
    const uint32_t cl = uint32_t(cy) * uint32_t(m) + uint32_t(cx);  // Philox counter: row-major cell
    const uint32_t cell = rep.coff + uint32_t(col) * uint32_t(rep.hh) + a;
    // Column and row parts of the neighbour indices: the columns cx - 1, cx + 1
    // have parity 1 - px and half-columns X - 1 + px, X + px (periodically),
    // the rows cy -+ 1 parity 1 - py and half-rows row - 1 + py, row + py.
    uint32_t xp[3], yp[3];
    {
        const uint32_t hh = uint32_t(rep.hh), hmu = uint32_t(hm);
        int hl = X - 1 + px, hr = X + px;
        hl = hl < 0 ? hl + hm : hl;
        hr = hr >= hm ? hr - hm : hr;
        const uint32_t xo = uint32_t(1 - px) * hh;
        xp[0] = xo + uint32_t(hl);
        xp[1] = uint32_t(px) * hh + uint32_t(X);
        xp[2] = xo + uint32_t(hr);
        int rl = int(row) - 1 + py, rr = int(row) + py;
        rl = rl < 0 ? rl + hm : rl;
        rr = rr >= hm ? rr - hm : rr;
        const uint32_t yo = rep.coff + uint32_t(1 - py) * 2u * hh;
        yp[0] = yo + uint32_t(rl) * hmu;
        yp[1] = rep.coff + uint32_t(py) * 2u * hh + row * hmu;
        yp[2] = yo + uint32_t(rr) * hmu;
    }
    // Fixed form: neighbour i (0..8, centre skipped as nbr index q) has its
    // occupancy in bits 4q..4q+3 of nocc and slots 0, 1 in mine[2q], mine[2q + 1].
    uint32_t nocc = 0;
    if constexpr (FIX) {
        const uint32_t sm = static_cast<uint32_t>(__cvta_generic_to_shared(mine));
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) continue;
            const int q = i < 4 ? i : i - 1;
            const uint32_t ci = yp[i / 3] + xp[i % 3];
            nocc |= uint32_t(occupancy<CAP, COH>(cnt, ci)) << (4 * q);
            cp_async8(sm + uint32_t(2 * q) * 8u, pos + ci);
            cp_async8(sm + uint32_t(2 * q + 1) * 8u, pos + rep.stride32 + ci);
        }
    } else {
        // FP64: the occupancies and slot 0 of every neighbour, staged before
        // the cell's own loads and draws (slots beyond 0 of the neighbours
        // that hold more disks are loaded in the test)
        const uint32_t sm = static_cast<uint32_t>(__cvta_generic_to_shared(mine));
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i == 4) continue;
            const int q = i < 4 ? i : i - 1;
            const uint32_t ci = yp[i / 3] + xp[i % 3];
            nocc |= uint32_t(occupancy<CAP, COH>(cnt, ci)) << (4 * q);
            cp_async16(sm + uint32_t(q) * blockDim.x * 16u, pos + ci);
        }
    }
    CellRegs<FIX, true> own;
    load_cell<FIX, true, CAP, COH>(cnt, pos, pid, rep.stride32, cell, own);
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
                // Only those neighbours are visited (bit 4q + 3 of the mask):
                // nearly every warp has a lane with one, but a lane rarely
                // has more than one.
                for (uint32_t cm = (nocc + 0x55555555u) & 0x88888888u; cm != 0u; cm &= cm - 1u) {
                    const int q = (__ffs(int(cm)) - 1) >> 2;
                    const int i = q + (q >= 4 ? 1 : 0);
                    const int ox = int((0x24924u >> (2 * i)) & 3u) - 1;  // i % 3 - 1
                    const int oy = int((0x2A540u >> (2 * i)) & 3u) - 1;  // i / 3 - 1
                    const int ni = int(nocc >> (4 * q)) & 0xF;
                    // the cell index is recomputed here, so that no register keeps it
                    const uint32_t ci = rep.coff + row_part(rep, wrap_cell(cy + oy, m)) + col_part(rep, wrap_cell(cx + ox, m));
                    for (int k = kEagerSlots; k < ni; ++k)
                        ok &= pair_clear<FIX>(ld_cell<COH>(pos + size_t(k) * rep.stride32 + ci), ox, oy, np, rep);
                }
            } else {
                cp_async_wait_all();  // a no-op after the first trial
                const double2* nb = reinterpret_cast<const double2*>(mine);
                // FP64 arithmetic bounds the FP64 form: a pair is tested only
                // while the move still stands
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (i == 4) continue;
                    const int q = i < 4 ? i : i - 1;
                    const int ox = i % 3 - 1, oy = i / 3 - 1;
                    const int ni = int(nocc >> (4 * q)) & 0xF;
                    if (ok && ni >= 1) ok = pair_clear<FIX>(nb[size_t(q) * blockDim.x], ox, oy, np, rep);
                }
                // neighbours of two or more disks (a nibble n >= 2 is the one
                // whose n + 6 sets its bit 3): their further slots from memory
                for (uint32_t cm = (nocc + 0x66666666u) & 0x88888888u; cm != 0u && ok; cm &= cm - 1u) {
                    const int q = (__ffs(int(cm)) - 1) >> 2;
                    const int i = q + (q >= 4 ? 1 : 0);
                    const int ox = int((0x24924u >> (2 * i)) & 3u) - 1;  // i % 3 - 1
                    const int oy = int((0x2A540u >> (2 * i)) & 3u) - 1;  // i / 3 - 1
                    const int ni = int(nocc >> (4 * q)) & 0xF;
                    const uint32_t ci = rep.coff + row_part(rep, wrap_cell(cy + oy, m)) + col_part(rep, wrap_cell(cx + ox, m));
                    for (int k = 1; k < ni && ok; ++k)
                        ok = pair_clear<FIX>(ld_cell<COH>(pos + size_t(k) * rep.stride32 + ci), ox, oy, np, rep);
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
            const uint32_t na = try_cell<FIX, kEagerSlots, NTC>(rep, f.sweep, cl, P, n, neighbours_clear);
            acc += na;
            // written back in id order (the ids too, since the sort may have permuted them)
            if (na > 0 || n > 1) {
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
            for (int q = 0; q < n; ++q) {
                P2<FIX> v = own.template slot<COH>(q, pos, rep.stride32);
                int32_t id = own.template slot_id<COH>(q, pid, rep.stride32);
                int k = q;
                for (; k > 0 && si[k - 1] > id; --k) {
                    sp[k] = sp[k - 1];
                    si[k] = si[k - 1];
                }
                sp[k] = v;
                si[k] = id;
            }
            acc += try_cell_in<FIX, CAP, NTC>(rep, f.sweep, cl, SmemCell<FIX>{sp}, n, neighbours_clear);
            for (int q = 0; q < n; ++q) {
                pos[size_t(q) * rep.stride32 + cell] = sp[q];
                pid[size_t(q) * rep.stride32 + cell] = si[q];
            }
        }
        att += uint32_t(rep.nt);
    }
    // no copy may still be landing in shared memory when the thread moves on
    cp_async_wait_all();
}

}  // namespace hd
