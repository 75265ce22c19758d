// hd_sweep.cu -- the checkerboard sweep of massively parallel local Monte
// Carlo for hard disks (Engel et al., arXiv:1211.1645, Sec. II.B).
//
// Layout (per replica, concatenated over replicas): an m x m grid of cells in
// the current shifted frame; cell c holds cnt[c] <= CAP disks in slots
// c*CAP .. c*CAP+cnt[c]-1, ordered by ascending disk id, each slot holding
// the disk's offset inside the cell (double2 in [0,w)^2, or int2 in
// [0,W)^2 in units of 2^-24 sigma) and its id.  Cell-local coordinates are
// the paper's remedy for cancellation at large L (Sec. II.B).
//
// One sweep = k_rebuild (move every disk into the new shifted frame: each new
// cell gathers from the 2 x 2 old cells that can feed it) followed by four
// k_pass launches, one per colour in the sweep's random order.  Cells of one
// colour are never neighbours, so every thread of a pass owns its cell
// outright and only reads the (unchanging) cells of the other colours.
#include <type_traits>

#include "hd_kernels.h"

namespace hd {

__global__ void k_draws(const Rep* __restrict__ reps, int R, Frame* __restrict__ table,
                        Frame* __restrict__ cur, uint64_t* __restrict__ sweep_ctr, int nchunk) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const Rep rep = reps[r];
    Frame* t = table + size_t(r) * (kMaxChunk + 1);
    t[0] = cur[r];
    const uint64_t s0 = sweep_ctr[r];
    Frame f;
    for (int j = 1; j <= nchunk; ++j) {
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
    cur[r] = t[nchunk];
    sweep_ctr[r] = s0 + uint64_t(nchunk);
}

template <class T, int CAP>
__device__ __forceinline__ T pick(const T (&a)[CAP], int s) {
    T v = a[0];
#pragma unroll
    for (int q = 1; q < CAP; ++q)
        if (q == s) v = a[q];
    return v;
}

template <class T, int CAP>
__device__ __forceinline__ void place(T (&a)[CAP], int s, T v) {
#pragma unroll
    for (int q = 0; q < CAP; ++q)
        if (q == s) a[q] = v;
}

__device__ __forceinline__ uint32_t pick_word(const uint4& w0, const uint4& w1, int i) {
    switch (i) {
        case 0: return w0.x;
        case 1: return w0.y;
        case 2: return w0.z;
        case 3: return w0.w;
        case 4: return w1.x;
        case 5: return w1.y;
        case 6: return w1.z;
        default: return w1.w;
    }
}

template <bool FIX>
using P2 = std::conditional_t<FIX, int2, double2>;

// ---------------------------------------------------------------------------
// Rebuild: gather each new cell from the 2 x 2 old cells that can feed it.
// With d = old shift - new shift in (-w, w), a coordinate u + d lies in
// (-w, 2w), so a disk moves by at most one cell per axis, toward -x when
// d < 0 is impossible for d >= 0: new cell c receives from old c and c-1
// (d >= 0) or from old c and c+1 (d < 0).
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_rebuild(const Rep* __restrict__ reps, int R, const Frame* __restrict__ table, int j,
          const uint8_t* __restrict__ cnt_o, const P2<FIX>* __restrict__ pos_o, const int32_t* __restrict__ pid_o,
          uint8_t* __restrict__ cnt_n, P2<FIX>* __restrict__ pos_n, int32_t* __restrict__ pid_n,
          int* __restrict__ err) {
    const int r = find_rep<false>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int64_t c = int64_t(blockIdx.x - rep.blk_cell) * blockDim.x + threadIdx.x;
    if (c >= int64_t(m) * m) return;
    const int cx = int(c % m), cy = int(c / m);
    const Frame fo = table[size_t(r) * (kMaxChunk + 1) + j - 1];
    const Frame fn = table[size_t(r) * (kMaxChunk + 1) + j];

    int oxn, oyn;
    double dx64 = 0.0, dy64 = 0.0;
    int32_t dxf = 0, dyf = 0;
    if constexpr (FIX) {
        dxf = fo.Sx - fn.Sx;
        dyf = fo.Sy - fn.Sy;
        oxn = dxf >= 0 ? -1 : 1;
        oyn = dyf >= 0 ? -1 : 1;
    } else {
        dx64 = __dsub_rn(fo.sx, fn.sx);
        dy64 = __dsub_rn(fo.sy, fn.sy);
        oxn = dx64 >= 0.0 ? -1 : 1;
        oyn = dy64 >= 0.0 ? -1 : 1;
    }

    int n = 0;
    bool over = false;
    int32_t ids[CAP];
    P2<FIX> pp[CAP];
#pragma unroll
    for (int q = 0; q < CAP; ++q) ids[q] = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int ocx = wrap_cell(cx + ((b & 1) ? oxn : 0), m);
        const int ocy = wrap_cell(cy + ((b & 2) ? oyn : 0), m);
        const int64_t oc = rep.cell_off + int64_t(ocy) * m + ocx;
        const int kn = cnt_o[oc];
        for (int k = 0; k < kn; ++k) {
            const P2<FIX> q = pos_o[oc * CAP + k];
            int tcx, tcy;
            P2<FIX> nq;
            if constexpr (FIX) {
                frame_change_fixed(dxf, rep.W, m, ocx, q.x, tcx, nq.x);
                frame_change_fixed(dyf, rep.W, m, ocy, q.y, tcy, nq.y);
            } else {
                frame_change_fp64(dx64, rep.w, rep.w_below, m, ocx, q.x, tcx, nq.x);
                frame_change_fp64(dy64, rep.w, rep.w_below, m, ocy, q.y, tcy, nq.y);
            }
            if (tcx != cx || tcy != cy) continue;
            if (n >= CAP) {
                over = true;
                continue;
            }
            const int32_t id = pid_o[oc * CAP + k];
            // insertion by ascending id, fully unrolled so the arrays stay in registers
            bool done = false;
#pragma unroll
            for (int s = CAP - 1; s >= 0; --s) {
                if (!done && s <= n) {
                    if (s > 0 && ids[s - 1] > id) {
                        ids[s] = ids[s - 1];
                        pp[s] = pp[s - 1];
                    } else {
                        ids[s] = id;
                        pp[s] = nq;
                        done = true;
                    }
                }
            }
            ++n;
        }
    }
    const int64_t cell = rep.cell_off + c;
    cnt_n[cell] = uint8_t(n);
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
        if (q < n) {
            pos_n[cell * CAP + q] = pp[q];
            pid_n[cell * CAP + q] = ids[q];
        }
    }
    if (over) atomicOr(err, 1);
}

// ---------------------------------------------------------------------------
// One colour pass: every active cell shuffles its occupants (Fisher-Yates,
// one 32-bit word per swap) and makes nt serial trial moves; trial t moves
// the occupant at position t mod n of the shuffled order (Sec. II.B).
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_pass(const Rep* __restrict__ reps, int R, const Frame* __restrict__ table, int j, int p,
       const uint8_t* __restrict__ cnt, P2<FIX>* pos, unsigned long long* __restrict__ counters) {
    const int r = find_rep<true>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m, hm = rep.hm;
    const int64_t a = int64_t(blockIdx.x - rep.blk_act) * blockDim.x + threadIdx.x;
    const Frame f = table[size_t(r) * (kMaxChunk + 1) + j];
    const int col = int(f.perm >> (2 * p)) & 3;
    uint32_t att = 0, acc = 0;
    if (a < int64_t(hm) * hm) {
        const int cx = 2 * int(a % hm) + (col & 1);
        const int cy = 2 * int(a / hm) + (col >> 1);
        const uint32_t cl = uint32_t(cy) * uint32_t(m) + uint32_t(cx);
        const int64_t cell = rep.cell_off + cl;
        const int n = cnt[cell];
        if (n > 0) {
            P2<FIX> P[CAP];
#pragma unroll
            for (int q = 0; q < CAP; ++q)
                if (q < n) P[q] = pos[cell * CAP + q];
                else P[q] = P2<FIX>{};

            // shuffle of the occupants (ascending ids) -> order, one nibble per slot
            uint64_t order = 0xFEDCBA9876543210ull;
            uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0;
            if (n > 1) w0 = philox(f.sweep, 0u, cl, kTagShuffle, rep.key0, rep.key1);
            if (CAP > 5 && n > 5) w1 = philox(f.sweep, 1u, cl, kTagShuffle, rep.key0, rep.key1);
#pragma unroll
            for (int k = CAP - 1; k >= 1; --k) {
                if (k < n) {
                    const uint32_t jj = bounded(pick_word(w0, w1, n - 1 - k), uint32_t(k + 1));
                    const uint64_t vk = (order >> (4 * k)) & 0xFull;
                    const uint64_t vj = (order >> (4 * jj)) & 0xFull;
                    order &= ~((0xFull << (4 * k)) | (0xFull << (4 * jj)));
                    order |= (vj << (4 * k)) | (vk << (4 * jj));
                }
            }

            for (int t = 0; t < rep.nt; ++t) {
                const uint4 u = philox(f.sweep, uint32_t(t), cl, kTagTrial, rep.key0, rep.key1);
                const int slot = int((order >> (4 * (t % n))) & 0xFull);
                const P2<FIX> me = pick(P, slot);
                P2<FIX> np;
                bool ok;
                if constexpr (FIX) {
                    const uint32_t span = uint32_t(2 * rep.D + 1);
                    np.x = me.x + (int32_t(bounded(u.x, span)) - rep.D);
                    np.y = me.y + (int32_t(bounded(u.y, span)) - rep.D);
                    ok = np.x >= 0 && np.x < rep.W && np.y >= 0 && np.y < rep.W;
                } else {
                    np.x = __dadd_rn(me.x, step_fp64(u.x, u.y, rep.delta));
                    np.y = __dadd_rn(me.y, step_fp64(u.z, u.w, rep.delta));
                    ok = np.x >= 0.0 && np.x < rep.w && np.y >= 0.0 && np.y < rep.w;
                }
                if (ok) {
                    // occupants of the own cell other than the moving disk
#pragma unroll
                    for (int q = 0; q < CAP; ++q) {
                        if (q < n && q != slot && ok) {
                            if constexpr (FIX) {
                                const int32_t rx = P[q].x - np.x, ry = P[q].y - np.y;
                                ok = (int64_t(rx) * rx + int64_t(ry) * ry) >= kFxDiam2;
                            } else {
                                const double rx = __dsub_rn(P[q].x, np.x), ry = __dsub_rn(P[q].y, np.y);
                                ok = !(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)) < 4.0);
                            }
                        }
                    }
                    // the eight neighbouring cells (other colours, not written in this pass)
                    for (int nb = 0; nb < 9 && ok; ++nb) {
                        if (nb == 4) continue;
                        const int ox = nb % 3 - 1, oy = nb / 3 - 1;
                        const int64_t nc = rep.cell_off + int64_t(wrap_cell(cy + oy, m)) * m + wrap_cell(cx + ox, m);
                        const int nn = cnt[nc];
                        for (int k = 0; k < nn && ok; ++k) {
                            const P2<FIX> q = pos[nc * CAP + k];
                            if constexpr (FIX) {
                                const int32_t rx = (q.x + ox * rep.W) - np.x;
                                const int32_t ry = (q.y + oy * rep.W) - np.y;
                                ok = (int64_t(rx) * rx + int64_t(ry) * ry) >= kFxDiam2;
                            } else {
                                const double offx = ox < 0 ? -rep.w : (ox > 0 ? rep.w : 0.0);
                                const double offy = oy < 0 ? -rep.w : (oy > 0 ? rep.w : 0.0);
                                const double rx = __dsub_rn(__dadd_rn(q.x, offx), np.x);
                                const double ry = __dsub_rn(__dadd_rn(q.y, offy), np.y);
                                ok = !(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)) < 4.0);
                            }
                        }
                    }
                }
                ++att;
                if (ok) {
                    place(P, slot, np);
                    ++acc;
                }
            }
            if (acc > 0) {
#pragma unroll
                for (int q = 0; q < CAP; ++q)
                    if (q < n) pos[cell * CAP + q] = P[q];
            }
        }
    }
    // block-level sums of the trial counters, one atomic pair per block
    __shared__ unsigned int s_att[32], s_acc[32];
    att = __reduce_add_sync(0xffffffffu, att);
    acc = __reduce_add_sync(0xffffffffu, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_att[warp] = att;
        s_acc[warp] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ta = 0, tc = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            ta += s_att[w];
            tc += s_acc[w];
        }
        if (ta) atomicAdd(&counters[2 * r], ta);
        if (tc) atomicAdd(&counters[2 * r + 1], tc);
    }
}

// ---------------------------------------------------------------------------
// Global positions from the cell frame: X = (cx w + u) + shift, wrapped once.
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_positions(const Rep* __restrict__ reps, int R, const Frame* __restrict__ cur, const uint8_t* __restrict__ cnt,
            const P2<FIX>* __restrict__ pos, const int32_t* __restrict__ pid, double* __restrict__ xy) {
    const int r = find_rep<false>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int64_t c = int64_t(blockIdx.x - rep.blk_cell) * blockDim.x + threadIdx.x;
    if (c >= int64_t(m) * m) return;
    const int cx = int(c % m), cy = int(c / m);
    const Frame f = cur[r];
    const int64_t cell = rep.cell_off + c;
    const int n = cnt[cell];
    for (int k = 0; k < n; ++k) {
        const P2<FIX> q = pos[cell * CAP + k];
        const int64_t id = rep.id_off + pid[cell * CAP + k];
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
    k_draws<<<(c.R + 63) / 64, 64, 0, c.stream>>>(c.reps, c.R, table, cur, sweep_ctr, nchunk);
    return cudaGetLastError();
}

template <bool FIX, int CAP>
static void rebuild_t(const LaunchCfg& c, const Frame* table, int j, CellBufs a, CellBufs b, int* err) {
    k_rebuild<FIX, CAP><<<c.blocks_cell, c.threads, 0, c.stream>>>(
        c.reps, c.R, table, j, a.cnt, (const P2<FIX>*)a.pos, a.pid, b.cnt, (P2<FIX>*)b.pos, b.pid, err);
}

cudaError_t launch_rebuild(const LaunchCfg& c, const Frame* table, int j, CellBufs from, CellBufs to, int* err) {
    if (c.fixed) {
        if (c.cap == 4) rebuild_t<true, 4>(c, table, j, from, to, err);
        else rebuild_t<true, 9>(c, table, j, from, to, err);
    } else {
        if (c.cap == 4) rebuild_t<false, 4>(c, table, j, from, to, err);
        else rebuild_t<false, 9>(c, table, j, from, to, err);
    }
    return cudaGetLastError();
}

template <bool FIX, int CAP>
static void pass_t(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                   unsigned long long* counters) {
    k_pass<FIX, CAP><<<c.blocks_act, c.threads, 0, c.stream>>>(c.reps, c.R, table, j, p, cells.cnt,
                                                                 (P2<FIX>*)cells.pos, counters);
}

cudaError_t launch_pass(const LaunchCfg& c, const Frame* table, int j, int p, CellBufs cells,
                        unsigned long long* counters) {
    if (c.fixed) {
        if (c.cap == 4) pass_t<true, 4>(c, table, j, p, cells, counters);
        else pass_t<true, 9>(c, table, j, p, cells, counters);
    } else {
        if (c.cap == 4) pass_t<false, 4>(c, table, j, p, cells, counters);
        else pass_t<false, 9>(c, table, j, p, cells, counters);
    }
    return cudaGetLastError();
}

template <bool FIX, int CAP>
static void positions_t(const LaunchCfg& c, const Frame* cur, CellBufs cells, double* xy) {
    k_positions<FIX, CAP><<<c.blocks_cell, c.threads, 0, c.stream>>>(c.reps, c.R, cur, cells.cnt,
                                                                       (const P2<FIX>*)cells.pos, cells.pid, xy);
}

cudaError_t launch_positions(const LaunchCfg& c, const Frame* cur, CellBufs cells, double* xy) {
    if (c.fixed) {
        if (c.cap == 4) positions_t<true, 4>(c, cur, cells, xy);
        else positions_t<true, 9>(c, cur, cells, xy);
    } else {
        if (c.cap == 4) positions_t<false, 4>(c, cur, cells, xy);
        else positions_t<false, 9>(c, cur, cells, xy);
    }
    return cudaGetLastError();
}

}  // namespace hd
