// hd_fused.cu -- one whole checkerboard sweep per kernel launch, staged in
// shared memory (Engel et al., arXiv:1211.1645, Sec. II.B).
//
// A thread block owns a T x T tile of the new (shifted) cell frame and stages
// the tile plus a halo of 4 cells on every side (S = T + 8 cells per side):
//   1. scatter: every old cell that can feed the staged region moves each of
//      its disks into the new frame (the per-disk frame change of the random
//      grid shift) and claims a slot of the destination cell in shared memory;
//      the work is done in unwrapped local coordinates, so a box smaller than
//      the staged region (which then holds several copies of a cell) is
//      handled the same way;
//   1b. each cell with several occupants is ordered by id (the base order of
//      the shuffle); owned cells' occupancy and ids are written out;
//   2. the four colour passes run in shared memory.  A pass updates a cell
//      from its 3 x 3 neighbourhood as it stood after the previous pass, so
//      the region that is still exact shrinks by one cell per pass: pass p
//      (0-based) updates active cells within 3 - p cells of the tile.  Halo
//      cells are also updated by the blocks that own them; the draws are keyed
//      by the global cell index, so every copy evolves identically and the
//      owner's copy is the one written back.  Occupied active cells are first
//      compacted into two lists (one occupant / several), so no lane idles on
//      an empty cell and single-occupant warps skip the shuffle draw;
//   3. owned cells' offsets are written out.
// Each sweep reads the old frame once (plus the halo) and writes the new frame
// once, with all per-trial neighbour reads served from shared memory.
//
// Shared-memory cells are stored in colour planes (the four parities of the
// local coordinates), so the threads of a warp that work on consecutive
// active cells touch consecutive words.
#include "hd_cell.cuh"
#include "hd_kernels.h"

namespace hd {

template <bool FIX, int CAP, int T>
struct Fused {
    static constexpr int kHalo = 4;
    static constexpr int S = T + 2 * kHalo;  // staged side (even)
    static constexpr int H = S / 2;          // colour-plane side
    static constexpr int NC = S * S;
    static constexpr int SO = S + 4;         // old cells read: [X0 - 6, X0 + T + 6), even origin
    static constexpr int HO = SO / 2;
    static constexpr int kCntBytes = (NC + 3) & ~3;
    static constexpr size_t kPosBytes = size_t(CAP) * NC * sizeof(P2<FIX>);
    static constexpr size_t kPidBytes = size_t(CAP) * NC * sizeof(int32_t);
    static constexpr size_t kListBytes = size_t(2) * H * H * sizeof(uint16_t);
    static constexpr size_t kSmem = kPosBytes + kPidBytes + kCntBytes + kListBytes;

    __device__ static __forceinline__ int plane(int lx, int ly) {
        return (((ly & 1) << 1) | (lx & 1)) * (H * H) + (ly >> 1) * H + (lx >> 1);
    }
};

__device__ __forceinline__ int mod_cell(int v, int m) {
    v %= m;
    return v < 0 ? v + m : v;
}

// Cell difference b - a in {-1, 0, 1} on a periodic axis of m >= 4 cells.
__device__ __forceinline__ int cell_step(int a, int b, int m) {
    int d = b - a;
    if (d > 1) d -= m;
    else if (d < -1) d += m;
    return d;
}

template <bool FIX, int CAP, int T, int NT>
__global__ void __launch_bounds__(NT)
k_sweep_fused(const Rep* __restrict__ reps, int R, const Frame* __restrict__ table, int j,
              const uint8_t* __restrict__ cnt_o, const P2<FIX>* __restrict__ pos_o, const int32_t* __restrict__ pid_o,
              uint8_t* __restrict__ cnt_n, P2<FIX>* __restrict__ pos_n, int32_t* __restrict__ pid_n,
              unsigned long long* __restrict__ counters, int* __restrict__ err) {
    using F = Fused<FIX, CAP, T>;
    extern __shared__ __align__(16) unsigned char smem[];
    P2<FIX>* s_pos = reinterpret_cast<P2<FIX>*>(smem);                                 // [CAP][NC]
    int32_t* s_pid = reinterpret_cast<int32_t*>(smem + F::kPosBytes);                  // [CAP][NC]
    uint8_t* s_cnt = smem + F::kPosBytes + F::kPidBytes;                                // [NC]
    uint16_t* s_list = reinterpret_cast<uint16_t*>(s_cnt + F::kCntBytes);              // [2][H*H]
    __shared__ int s_len[2];
    pdl_begin();

    const int r = find_rep<kGridTile>(reps, R, blockIdx.x);
    const Rep rep = reps[r];
    const int m = rep.m;
    const int tiles_x = (m + T - 1) / T;
    const int tile = blockIdx.x - rep.blk_tile;
    const int X0 = (tile % tiles_x) * T, Y0 = (tile / tiles_x) * T;
    const size_t tb = size_t(r) * (kMaxChunk + 1);
    const Frame fn = table[tb + j];
    const ShiftDelta<FIX> sd(table[tb + j - 1], fn);

    for (int w = threadIdx.x; w < F::kCntBytes / 4; w += NT) reinterpret_cast<uint32_t*>(s_cnt)[w] = 0u;
    __syncthreads();

    // ---- 1. scatter the old disks into the staged new frame ----------------
    bool over = false;
    for (int e = threadIdx.x; e < 4 * F::HO * F::HO; e += NT) {
        const int pl = e / (F::HO * F::HO), rem = e - pl * (F::HO * F::HO);
        const int lxo = 2 * (rem % F::HO) + (pl & 1), lyo = 2 * (rem / F::HO) + (pl >> 1);
        const int gxo = mod_cell(X0 - F::kHalo - 2 + lxo, m), gyo = mod_cell(Y0 - F::kHalo - 2 + lyo, m);
        const uint32_t oc = rep.coff + row_part(rep, gyo) + col_part(rep, gxo);
        const int n = occupancy<CAP>(cnt_o, oc);
        if (n == 0) continue;
        CellRegs<FIX, true> src;
        load_cell<FIX, true, CAP>(cnt_o, pos_o, pid_o, rep.stride32, oc, src);
        for (int k = 0; k < n; ++k) {
            const P2<FIX> q = src.slot(k, pos_o, rep.stride32);
            int tcx, tcy;
            P2<FIX> nq;
            if constexpr (FIX) {
                frame_change_fixed(sd.fx, rep.W, m, gxo, q.x, tcx, nq.x);
                frame_change_fixed(sd.fy, rep.W, m, gyo, q.y, tcy, nq.y);
            } else {
                frame_change_fp64(sd.dx, rep.w, rep.w_below, m, gxo, q.x, tcx, nq.x);
                frame_change_fp64(sd.dy, rep.w, rep.w_below, m, gyo, q.y, tcy, nq.y);
            }
            const int lx = lxo - 2 + cell_step(gxo, tcx, m), ly = lyo - 2 + cell_step(gyo, tcy, m);
            if (lx < 0 || lx >= F::S || ly < 0 || ly >= F::S) continue;
            const int pl2 = F::plane(lx, ly);
            const int s = claim_slot(s_cnt, uint32_t(pl2));
            if (s < CAP) {
                s_pos[s * F::NC + pl2] = nq;
                s_pid[s * F::NC + pl2] = src.slot_id(k, pid_o, rep.stride32);
            } else {
                over = true;
            }
        }
    }
    if (over) atomicOr(err, 1);
    __syncthreads();

    // ---- 1b. order crowded cells by id; write owned occupancy and ids ------
    for (int sc = threadIdx.x; sc < F::NC; sc += NT) {
        const int lx = sc % F::S, ly = sc / F::S;
        const int pl = F::plane(lx, ly);
        const int n = min(int(s_cnt[pl]), CAP);
        int32_t ids[CAP];
        if (n > 1) {
            P2<FIX> P[CAP];
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                P[q] = s_pos[q * F::NC + pl];
                ids[q] = s_pid[q * F::NC + pl];
            }
            sort_by_id<FIX, CAP>(P, ids, n);
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                if (q < n) {
                    s_pos[q * F::NC + pl] = P[q];
                    s_pid[q * F::NC + pl] = ids[q];
                }
            }
        } else {
            ids[0] = s_pid[pl];
        }
        const bool own = lx >= F::kHalo && ly >= F::kHalo && lx < F::kHalo + T && ly < F::kHalo + T &&
                         X0 + lx - F::kHalo < m && Y0 + ly - F::kHalo < m;
        if (own) {
            const uint32_t cell = rep.coff + row_part(rep, Y0 + ly - F::kHalo) + col_part(rep, X0 + lx - F::kHalo);
            cnt_n[cell] = uint8_t(n);
#pragma unroll
            for (int q = 0; q < CAP; ++q)
                if (q < n) pid_n[size_t(q) * rep.stride32 + cell] = ids[q];
        }
    }
    __syncthreads();

    // ---- 2. four colour passes in shared memory ---------------------------
    uint32_t att = 0, acc = 0;
    const int lane = threadIdx.x & 31;
    for (int p = 0; p < 4; ++p) {
        const int col = int(fn.perm >> (2 * p)) & 3;
        const int h = 3 - p;  // rings of halo still exact after this pass
        const int lo = F::kHalo - h, hi = F::kHalo + T + h;
        const int px = col & 1, py = col >> 1;
        if (threadIdx.x < 2) s_len[threadIdx.x] = 0;
        __syncthreads();
        // compact the occupied active cells of the exact region into two lists
        for (int a0 = 0; a0 < F::H * F::H; a0 += NT) {
            const int a = a0 + int(threadIdx.x);
            int n = 0;
            if (a < F::H * F::H) {
                const int lx = 2 * (a % F::H) + px, ly = 2 * (a / F::H) + py;
                if (lx >= lo && lx < hi && ly >= lo && ly < hi) n = s_cnt[col * F::H * F::H + a];
            }
#pragma unroll
            for (int list = 0; list < 2; ++list) {
                const bool mine = list == 0 ? n == 1 : n > 1;
                const unsigned ball = __ballot_sync(0xffffffffu, mine);
                if (ball == 0u) continue;
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_len[list], __popc(ball));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (mine) s_list[list * F::H * F::H + base + __popc(ball & ((1u << lane) - 1u))] = uint16_t(a);
            }
        }
        __syncthreads();
        const int L1 = s_len[0], Ltot = L1 + s_len[1];
        for (int e = threadIdx.x; e < Ltot; e += NT) {
            const int a = e < L1 ? s_list[e] : s_list[F::H * F::H + (e - L1)];
            const int lx = 2 * (a % F::H) + px, ly = 2 * (a / F::H) + py;
            const int pl = col * F::H * F::H + a;
            const int n = min(int(s_cnt[pl]), CAP);
            const int gx = mod_cell(X0 - F::kHalo + lx, m), gy = mod_cell(Y0 - F::kHalo + ly, m);
            const uint32_t cl = uint32_t(gy) * uint32_t(m) + uint32_t(gx);
            const bool own = lx >= F::kHalo && ly >= F::kHalo && lx < F::kHalo + T && ly < F::kHalo + T &&
                             X0 + lx - F::kHalo < m && Y0 + ly - F::kHalo < m;
            P2<FIX> P[CAP];
#pragma unroll
            for (int q = 0; q < CAP; ++q) P[q] = s_pos[q * F::NC + pl];
            auto neighbours_clear = [&](const P2<FIX>& np) {
                bool ok = true;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (i == 4) continue;
                    const int ox = i % 3 - 1, oy = i / 3 - 1;
                    const int npl = F::plane(lx + ox, ly + oy);
                    const int nn = min(int(s_cnt[npl]), CAP);
                    for (int k = 0; k < nn; ++k) ok = ok && pair_clear<FIX>(s_pos[k * F::NC + npl], ox, oy, np, rep);
                }
                return ok;
            };
            const uint32_t got = try_cell<FIX, CAP>(rep, fn.sweep, cl, P, n, neighbours_clear);
            if (own) {
                att += uint32_t(rep.nt);
                acc += got;
            }
            if (got > 0) {
#pragma unroll
                for (int q = 0; q < CAP; ++q)
                    if (q < n) s_pos[q * F::NC + pl] = P[q];
            }
        }
        __syncthreads();
    }

    // ---- 3. write the owned tile cells' offsets -----------------------------
    for (int sc = threadIdx.x; sc < T * T; sc += NT) {
        const int tx = sc % T, ty = sc / T;
        if (X0 + tx >= m || Y0 + ty >= m) continue;
        const int pl = F::plane(tx + F::kHalo, ty + F::kHalo);
        const uint32_t cell = rep.coff + row_part(rep, Y0 + ty) + col_part(rep, X0 + tx);
        const int n = min(int(s_cnt[pl]), CAP);
#pragma unroll
        for (int q = 0; q < CAP; ++q)
            if (q < n) pos_n[size_t(q) * rep.stride32 + cell] = s_pos[q * F::NC + pl];
    }
    block_count(att, acc, counters, r);
}

// Tile side used by the fused sweep for a given form and capacity.
int fused_tile(bool fixed, int cap) {
    if (fixed) return cap == 4 ? 32 : 16;
    return cap == 4 ? 16 : 8;
}

template <bool FIX, int CAP, int T, int NT>
static cudaError_t fused_t(const LaunchCfg& c, const Frame* table, int j, CellBufs a, CellBufs b,
                           unsigned long long* counters, int* err) {
    constexpr size_t smem = Fused<FIX, CAP, T>::kSmem;
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_sweep_fused<FIX, CAP, T, NT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    return launch_k(k_sweep_fused<FIX, CAP, T, NT>, dim3(c.blocks_tile), dim3(NT), smem, c.stream, c.reps, c.R, table,
                    j, (const uint8_t*)a.cnt, (const P2<FIX>*)a.pos, (const int32_t*)a.pid, b.cnt, (P2<FIX>*)b.pos,
                    b.pid, counters, err);
}

cudaError_t launch_sweep_fused(const LaunchCfg& c, const Frame* table, int j, CellBufs from, CellBufs to,
                               unsigned long long* counters, int* err) {
    if (c.fixed) {
        if (c.cap == 4) return fused_t<true, 4, 32, 512>(c, table, j, from, to, counters, err);
        return fused_t<true, 9, 16, 256>(c, table, j, from, to, counters, err);
    }
    if (c.cap == 4) return fused_t<false, 4, 16, 256>(c, table, j, from, to, counters, err);
    return fused_t<false, 9, 8, 128>(c, table, j, from, to, counters, err);
}

}  // namespace hd
