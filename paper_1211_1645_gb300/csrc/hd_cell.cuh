// hd_cell.cuh -- per-cell steps of the checkerboard sweep (Engel et al.,
// arXiv:1211.1645, Sec. II.B), shared by the split kernels (one launch per
// rebuild and per colour pass) and the fused kernel (one launch per sweep):
//   sort_by_id   orders a cell's occupants by id (the shuffle's base order);
//   claim_slot   claims a slot of a destination cell during the rebuild;
//   try_cell     shuffles one active cell's occupants and makes its serial
//                trial moves against the cell itself and its neighbours.
#pragma once

#include <climits>
#include <type_traits>

#include "hd_device.cuh"

namespace hd {

template <bool FIX>
using P2 = std::conditional_t<FIX, int2, double2>;

// Slots 0 and 1 are loaded unconditionally (together they hold nearly every
// disk at liquid densities); higher slots only when the cell is that full.
constexpr int kEagerSlots = 2;

// Loads of cell data.  COH = false: through the read-only data path, valid
// while no block of the launch writes the cells it reads (one launch per
// rebuild and per colour pass).  COH = true: coherent loads cached in L2 only
// (ld.global.cg), for a launch whose blocks read cells that other blocks
// wrote earlier in the same launch, ordered by acquire / release flags.
template <bool COH, class T>
__device__ __forceinline__ T ld_cell(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// One cell as loaded by a thread: occupancy and the first kEagerSlots slots
// in registers; a higher slot is fetched when a (rare) crowded cell needs it.
template <bool FIX, bool IDS>
struct CellRegs {
    uint32_t c;           // cell index; slot k of the cell is entry k * stride + c
    P2<FIX> s[kEagerSlots];
    int32_t id[IDS ? kEagerSlots : 1];
    int n;

    template <bool COH = false>
    __device__ __forceinline__ P2<FIX> slot(int k, const P2<FIX>* __restrict__ pos, uint32_t stride) const {
        if (k == 0) return s[0];
        if (k == 1) return s[1];
        return ld_cell<COH>(pos + size_t(k) * stride + c);
    }
    template <bool COH = false>
    __device__ __forceinline__ int32_t slot_id(int k, const int32_t* __restrict__ pid, uint32_t stride) const {
        if constexpr (IDS) {
            if (k == 0) return id[0];
            if (k == 1) return id[1];
            return ld_cell<COH>(pid + size_t(k) * stride + c);
        }
        return 0;
    }
};

// Occupancy of a cell, clamped to its capacity (a count above capacity only
// arises after an overflow, which the kernels report through the error flag).
template <int CAP, bool COH = false>
__device__ __forceinline__ int occupancy(const uint8_t* __restrict__ cnt, uint32_t c) {
    const int n = ld_cell<COH>(cnt + c);
    return n < CAP ? n : CAP;
}

template <bool FIX, bool IDS, int CAP = 4, bool COH = false>
__device__ __forceinline__ void load_cell(const uint8_t* __restrict__ cnt, const P2<FIX>* __restrict__ pos,
                                          const int32_t* __restrict__ pid, uint32_t stride, uint32_t c,
                                          CellRegs<FIX, IDS>& out) {
    out.n = occupancy<CAP, COH>(cnt, c);
    out.c = c;
#pragma unroll
    for (int k = 0; k < kEagerSlots; ++k) {
        out.s[k] = ld_cell<COH>(pos + size_t(k) * stride + c);
        if constexpr (IDS) out.id[k] = ld_cell<COH>(pid + size_t(k) * stride + c);
    }
}

// Shift difference between two frames (old minus new) and the direction of
// the second feeding cell per axis (-1: old c-1 also feeds c; +1: old c+1).
template <bool FIX>
struct ShiftDelta {
    double dx, dy;
    int32_t fx, fy;
    int ox, oy;

    __device__ __forceinline__ ShiftDelta(const Frame& fo, const Frame& fn) {
        if constexpr (FIX) {
            dx = dy = 0.0;
            fx = fo.Sx - fn.Sx;
            fy = fo.Sy - fn.Sy;
            ox = fx >= 0 ? -1 : 1;
            oy = fy >= 0 ? -1 : 1;
        } else {
            fx = fy = 0;
            dx = __dsub_rn(fo.sx, fn.sx);
            dy = __dsub_rn(fo.sy, fn.sy);
            ox = dx >= 0.0 ? -1 : 1;
            oy = dy >= 0.0 ? -1 : 1;
        }
    }
};

// The occupants of one new cell, ascending id; id INT_MAX marks an empty slot.
template <bool FIX, int CAP>
struct NewCell {
    int32_t id[CAP];
    P2<FIX> p[CAP];
    int n;
    bool over;
};

template <bool FIX, int CAP>
__device__ __forceinline__ void cswap(NewCell<FIX, CAP>& c, int a, int b) {
    if (c.id[b] < c.id[a]) {
        const int32_t t = c.id[a];
        c.id[a] = c.id[b];
        c.id[b] = t;
        const P2<FIX> u = c.p[a];
        c.p[a] = c.p[b];
        c.p[b] = u;
    }
}

// Order the first n occupants of a cell by ascending id, in registers
// (slots at or beyond n are padded with id INT_MAX so they stay last).
template <bool FIX, int CAP>
__device__ __forceinline__ void sort_by_id(P2<FIX> (&P)[CAP], int32_t (&id)[CAP], int n) {
    NewCell<FIX, CAP> c;
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
        c.p[q] = P[q];
        c.id[q] = q < n ? id[q] : INT_MAX;
    }
    if constexpr (CAP == 4) {
        cswap(c, 0, 1);
        cswap(c, 2, 3);
        cswap(c, 0, 2);
        cswap(c, 1, 3);
        cswap(c, 1, 2);
    } else {
#pragma unroll
        for (int i = 1; i < CAP; ++i)
#pragma unroll
            for (int s = i; s > 0; --s) cswap(c, s - 1, s);
    }
#pragma unroll
    for (int q = 0; q < CAP; ++q) {
        P[q] = c.p[q];
        id[q] = c.id[q];
    }
}

// Claim the next free slot of cell di by adding one to its occupancy byte;
// returns the slot.  The byte counters of four consecutive cells share one
// 32-bit word (the counter array is 4-byte aligned and padded).
__device__ __forceinline__ int claim_slot(uint8_t* cnt, uint32_t di) {
    unsigned int* word = reinterpret_cast<unsigned int*>(cnt) + (di >> 2);
    const unsigned int shift = 8u * (di & 3u);
    const unsigned int old = atomicAdd(word, 1u << shift);
    return int((old >> shift) & 0xFFu);
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

// The FP64 overlap test proper: the centre distance of q (its cell (ox, oy)
// cells away) and np is at least 2 sigma.  Not inlined, so that the compiler
// cannot turn the rarely taken call into FP64 instructions issued under a
// false predicate on every pair test.
static __device__ __noinline__ bool pair_clear_fp64_exact(double qx0, double qy0, int ox, int oy, double npx, double npy,
                                                   double w) {
    // (q + 0) is q itself for the non-negative cell offsets, so a zero cell
    // difference skips that addition (an FP64 operation saved)
    const double qx = ox == 0 ? qx0 : __dadd_rn(qx0, ox < 0 ? -w : w);
    const double qy = oy == 0 ? qy0 : __dadd_rn(qy0, oy < 0 ? -w : w);
    const double rx = __dsub_rn(qx, npx);
    const double ry = __dsub_rn(qy, npy);
    return !(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)) < 4.0);
}

// Overlap test of a proposed position np against one occupant q whose cell is
// (ox, oy) cells away from the moving disk's cell: true when clear (the centre
// distance is at least 2 sigma).
template <bool FIX>
__device__ __forceinline__ bool pair_clear(const P2<FIX>& q, int ox, int oy, const P2<FIX>& np, const Rep& rep) {
    if constexpr (FIX) {
        const int32_t rx = (q.x + ox * rep.W) - np.x;
        const int32_t ry = (q.y + oy * rep.W) - np.y;
        // d^2 >= 2^50 exactly when the high word of the (non-negative, < 2^63)
        // 64-bit square sum is >= 2^18: one 32-bit compare
        const uint64_t d2 = uint64_t(int64_t(rx) * rx) + uint64_t(int64_t(ry) * ry);
        static_assert(kFxDiam2 == (int64_t(1) << 50), "the high-word test assumes (2 sigma)^2 = 2^50");
        return uint32_t(d2 >> 32) >= (1u << 18);
    } else {
        // GB300's FP64 pipe is narrow, so the pair is first decided in float:
        // when the float estimate of d^2 lies outside [d2_lo, d2_hi), which
        // brackets 4 by the estimate's error bound (see plan_replica), it is
        // on the same side of 4 as the FP64 value below.  Only pairs within
        // that band of contact run the FP64 test.
        const float npx = approx_f32(np.x), npy = approx_f32(np.y);
        const float fx = approx_f32(q.x), fy = approx_f32(q.y);
        const float ax = ox == 0 ? fx : __fadd_rn(fx, ox < 0 ? -rep.wf : rep.wf);
        const float ay = oy == 0 ? fy : __fadd_rn(fy, oy < 0 ? -rep.wf : rep.wf);
        const float sx = __fsub_rn(ax, npx), sy = __fsub_rn(ay, npy);
        const float d2f = __fadd_rn(__fmul_rn(sx, sx), __fmul_rn(sy, sy));
        if (d2f >= rep.d2_hi) return true;
        if (d2f < rep.d2_lo) return false;
        return pair_clear_fp64_exact(q.x, q.y, ox, oy, np.x, np.y, rep.w);
    }
}

// One active cell with n >= 1 occupants P[0..n) (ascending id): Fisher-Yates
// shuffle with one 32-bit word per swap, then rep.nt serial trials; trial t
// moves the occupant at position t mod n of the shuffled order by a step
// uniform in [-delta, delta]^2, rejected if it leaves the cell or comes
// closer than 2 sigma to another occupant or to a disk of the eight
// neighbouring cells (`neighbours_clear(np)`).  Updates P; returns accepts.
// NTC > 0: rep.nt is known to be NTC at compile time (one trial per
// occupied cell is the usual case at liquid and solid densities with the
// smallest cells), which lets the compiler bound every value's live range;
// NTC = 0 reads rep.nt.
// u0_in (fixed form, nullable): trial 0's block, when the caller has drawn it
// already (to overlap the generator with its loads).
// A cell's occupants as try_cell sees them: in registers (slot q of a
// register array, a run-time q picked by compile-time selects) or in shared
// memory (any slot read directly).
template <bool FIX, int CAP>
struct RegCell {
    P2<FIX> (&P)[CAP];
    __device__ __forceinline__ P2<FIX> operator[](int q) const { return P[q]; }
    __device__ __forceinline__ P2<FIX> pick(int slot) const {
        P2<FIX> me = P[0];
#pragma unroll
        for (int q = 1; q < CAP; ++q)
            if (q == slot) me = P[q];
        return me;
    }
    __device__ __forceinline__ void put(int slot, const P2<FIX>& v) const {
#pragma unroll
        for (int q = 0; q < CAP; ++q)
            if (q == slot) P[q] = v;
    }
};

template <bool FIX>
struct SmemCell {
    P2<FIX>* P;  // shared memory, slot q at P[q]
    __device__ __forceinline__ P2<FIX> operator[](int q) const { return P[q]; }
    __device__ __forceinline__ P2<FIX> pick(int slot) const { return P[slot]; }
    __device__ __forceinline__ void put(int slot, const P2<FIX>& v) const { P[slot] = v; }
};

template <bool FIX, int CAP, int NTC = 0, class Cell, class NbrClear>
__device__ __forceinline__ uint32_t try_cell_in(const Rep& rep, uint32_t sweep, uint32_t cl, const Cell& P, int n,
                                                NbrClear&& neighbours_clear, const uint4* u0_in = nullptr) {
    uint64_t order = 0xFEDCBA9876543210ull;  // position -> slot, one nibble each
    // The fixed-point step uses two words of a trial block; the other two of
    // trial 0's block are the first two swap words, so a cell of up to three
    // occupants needs a single generator call.  The FP64 step uses all four.
    uint4 u0 = make_uint4(0, 0, 0, 0);
    if constexpr (FIX) u0 = u0_in ? *u0_in : philox(sweep, 0u, cl, kTagTrial, rep.key0, rep.key1);
    if (n > 1) {
        uint4 w0, w1 = make_uint4(0, 0, 0, 0);
        if constexpr (FIX) {
            w0 = make_uint4(u0.z, u0.w, 0u, 0u);
            if (n > 3) {
                const uint4 a = philox(sweep, 0u, cl, kTagShuffle, rep.key0, rep.key1);
                w0.z = a.x;
                w0.w = a.y;
                w1 = make_uint4(a.z, a.w, 0u, 0u);
                if (CAP > 7 && n > 7) {
                    const uint4 b = philox(sweep, 1u, cl, kTagShuffle, rep.key0, rep.key1);
                    w1.z = b.x;
                    w1.w = b.y;
                }
            }
        } else {
            w0 = philox(sweep, 0u, cl, kTagShuffle, rep.key0, rep.key1);
            if (CAP > 5 && n > 5) w1 = philox(sweep, 1u, cl, kTagShuffle, rep.key0, rep.key1);
        }
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
    }
    uint32_t acc = 0;
    const int nt = NTC > 0 ? NTC : rep.nt;
    for (int t = 0; t < nt; ++t) {
        const uint4 u = (FIX && t == 0) ? u0 : philox(sweep, uint32_t(t), cl, kTagTrial, rep.key0, rep.key1);
        const int slot = int((order >> (4 * (n == 1 ? 0 : t % n))) & 0xFull);
        const P2<FIX> me = P.pick(slot);
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
            ok = nonneg_bits(np.x) && below_pos_bits(np.x, rep.w) && nonneg_bits(np.y) && below_pos_bits(np.y, rep.w);
        }
        // The tests run whatever the boundary test said (a warp rarely skips
        // them all), without branches: a slot that is not an occupant, or the
        // moving disk itself, masks its own result.  A move outside the cell
        // keeps every difference within int32 (|dx| < 3W).
        if constexpr (FIX) {
#pragma unroll
            for (int q = 0; q < CAP; ++q)
                ok &= pair_clear<FIX>(P[q], 0, 0, np, rep) | (q >= n) | (q == slot);
        } else {
            // FP64 arithmetic bounds the FP64 form: a warp skips a test no lane needs
#pragma unroll
            for (int q = 0; q < CAP; ++q)
                if (ok && q < n && q != slot) ok = pair_clear<FIX>(P[q], 0, 0, np, rep);
        }
        if (FIX || ok) ok &= neighbours_clear(np);  // the FP64 form loads neighbours lazily: skip when rejected
        if (ok) {
            P.put(slot, np);
            ++acc;
        }
    }
    return acc;
}

// try_cell_in on occupants held in a register array.
template <bool FIX, int CAP, int NTC = 0, class NbrClear>
__device__ __forceinline__ uint32_t try_cell(const Rep& rep, uint32_t sweep, uint32_t cl, P2<FIX> (&P)[CAP], int n,
                                             NbrClear&& neighbours_clear, const uint4* u0_in = nullptr) {
    return try_cell_in<FIX, CAP, NTC>(rep, sweep, cl, RegCell<FIX, CAP>{P}, n, neighbours_clear, u0_in);
}

// Sum two per-thread counters over the block and add them to counters[2r],
// counters[2r + 1] with one atomic each.  Every thread of the block must call.
__device__ __forceinline__ void block_count(uint32_t att, uint32_t acc, unsigned long long* counters, int r) {
    __shared__ unsigned int s_cnt[2][32];
    att = __reduce_add_sync(0xffffffffu, att);
    acc = __reduce_add_sync(0xffffffffu, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_cnt[0][warp] = att;
        s_cnt[1][warp] = acc;
    }
    __syncthreads();
    if (warp == 0) {
        const bool live = lane < int(blockDim.x >> 5);
        const unsigned int ta = __reduce_add_sync(0xffffffffu, live ? s_cnt[0][lane] : 0u);
        const unsigned int tc = __reduce_add_sync(0xffffffffu, live ? s_cnt[1][lane] : 0u);
        if (lane == 0 && ta) atomicAdd(&counters[2 * r], (unsigned long long)ta);
        if (lane == 1 && tc) atomicAdd(&counters[2 * r + 1], (unsigned long long)tc);
    }
}

}  // namespace hd
