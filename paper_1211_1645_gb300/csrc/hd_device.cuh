// hd_device.cuh -- device-side building blocks of the MPMC hard-disk kernels:
// the counter-based generator, per-replica constants, the per-sweep draw
// table and small helpers shared by the sweep and measurement kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hd {

// Fourth Philox counter word: keeps the draw streams of one sweep disjoint.
constexpr uint32_t kTagSweep = 1u;    // grid shift and colour order of a sweep
constexpr uint32_t kTagShuffle = 2u;  // occupant shuffle of one cell
constexpr uint32_t kTagTrial = 3u;    // one trial move of one cell

constexpr int kMaxChunk = 256;        // sweeps per draw table
constexpr int64_t kFxDiam2 = int64_t(1) << 50;  // (2 sigma)^2 in (2^-24 sigma)^2

// Constants of one replica (one independent chain).  Read-only in kernels.
struct Rep {
    int64_t N;
    int64_t cell_off;   // first cell of the replica in the concatenated cell arrays
    int64_t id_off;     // first disk of the replica in the global id order
    int64_t LF;         // fixed point: box side m * W
    int64_t stride;     // distance between slot planes (cells of all replicas)
    uint32_t coff;      // cell_off as 32 bits (all cell and slot indices fit in 32 bits)
    uint32_t stride32;  // stride as 32 bits
    int32_t hh;         // cells per colour plane, (m/2)^2
    int32_t m, hm;      // cells per side, m / 2
    int32_t nt;         // trial moves per occupied active cell per pass
    int32_t blk_cell;   // first block of the replica in whole-cell grids
    int32_t blk_act;    // first block of the replica in active-cell grids
    int32_t blk_tile;   // first block of the replica in fused-sweep tile grids
    uint32_t hm_mul;    // hm_mul, hm_sh: divide by hm with div_by
    int32_t W, D;       // fixed point: cell side, maximum step (units 2^-24 sigma)
    int32_t hist_R;     // cell reach of the contact histogram
    int32_t hm_sh;
    int32_t blk_t32;    // first block of the replica in 32-column tile grids (32 x threads/32 cells)
    int32_t tiles_x;    // such tiles per row of cells, ceil(m / 32)
    uint32_t tx_mul;    // tx_mul, tx_sh: divide by tiles_x >= 2 with div_by
    int32_t tx_sh;
    int32_t blk_seg;    // first block of the replica in half-row segment grids (one colour plane)
    int32_t nseg;       // segments per half-row, ceil((m/2) / threads)
    int32_t segw;       // half-columns per segment, ceil((m/2) / nseg)
    uint32_t seg_mul;   // seg_mul, seg_sh: divide by nseg >= 2 with div_by
    int32_t seg_sh;
    int32_t band0;      // first band (two cell rows) of the replica in the persistent sweep's progress words
    double w, w_below;  // FP64 cell side and the largest double below it
    double L, delta;    // FP64 box side and maximum step (sigma units)
    double Lm;          // realised box side (fixed form: m W 2^-24) for g(r) and eta
    double sigma;       // disk radius (output scale)
    double dr;          // realised histogram bin width (sigma units)
    uint32_t key0, key1;
    // FP64 form's float pre-tests (see pair_clear, k_hist_tile, k_psi6): the
    // cell side in float; floats bracketing (2 sigma)^2 = 4, and the
    // histogram's squared range [edge_0, edge_K), by the error bounds of the
    // float estimates of d^2; that bound for pairs two cells apart (psi_6)
    float wf, d2_lo, d2_hi, h_lo, h_hi, psi_m;
};

// Draws of one sweep: the shift of its cell frame and its colour order.
struct Frame {
    double sx, sy;   // FP64 shift in [0, w)
    int32_t Sx, Sy;  // fixed-point shift in [0, W)
    uint32_t sweep;  // first Philox counter word of the sweep
    uint32_t perm;   // colour of pass p = (perm >> 2p) & 3
};

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 multiply-xor
// bijection with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t rk0 = k0 + uint32_t(round) * 0x9E3779B9u;
        const uint32_t rk1 = k1 + uint32_t(round) * 0xBB67AE85u;
        const uint64_t p0 = uint64_t(0xD2511F53u) * c0;  // one 32x32 -> 64 multiply per word
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t y0 = uint32_t(p1 >> 32) ^ c1 ^ rk0;
        const uint32_t y2 = uint32_t(p0 >> 32) ^ c3 ^ rk1;
        c0 = y0;
        c1 = uint32_t(p1);
        c2 = y2;
        c3 = uint32_t(p0);
    }
    return make_uint4(c0, c1, c2, c3);
}

// Programmatic dependent launch: allow the next kernel of the stream to be
// scheduled once every block of this one has started, and wait until the
// previous kernel has completed and its memory is visible.  Both are no-ops
// when the launch did not opt in.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// A float within a relative 2^-20 of x (|x| < 2^128), from the high word of
// x alone (integer operations only, no FP64 instruction): the exponent
// rebiased from 1023 to 127 and the 20 mantissa bits of the high word widened
// to the float's 23 (truncation toward zero); |x| < 2^-126 gives 0.
__device__ __forceinline__ float approx_f32(double x) {
    const uint32_t hi = uint32_t(__double2hiint(x));
    const uint32_t mag = hi & 0x7FFFFFFFu;
    const uint32_t f = mag < (897u << 20) ? 0u : ((mag - (896u << 20)) << 3);
    return __uint_as_float(f | (hi & 0x80000000u));
}

// floor(word * n / 2^32): an integer in [0, n).
__device__ __forceinline__ uint32_t bounded(uint32_t word, uint32_t n) { return __umulhi(word, n); }

// n / d for a divisor d >= 2 fixed per replica, by one multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d),
// mul = floor(2^32 (2^l - d) / d) + 1 and sh = l - 1, t = umulhi(mul, n)
// and q = (t + ((n - t) >> 1)) >> sh, exact for every 32-bit n.
__device__ __forceinline__ uint32_t div_by(uint32_t n, uint32_t mul, int sh) {
    const uint32_t t = __umulhi(mul, n);
    return (t + ((n - t) >> 1)) >> sh;
}

// Origin (X0, Y0) of block b (replica-local) of a 32-column tile grid whose
// tiles are 32 x rows cells, row-major over tiles.
__device__ __forceinline__ void tile32_origin(const Rep& r, uint32_t b, int rows, int& X0, int& Y0) {
    const uint32_t ty = r.tiles_x > 1 ? div_by(b, r.tx_mul, r.tx_sh) : b;
    X0 = int(b - ty * uint32_t(r.tiles_x)) * 32;
    Y0 = int(ty) * rows;
}

__device__ __forceinline__ int wrap_cell(int c, int m) { return c < 0 ? c + m : (c >= m ? c - m : c); }

// Cells are stored in four colour planes (parities of cx and cy), each an
// (m/2) x (m/2) row-major array; slot k of every cell lives in its own plane
// at distance k * stride.  The cells a warp touches in a colour pass -- its
// 32 active cells and each of their eight neighbours -- are then consecutive
// entries of one plane.
__host__ __device__ __forceinline__ int64_t cell_index(const Rep& r, int cx, int cy) {
    return r.cell_off + int64_t(((cy & 1) << 1) | (cx & 1)) * r.hm * r.hm + int64_t(cy >> 1) * r.hm + (cx >> 1);
}

// Inverse of cell_index for a replica-local planar position a in [0, m^2)
// (the plane by three comparisons, the row by div_by).
__device__ __forceinline__ void cell_coords(const Rep& r, int64_t a, int& cx, int& cy) {
    const uint32_t au = uint32_t(a), hh = uint32_t(r.hh), hm = uint32_t(r.hm);
    const uint32_t plane = uint32_t(au >= hh) + uint32_t(au >= 2u * hh) + uint32_t(au >= 3u * hh);
    const uint32_t rem = au - plane * hh;
    const uint32_t row = div_by(rem, r.hm_mul, r.hm_sh);
    cx = 2 * int(rem - row * hm) + int(plane & 1);
    cy = 2 * int(row) + int(plane >> 1);
}

// Column part and row part of a 32-bit colour-planar cell index:
// cell_index = coff + row_part(cy) + col_part(cx).
__device__ __forceinline__ uint32_t col_part(const Rep& r, int cx) {
    return uint32_t(cx & 1) * uint32_t(r.hh) + uint32_t(cx >> 1);
}
__device__ __forceinline__ uint32_t row_part(const Rep& r, int cy) {
    return uint32_t(cy & 1) * uint32_t(2 * r.hh) + uint32_t(cy >> 1) * uint32_t(r.hm);
}

// Grids over all replicas: whole cells, active cells of one colour, tiles.
enum GridKind { kGridCell = 0, kGridAct = 1, kGridTile = 2, kGridT32 = 3, kGridSeg = 4 };

// Replica owning block `blk`, given per-replica first blocks (ascending).
template <int KIND>
__device__ __forceinline__ int find_rep(const Rep* __restrict__ reps, int R, int blk) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int start = KIND == kGridAct    ? reps[mid].blk_act
                          : KIND == kGridTile ? reps[mid].blk_tile
                          : KIND == kGridT32  ? reps[mid].blk_t32
                          : KIND == kGridSeg  ? reps[mid].blk_seg
                                              : reps[mid].blk_cell;
        if (start <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// GB300's FP64 pipe is narrow, so the FP64 form does on integer units what
// needs no rounding: the conversion of an integer of at most 53 bits, a
// scaling by a power of two, and comparisons.  The values involved are
// finite and never NaN.
//
// double(v) for 0 < |v| < 2^53 (exact): the leading one moved to bit 52 and
// dropped, the exponent from the leading-zero count.
__device__ __forceinline__ double exact_from_i53(int64_t v) {
    const uint64_t s = v < 0 ? (uint64_t(1) << 63) : 0u;
    const uint64_t a = v < 0 ? uint64_t(-v) : uint64_t(v);
    const int lz = __clzll(static_cast<long long>(a));  // >= 11
    const uint64_t mant = (a << (lz - 11)) & ((uint64_t(1) << 52) - 1u);
    return __longlong_as_double(static_cast<long long>(s | (uint64_t(1023 + 63 - lz) << 52) | mant));
}

// x * 2^-53 for x = 0 or |x| >= 2^-900 (the step's delta * v with delta 0
// or at least 2^-900, |v| >= 1, checked on the host): x itself for a zero,
// else the exponent lowered by 53, exact since the result stays normal.
__device__ __forceinline__ double scale_2m53(double x) {
    const long long b = __double_as_longlong(x);
    return ((b >> 52) & 0x7FF) == 0 ? x : __longlong_as_double(b - (static_cast<long long>(53) << 52));
}

// x >= 0.0 (-0.0 included) and x < y for finite x and finite y > 0, on the
// bits: a non-negative double orders as its bit pattern; a negative one
// (sign bit set) is a negative integer, below any positive y.
__device__ __forceinline__ bool nonneg_bits(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == static_cast<long long>(0x8000000000000000ull);
}
__device__ __forceinline__ bool below_pos_bits(double x, double y) {
    return __double_as_longlong(x) < __double_as_longlong(y);
}

// Symmetric FP64 step in (-delta, delta) from two 32-bit words: a 53-bit
// integer k gives (2k + 1 - 2^53) * 2^-53, a set symmetric about zero;
// computed as delta * v rounded once, then scaled exactly.
__device__ __forceinline__ double step_fp64(uint32_t hi, uint32_t lo, double delta) {
    const uint64_t k = (uint64_t(hi >> 6) << 27) | uint64_t(lo >> 5);
    const int64_t v = int64_t(2 * k + 1) - (int64_t(1) << 53);  // odd, never 0
    return scale_2m53(__dmul_rn(delta, exact_from_i53(v)));
}

// Move one coordinate of one disk into the next cell frame (FP64).  d is the
// old shift minus the new one, |d| < w.  Edge cases at the last ulp are
// resolved toward staying inside [0, w).
__device__ __forceinline__ void frame_change_fp64(double d, double w, double w_below, int m, int c,
                                                  double u, int& c_out, double& u_out) {
    double t = __dadd_rn(u, d);
    if (!nonneg_bits(t)) {
        const double v = __dadd_rn(t, w);
        if (below_pos_bits(v, w)) {
            c -= 1;
            t = v;
        } else {
            t = 0.0;
        }
    } else if (!below_pos_bits(t, w)) {
        t = __dsub_rn(t, w);
        c += 1;
        if (!below_pos_bits(t, w)) t = w_below;
    }
    c_out = wrap_cell(c, m);
    u_out = t;
}

__device__ __forceinline__ void frame_change_fixed(int32_t d, int32_t W, int m, int c, int32_t u,
                                                   int& c_out, int32_t& u_out) {
    int32_t t = u + d;
    if (t < 0) {
        t += W;
        c -= 1;
    } else if (t >= W) {
        t -= W;
        c += 1;
    }
    c_out = wrap_cell(c, m);
    u_out = t;
}

}  // namespace hd
