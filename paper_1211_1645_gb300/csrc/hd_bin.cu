// hd_bin.cu -- positions given by the caller (hd_set_positions) binned into
// the unshifted cell frame on the device (Engel et al., arXiv:1211.1645,
// Sec. II.B: cell-relative coordinates).
#include "hd_cell.cuh"
#include "hd_kernels.h"
#include "hd_bin.h"

namespace hd {

// ---------------------------------------------------------------------------
// Binning of caller positions into the unshifted cell frame (hd_set_positions):
// one thread per disk, the same arithmetic as the host binning of the
// initial lattice and as the oracle, slots claimed with byte-lane atomics
// (the colour pass orders a cell by id).  Input errors set err bits
// kErrBinOverflow / kErrBinInput and leave the disk out.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_fp64_dev(double t, const Rep& r, int& c, double& u) {
    int cc = int(__ddiv_rn(t, r.w));
    if (cc > r.m - 1) cc = r.m - 1;
    if (cc < 0) cc = 0;
    double uu = __dsub_rn(t, __dmul_rn(double(cc), r.w));
    if (uu < 0.0 && cc > 0) {
        cc -= 1;
        uu = __dsub_rn(t, __dmul_rn(double(cc), r.w));
    }
    if (uu >= r.w && cc < r.m - 1) {
        cc += 1;
        uu = __dsub_rn(t, __dmul_rn(double(cc), r.w));
    }
    if (uu < 0.0) uu = 0.0;
    if (uu >= r.w) uu = r.w_below;
    c = cc;
    u = uu;
}

// floor(X / W) for 0 <= X < 2^53 and 0 < W < 2^31 with a quotient below 2^31:
// a float estimate (relative error below 2^-21, so within one of the
// quotient for quotients below 2^20, and corrected step by step otherwise)
// made exact with integer arithmetic, instead of a 64-bit integer division.
__device__ __forceinline__ int64_t floor_div_pos(int64_t X, int32_t W) {
    int64_t q = int64_t(__fmul_rn(__ll2float_rn(X), __frcp_rn(float(W))));
    int64_t r = X - q * int64_t(W);
    while (r < 0) {
        --q;
        r += W;
    }
    while (r >= int64_t(W)) {
        ++q;
        r -= W;
    }
    return q;
}

template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_bin(const Rep* __restrict__ reps, int R, int64_t Ntot, double sigma, const double* __restrict__ xy,
      uint8_t* __restrict__ cnt, P2<FIX>* __restrict__ pos, int32_t* __restrict__ pid, int* __restrict__ err) {
    pdl_begin();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= Ntot) return;
    int lo = 0, hi = R - 1;  // replica of global id i: last one with id_off <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reps[mid].id_off <= i) lo = mid; else hi = mid - 1;
    }
    const Rep& rep = reps[lo];
    // a division by 1 is exact: skip it (the FP64 pipe is narrow)
    const double px = sigma == 1.0 ? xy[2 * i] : __ddiv_rn(xy[2 * i], sigma);
    const double py = sigma == 1.0 ? xy[2 * i + 1] : __ddiv_rn(xy[2 * i + 1], sigma);
    if (!isfinite(px) || !isfinite(py)) {
        atomicOr(err, kErrBinInput);
        return;
    }
    int cx, cy;
    P2<FIX> q;
    if constexpr (FIX) {
        int64_t X = llround(__dmul_rn(px, 16777216.0));
        int64_t Y = llround(__dmul_rn(py, 16777216.0));
        // wrapped into [0, LF); a coordinate already inside needs no division
        if (X < 0 || X >= rep.LF) {
            X %= rep.LF;
            if (X < 0) X += rep.LF;
        }
        if (Y < 0 || Y >= rep.LF) {
            Y %= rep.LF;
            if (Y < 0) Y += rep.LF;
        }
        cx = int(floor_div_pos(X, rep.W));
        cy = int(floor_div_pos(Y, rep.W));
        q.x = int32_t(X - int64_t(cx) * rep.W);
        q.y = int32_t(Y - int64_t(cy) * rep.W);
    } else {
        // fmod returns a coordinate already in [0, L) unchanged
        double x = (px >= 0.0 && px < rep.L) ? px : fmod(px, rep.L);
        double y = (py >= 0.0 && py < rep.L) ? py : fmod(py, rep.L);
        if (x < 0.0) x = __dadd_rn(x, rep.L);
        if (y < 0.0) y = __dadd_rn(y, rep.L);
        if (x >= rep.L) x = 0.0;
        if (y >= rep.L) y = 0.0;
        bin_fp64_dev(x, rep, cx, q.x);
        bin_fp64_dev(y, rep, cy, q.y);
    }
    const uint32_t c = rep.coff + row_part(rep, cy) + col_part(rep, cx);
    const int s = claim_slot(cnt, c);
    if (s >= CAP) {
        atomicOr(err, kErrBinOverflow);
        return;
    }
    pos[size_t(s) * rep.stride32 + c] = q;
    pid[size_t(s) * rep.stride32 + c] = int32_t(i - rep.id_off);
}

template <bool FIX, int CAP>
static cudaError_t bin_t(const LaunchCfg& c, int64_t Ntot, double sigma, const double* xy, CellBufs to, int* err) {
    return launch_k(k_bin<FIX, CAP>, dim3(unsigned((Ntot + 255) / 256)), dim3(256), 0, c.stream, c.reps, c.R, Ntot,
                    sigma, xy, to.cnt, (P2<FIX>*)to.pos, to.pid, err);
}

cudaError_t launch_bin(const LaunchCfg& c, int64_t Ntot, double sigma, const double* xy, CellBufs to, int* err) {
    if (c.fixed) return c.cap == 4 ? bin_t<true, 4>(c, Ntot, sigma, xy, to, err) : bin_t<true, 9>(c, Ntot, sigma, xy, to, err);
    return c.cap == 4 ? bin_t<false, 4>(c, Ntot, sigma, xy, to, err) : bin_t<false, 9>(c, Ntot, sigma, xy, to, err);
}

}  // namespace hd
