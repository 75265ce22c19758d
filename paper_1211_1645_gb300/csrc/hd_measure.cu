// hd_measure.cu -- measurements on the MPMC cell frame (Engel et al.,
// arXiv:1211.1645): the contact-shell pair histogram and the contact-value
// pressure (Sec. II.C.1, Eqs. 2 and 4), and the local / global
// bond-orientational order psi_6 (Sec. III, Eq. 8).
//
// Pair vectors are formed in the cell frame: for disks i and j whose cells
// differ by (dcx, dcy), r = (u_j + dcx * w) - u_i, which is exact in the
// fixed-point form and has one fixed rounding order in FP64.
#include <mutex>
#include <type_traits>

#include "hd_kernels.h"

namespace hd {

template <bool FIX>
using P2 = std::conditional_t<FIX, int2, double2>;

constexpr int kMaxFitBins = 512;

// ---------------------------------------------------------------------------
// Contact-shell histogram: unordered pairs with 2 <= r < 2 + K dr, binned by
// comparing r^2 with squared bin edges; each pair is counted once, from its
// lower id (k_hist_global; the FP64 form of k_hist_tile) or, in the fixed
// form of k_hist_tile, from the upper half of the stencil (the same exact
// squared distance from either side, so the same counts).
// One thread per cell scans the (2R+1)^2 stencil; counts gather in a shared
// histogram and are flushed with one atomic per non-empty bin and block.
// k_hist_global reads the stencil from global memory (any reach R);
// k_hist_tile (reach up to kHistMaxHalo) first stages the block's 32 x rows
// tile of cells and a halo of R cells in shared memory, like k_psi6.
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_hist_global(const Rep* __restrict__ reps, int R, int K, const double* __restrict__ edges,
       const long long* __restrict__ edgesF, const uint8_t* __restrict__ cnt, const P2<FIX>* __restrict__ pos,
       const int32_t* __restrict__ pid, unsigned long long* __restrict__ hist) {
    extern __shared__ unsigned int s_bins[];
    pdl_begin();
    for (int b = threadIdx.x; b < K; b += blockDim.x) s_bins[b] = 0u;
    __syncthreads();
    const int r = find_rep<kGridCell>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int64_t a = int64_t(blockIdx.x - rep.blk_cell) * blockDim.x + threadIdx.x;
    if (a < int64_t(m) * m) {
        int cx, cy;
        cell_coords(rep, a, cx, cy);
        const int64_t cell = rep.cell_off + a;
        const int n = min(int(cnt[cell]), CAP);
        const int RR = rep.hist_R;
        const double e0 = edges[0], eK = edges[K];
        const long long f0 = edgesF[0], fK = edgesF[K];
        for (int k = 0; k < n; ++k) {
            const P2<FIX> me = pos[k * rep.stride + cell];
            const int32_t idme = pid[k * rep.stride + cell];
            for (int dcy = -RR; dcy <= RR; ++dcy) {
                for (int dcx = -RR; dcx <= RR; ++dcx) {
                    const int64_t nc = cell_index(rep, wrap_cell(cx + dcx, m), wrap_cell(cy + dcy, m));
                    const int nn = min(int(cnt[nc]), CAP);
                    for (int q = 0; q < nn; ++q) {
                        const int32_t idq = pid[q * rep.stride + nc];
                        if (idq <= idme) continue;
                        const P2<FIX> o = pos[q * rep.stride + nc];
                        int bin;
                        if constexpr (FIX) {
                            const long long rx = (static_cast<long long>(o.x) + static_cast<long long>(dcx) * rep.W) - me.x;
                            const long long ry = (static_cast<long long>(o.y) + static_cast<long long>(dcy) * rep.W) - me.y;
                            const long long r2 = rx * rx + ry * ry;
                            if (r2 < f0 || r2 >= fK) continue;
                            int lo = 0, hi = K - 1;  // largest k with edgesF[k] <= r2
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (__ldg(&edgesF[mid]) <= r2) lo = mid; else hi = mid - 1;
                            }
                            bin = lo;
                        } else {
                            const double rx = __dsub_rn(__dadd_rn(o.x, __dmul_rn(double(dcx), rep.w)), me.x);
                            const double ry = __dsub_rn(__dadd_rn(o.y, __dmul_rn(double(dcy), rep.w)), me.y);
                            const double r2 = __dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry));
                            if (r2 < e0 || r2 >= eK) continue;
                            int lo = 0, hi = K - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (__ldg(&edges[mid]) <= r2) lo = mid; else hi = mid - 1;
                            }
                            bin = lo;
                        }
                        atomicAdd(&s_bins[bin], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < K; b += blockDim.x)
        if (s_bins[b]) atomicAdd(&hist[size_t(r) * K + b], (unsigned long long)s_bins[b]);
}


constexpr int kHistMaxHalo = 4;

// The disks of a block's 32 x rows tile of cells as one list, so that every
// lane works on one disk (a lane per cell would make a warp repeat its scan
// as many times as its most crowded cell holds disks).  Entry: staged cell
// index << 4 | slot, in tile-cell order.  s_list holds blockDim * CAP
// entries, s_warp one int per warp.  Returns the number of disks; every
// thread of the block must call it, after the staging barrier.
__device__ __forceinline__ int tile_disk_list(const uint8_t* s_n, int SX, int halo, int X0, int Y0, int m,
                                              uint16_t* s_list, int* s_warp) {
    const int lx = int(threadIdx.x & 31u), ly = int(threadIdx.x >> 5);
    const int own = (ly + halo) * SX + lx + halo;
    const int n = (X0 + lx < m && Y0 + ly < m) ? int(s_n[own]) : 0;
    int v = n;  // inclusive warp scan of the occupancies
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lx >= o) v += u;
    }
    if (lx == 31) s_warp[ly] = v;
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
        const int t = s_warp[w];
        base += w < ly ? t : 0;
        total += t;
    }
    const int off = base + v - n;
    for (int q = 0; q < n; ++q) s_list[off + q] = uint16_t((own << 4) | q);
    __syncthreads();
    return total;
}

template <bool FIX, int CAP>
__host__ __device__ constexpr size_t hist_stage_bytes(int rows, int halo, int K) {
    return size_t(32 + 2 * halo) * size_t(rows + 2 * halo) * (CAP * (sizeof(P2<FIX>) + sizeof(int32_t)) + 1) + 16 +
           size_t(K + 1) * 8 + size_t(K) * 4;
}

// FP64 bin of a pair (o at cell offset (dcx, dcy) from me) among the K bins
// of squared edges edge[0..K], or -1 outside [edge_0, edge_K).  Out of line,
// so that its FP64 instructions issue only for the pairs the float pre-test
// leaves; the non-negative squared distance is compared through its bit
// pattern, which orders as the value does.
static __device__ __noinline__ int hist_bin_fp64(double ox, double oy, double mx, double my, int dcx, int dcy,
                                                 double w, const double* edge, int K) {
    const double rx = __dsub_rn(__dadd_rn(ox, __dmul_rn(double(dcx), w)), mx);
    const double ry = __dsub_rn(__dadd_rn(oy, __dmul_rn(double(dcy), w)), my);
    const long long b = __double_as_longlong(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)));
    if (b < __double_as_longlong(edge[0]) || b >= __double_as_longlong(edge[K])) return -1;
    int lo = 0, hi = K - 1;  // largest k with edge[k] <= r^2
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__double_as_longlong(edge[mid]) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool FIX, int CAP>
__global__ void __launch_bounds__(256)
k_hist_tile(const Rep* __restrict__ reps, int R, int K, const double* __restrict__ edges,
            const long long* __restrict__ edgesF, const uint8_t* __restrict__ cnt, const P2<FIX>* __restrict__ pos,
            const int32_t* __restrict__ pid, unsigned long long* __restrict__ hist, int H) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    pdl_begin();
    const int r = find_rep<kGridT32>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int rows = int(blockDim.x >> 5);
    int X0, Y0;
    tile32_origin(rep, uint32_t(blockIdx.x - rep.blk_t32), rows, X0, Y0);
    const int SX = 32 + 2 * H, nS = SX * (rows + 2 * H);
    P2<FIX>* s_pos = reinterpret_cast<P2<FIX>*>(s_raw);                  // [CAP][nS]
    int32_t* s_id = reinterpret_cast<int32_t*>(s_pos + size_t(CAP) * nS);  // [CAP][nS]
    uint8_t* s_n = reinterpret_cast<uint8_t*>(s_id + size_t(CAP) * nS);    // [nS]
    using E = std::conditional_t<FIX, long long, double>;
    E* s_edge = reinterpret_cast<E*>(s_raw + ((size_t(CAP) * nS * (sizeof(P2<FIX>) + 4) + nS + 15) & ~size_t(15)));
    unsigned int* s_bins = reinterpret_cast<unsigned int*>(s_edge + (K + 1));
    for (int b = threadIdx.x; b <= K; b += blockDim.x) {
        if constexpr (FIX) s_edge[b] = edgesF[b];
        else s_edge[b] = edges[b];
        if (b < K) s_bins[b] = 0u;
    }
    for (int t = threadIdx.x; t < nS; t += blockDim.x) {
        const int sy = t / SX, sx = t - sy * SX;
        const uint32_t c = uint32_t(rep.coff) + row_part(rep, wrap_cell(Y0 - H + sy, m)) +
                           col_part(rep, wrap_cell(X0 - H + sx, m));
        const int n = min(int(cnt[c]), CAP);
        s_n[t] = uint8_t(n);
        for (int q = 0; q < n; ++q) {
            s_pos[q * nS + t] = pos[size_t(q) * rep.stride32 + c];
            s_id[q * nS + t] = pid[size_t(q) * rep.stride32 + c];
        }
    }
    __syncthreads();
    __shared__ uint16_t s_list[256 * CAP];
    __shared__ int s_warp[8];
    const int D = tile_disk_list(s_n, SX, H, X0, Y0, m, s_list, s_warp);
    const int RR = rep.hist_R;
    const E lo_edge = s_edge[0], hi_edge = s_edge[K];
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const int own = int(s_list[d] >> 4), k = int(s_list[d] & 15u);
        const P2<FIX> me = s_pos[k * nS + own];
        const int32_t idme = FIX ? 0 : s_id[k * nS + own];  // the FP64 form's pair rule
        float mfx = 0.0f, mfy = 0.0f;  // FP64 form: float images of the disk's offsets
        if constexpr (!FIX) {
            mfx = approx_f32(me.x);
            mfy = approx_f32(me.y);
        }
        // Each unordered pair once.  Fixed form: from the cell whose offset to
        // the other is in the upper half of the stencil (dcy > 0, or dcy = 0
        // and dcx > 0), or within a cell from the lower slot -- the squared
        // distance is the same exact integer seen from either side, so the
        // counts equal those of a lower-id rule.  FP64: from the lower id,
        // whose rounding the oracle follows.
        for (int dcy = FIX ? 0 : -RR; dcy <= RR; ++dcy) {
            for (int dcx = (FIX && dcy == 0) ? 0 : -RR; dcx <= RR; ++dcx) {
                const int sc = own + dcy * SX + dcx;
                const int nn = s_n[sc];
                for (int q = (FIX && dcy == 0 && dcx == 0) ? k + 1 : 0; q < nn; ++q) {
                    if constexpr (!FIX) {
                        if (s_id[q * nS + sc] <= idme) continue;
                    }
                    const P2<FIX> o = s_pos[q * nS + sc];
                    E r2 = E(0);
                    if constexpr (FIX) {
                        // |offset| < (RR + 1) W <= 5 W < 2^31
                        const int32_t rx = (o.x + dcx * rep.W) - me.x;
                        const int32_t ry = (o.y + dcy * rep.W) - me.y;
                        r2 = int64_t(rx) * rx + int64_t(ry) * ry;
                    } else {
                        // float pre-test (as pair_clear's): a pair whose float
                        // estimate of r^2 lies outside the range widened by its
                        // error bound is outside it in FP64 too
                        const float sx = __fsub_rn(__fadd_rn(approx_f32(o.x), __fmul_rn(float(dcx), rep.wf)), mfx);
                        const float sy = __fsub_rn(__fadd_rn(approx_f32(o.y), __fmul_rn(float(dcy), rep.wf)), mfy);
                        const float d2f = __fadd_rn(__fmul_rn(sx, sx), __fmul_rn(sy, sy));
                        if (d2f < rep.h_lo || d2f >= rep.h_hi) continue;
                        const int bin = hist_bin_fp64(o.x, o.y, me.x, me.y, dcx, dcy, rep.w, s_edge, K);
                        if (bin >= 0) atomicAdd(&s_bins[bin], 1u);
                        continue;
                    }
                    if (r2 < lo_edge || r2 >= hi_edge) continue;
                    int lo = 0, hi = K - 1;  // largest k with edge[k] <= r2
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_edge[mid] <= r2) lo = mid; else hi = mid - 1;
                    }
                    atomicAdd(&s_bins[lo], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < K; b += blockDim.x)
        if (s_bins[b]) atomicAdd(&hist[size_t(r) * K + b], (unsigned long long)s_bins[b]);
}

// ---------------------------------------------------------------------------
// g(r) normalisation (Eq. 2, p = N^2 / 2), least-squares quartic in
// t = (r - 2 sigma) / (K dr) by Householder QR, value at contact, and the
// contact-value pressure (Eq. 4).  The design matrix depends on K alone, so
// k_fit_factor triangularises it once per context and k_fit applies the
// stored reflectors to each measurement's g(r): the same operations, in the
// same order, as a factorisation of [A | b] at every measurement.  One warp
// per replica: the K rows are spread over the lanes and every column norm
// and dot product is a warp sum.
// Factor layout: [0, 5K) the K x 5 matrix row-major after triangularisation
// (R on and above the diagonal, reflector j's tail below it); [5K, 5K + 5)
// v0_j, the first element of reflector j; [5K + 5, 5K + 10) v_j^T v_j, 0 for a
// column with zero norm (no reflector).
// res[4r + 0..3] = beta P / rho, g(2 sigma+), P* = beta P (2 sigma)^2, eta.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__global__ void __launch_bounds__(32) k_fit_factor(int K, double* __restrict__ qr) {
    __shared__ double A[kMaxFitBins * 5];
    const int lane = threadIdx.x;
    for (int k = lane; k < K; k += 32) {
        const double t = __ddiv_rn(__dadd_rn(double(k), 0.5), double(K));
        double tp = 1.0;
        for (int q = 0; q < 5; ++q) {
            A[k * 5 + q] = tp;
            tp = __dmul_rn(tp, t);
        }
    }
    __syncwarp();
    for (int j = 0; j < 5; ++j) {
        double part = 0.0;
        for (int i = j + lane; i < K; i += 32) part = __dadd_rn(part, __dmul_rn(A[i * 5 + j], A[i * 5 + j]));
        const double nrm2 = warp_sum(part);
        const double nrm = sqrt(nrm2);
        if (nrm == 0.0) {
            if (lane == 0) {
                qr[5 * K + j] = 0.0;
                qr[5 * K + 5 + j] = 0.0;
            }
            continue;
        }
        const double ajj = A[j * 5 + j];
        const double alpha = ajj > 0.0 ? -nrm : nrm;
        const double v0 = __dsub_rn(ajj, alpha);
        const double vtv = __dadd_rn(__dsub_rn(nrm2, __dmul_rn(ajj, ajj)), __dmul_rn(v0, v0));
        __syncwarp();
        if (lane == 0) A[j * 5 + j] = v0;  // v = (v0, A[j+1.., j])
        __syncwarp();
        for (int q = j + 1; q < 5; ++q) {
            double dp = 0.0;
            for (int i = j + lane; i < K; i += 32) dp = __dadd_rn(dp, __dmul_rn(A[i * 5 + j], A[i * 5 + q]));
            const double sc = __ddiv_rn(__dmul_rn(2.0, warp_sum(dp)), vtv);
            for (int i = j + lane; i < K; i += 32) A[i * 5 + q] = __dsub_rn(A[i * 5 + q], __dmul_rn(sc, A[i * 5 + j]));
            __syncwarp();
        }
        if (lane == 0) {
            A[j * 5 + j] = alpha;  // R diagonal
            qr[5 * K + j] = v0;
            qr[5 * K + 5 + j] = vtv;
        }
        __syncwarp();
    }
    for (int i = lane; i < 5 * K; i += 32) qr[i] = A[i];
}

__global__ void __launch_bounds__(32) k_fit(const Rep* __restrict__ reps, int K, const double* __restrict__ qr,
                                            const unsigned long long* __restrict__ hist, double* __restrict__ res) {
    pdl_begin();
    __shared__ double b[kMaxFitBins];
    const int r = blockIdx.x, lane = threadIdx.x;
    const Rep& rep = reps[r];
    const double PI = 3.14159265358979323846;
    const double V = __dmul_rn(rep.Lm, rep.Lm);
    const double p = __dmul_rn(__dmul_rn(double(rep.N), double(rep.N)), 0.5);
    const double dr = rep.dr;
    for (int k = lane; k < K; k += 32) {
        const double rk = __dadd_rn(2.0, __dmul_rn(__dadd_rn(double(k), 0.5), dr));
        const double shell = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, PI), rk), dr), V);
        b[k] = __ddiv_rn(__ddiv_rn(double(hist[size_t(r) * K + k]), p), shell);
    }
    __syncwarp();
    // b <- Q^T b, reflector by reflector
    for (int j = 0; j < 5; ++j) {
        const double vtv = qr[5 * K + 5 + j];
        if (vtv == 0.0) continue;
        const double v0 = qr[5 * K + j];
        double dp = 0.0;
        for (int i = j + lane; i < K; i += 32) dp = __dadd_rn(dp, __dmul_rn(i == j ? v0 : qr[i * 5 + j], b[i]));
        const double sc = __ddiv_rn(__dmul_rn(2.0, warp_sum(dp)), vtv);
        for (int i = j + lane; i < K; i += 32) b[i] = __dsub_rn(b[i], __dmul_rn(sc, i == j ? v0 : qr[i * 5 + j]));
        __syncwarp();
    }
    if (lane != 0) return;
    double coef[5];
    for (int j = 4; j >= 0; --j) {
        double acc = b[j];
        for (int q = j + 1; q < 5; ++q) acc = __dsub_rn(acc, __dmul_rn(qr[j * 5 + q], coef[q]));
        coef[j] = __ddiv_rn(acc, qr[j * 5 + j]);
    }
    const double g0 = coef[0];
    const double eta = __ddiv_rn(__dmul_rn(double(rep.N), PI), V);
    const double bp = __dadd_rn(1.0, __dmul_rn(__dmul_rn(2.0, eta), g0));
    res[4 * r + 0] = bp;
    res[4 * r + 1] = g0;
    res[4 * r + 2] = __dmul_rn(__dmul_rn(bp, 4.0), __ddiv_rn(double(rep.N), V));
    res[4 * r + 3] = eta;
}

// ---------------------------------------------------------------------------
// psi_6: six nearest neighbours by (r^2, id) from an expanding ring of cells
// (first the 5 x 5 stencil, then one ring more while the sixth neighbour is
// not strictly closer than the nearest point outside the scanned cells).
// exp(6 i phi) = z^6 / |z|^6, z = rx + i ry, summed in ascending (r^2, id).
// ---------------------------------------------------------------------------
template <bool FIX>
struct Nbr {
    // squared distances: exact integers (fixed form), or the bit patterns of
    // the non-negative FP64 values, which order as the values do (so the
    // list needs no FP64 comparison)
    using Key = long long;
    // pair offsets: 32-bit in the fixed form (the ring search never reaches
    // (RR + 1) W >= 2^31, so |r| < 2^31)
    using Off = std::conditional_t<FIX, int32_t, double>;
    Key key[6];
    int32_t id[6];
    Off rx[6], ry[6];
    int n;

    __device__ __forceinline__ void insert(Key k, int32_t i, Off x, Off y) {
        if (n == 6 && !(k < key[5] || (k == key[5] && i < id[5]))) return;
        bool done = false;
        const int top = n < 6 ? n : 5;
#pragma unroll
        for (int s = 5; s >= 0; --s) {
            if (!done && s <= top) {
                if (s > 0 && (k < key[s - 1] || (k == key[s - 1] && i < id[s - 1]))) {
                    key[s] = key[s - 1];
                    id[s] = id[s - 1];
                    rx[s] = rx[s - 1];
                    ry[s] = ry[s - 1];
                } else {
                    key[s] = k;
                    id[s] = i;
                    rx[s] = x;
                    ry[s] = y;
                    done = true;
                }
            }
        }
        if (n < 6) ++n;
    }
};

template <bool FIX, int CAP>
__device__ __forceinline__ void scan_cell(const Rep& rep, const uint8_t* __restrict__ cnt, const P2<FIX>* __restrict__ pos,
                                          const int32_t* __restrict__ pid, int cx, int cy, int dcx, int dcy,
                                          const P2<FIX>& me, int32_t idme, Nbr<FIX>& nb) {
    const int m = rep.m;
    const int64_t nc = cell_index(rep, wrap_cell(cx + dcx, m), wrap_cell(cy + dcy, m));
    const int nn = min(int(cnt[nc]), CAP);
    for (int q = 0; q < nn; ++q) {
        const int32_t idq = pid[q * rep.stride + nc];
        if (idq == idme) continue;
        const P2<FIX> o = pos[q * rep.stride + nc];
        if constexpr (FIX) {
            const int32_t rx = (o.x + dcx * rep.W) - me.x;
            const int32_t ry = (o.y + dcy * rep.W) - me.y;
            nb.insert(int64_t(rx) * rx + int64_t(ry) * ry, idq, rx, ry);
        } else {
            const double rx = __dsub_rn(__dadd_rn(o.x, __dmul_rn(double(dcx), rep.w)), me.x);
            const double ry = __dsub_rn(__dadd_rn(o.y, __dmul_rn(double(dcy), rep.w)), me.y);
            nb.insert(__double_as_longlong(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry))), idq, rx, ry);
        }
    }
}

// Cover test of the ring search: the sixth neighbour is strictly closer than
// any point outside the (2 RR + 1)^2 cells around the disk's cell.
template <bool FIX>
__device__ __forceinline__ bool ring_covers(const Rep& rep, const Nbr<FIX>& nb, const P2<FIX>& me, int RR) {
    if (nb.n < 6) return false;
    if constexpr (FIX) {
        long long cv = static_cast<long long>(me.x) + static_cast<long long>(RR) * rep.W;
        const long long c2 = static_cast<long long>(RR + 1) * rep.W - me.x;
        const long long c3 = static_cast<long long>(me.y) + static_cast<long long>(RR) * rep.W;
        const long long c4 = static_cast<long long>(RR + 1) * rep.W - me.y;
        cv = c2 < cv ? c2 : cv;
        cv = c3 < cv ? c3 : cv;
        cv = c4 < cv ? c4 : cv;
        return nb.key[5] < cv * cv;
    } else {
        double cv = __dadd_rn(me.x, __dmul_rn(double(RR), rep.w));
        const double c2 = __dsub_rn(__dmul_rn(double(RR + 1), rep.w), me.x);
        const double c3 = __dadd_rn(me.y, __dmul_rn(double(RR), rep.w));
        const double c4 = __dsub_rn(__dmul_rn(double(RR + 1), rep.w), me.y);
        cv = c2 < cv ? c2 : cv;
        cv = c3 < cv ? c3 : cv;
        cv = c4 < cv ? c4 : cv;
        return nb.key[5] < __double_as_longlong(__dmul_rn(cv, cv));
    }
}

// Shared-memory copy of the cells a psi_6 block reads: its 32 x rows tile of
// cells plus a halo of two cells (the 5 x 5 stencil of every tile cell).
constexpr int kPsiHalo = 2;
constexpr int kPsiSX = 32 + 2 * kPsiHalo;

template <bool FIX, int CAP>
__host__ __device__ constexpr size_t psi6_stage_bytes(int rows) {
    return size_t(kPsiSX) * size_t(rows + 2 * kPsiHalo) * (CAP * (sizeof(P2<FIX>) + sizeof(int32_t)) + 1);
}

// psi_6 of every disk.  A block stages its tile and halo in shared memory in
// one cooperative round of loads; each disk then scans its 5 x 5 stencil
// there, nearest cells first (so the six-neighbour list fills early and most
// later candidates are rejected by one comparison).  The rare disk whose six
// neighbours are not certified by the 5 x 5 stencil (low density) continues
// the ring search in global memory.
// Registers per thread: the fixed form runs at four blocks of 256 per SM
// (64 registers, a few spilled, 0.238 -> 0.211 ms at N = 1M: more resident
// warps hide the insertion's dependency chains); the FP64 form at 118
// registers (no spill).
template <bool FIX, int CAP>
__global__ void __launch_bounds__(256, FIX ? 4 : 1)
k_psi6(const Rep* __restrict__ reps, int R, const uint8_t* __restrict__ cnt, const P2<FIX>* __restrict__ pos,
       const int32_t* __restrict__ pid, double2* __restrict__ local, ExactPair* __restrict__ partial,
       int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    pdl_begin();
    const int r = find_rep<kGridT32>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int rows = int(blockDim.x >> 5);
    int X0, Y0;
    tile32_origin(rep, uint32_t(blockIdx.x - rep.blk_t32), rows, X0, Y0);
    const int nS = kPsiSX * (rows + 2 * kPsiHalo);
    P2<FIX>* s_pos = reinterpret_cast<P2<FIX>*>(s_raw);                  // [CAP][nS]
    int32_t* s_id = reinterpret_cast<int32_t*>(s_pos + size_t(CAP) * nS);  // [CAP][nS]
    uint8_t* s_n = reinterpret_cast<uint8_t*>(s_id + size_t(CAP) * nS);    // [nS]
    for (int t = threadIdx.x; t < nS; t += blockDim.x) {
        const int sy = t / kPsiSX, sx = t - sy * kPsiSX;
        const uint32_t c = uint32_t(rep.coff) + row_part(rep, wrap_cell(Y0 - kPsiHalo + sy, m)) +
                           col_part(rep, wrap_cell(X0 - kPsiHalo + sx, m));
        const int n = min(int(cnt[c]), CAP);
        s_n[t] = uint8_t(n);
        for (int q = 0; q < n; ++q) {
            s_pos[q * nS + t] = pos[size_t(q) * rep.stride32 + c];
            s_id[q * nS + t] = pid[size_t(q) * rep.stride32 + c];
        }
    }
    __syncthreads();

    __shared__ uint16_t s_list[256 * CAP];
    __shared__ int s_warp[8];
    const int D = tile_disk_list(s_n, kPsiSX, kPsiHalo, X0, Y0, m, s_list, s_warp);
    Exact192 sr = exact_zero(), si = exact_zero();  // exact sums of this thread's psi_j
    int rmax = (m - 1) / 2;
    if constexpr (FIX) {
        const int lim = int((int64_t(1) << 31) / rep.W) - 1;
        if (lim < rmax) rmax = lim;
    }
    {
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            const int own = int(s_list[d] >> 4), k = int(s_list[d] & 15u);
            const int sy = own / kPsiSX;
            const int cx = X0 + (own - sy * kPsiSX) - kPsiHalo, cy = Y0 + sy - kPsiHalo;
            const P2<FIX> me = s_pos[k * nS + own];
            const int32_t idme = s_id[k * nS + own];
            float mfx = 0.0f, mfy = 0.0f;  // FP64 form: float images of the disk's offsets
            if constexpr (!FIX) {
                mfx = approx_f32(me.x);
                mfy = approx_f32(me.y);
            }
            Nbr<FIX> nb;
            nb.n = 0;
            bool ok = false;
            if (rmax >= 2) {
                // rings 0, 1, 2 of the staged stencil, nearest first
#pragma unroll 1
                for (int ring = 0; ring <= 2; ++ring) {
                    for (int dcy = -ring; dcy <= ring; ++dcy) {
                        for (int dcx = -ring; dcx <= ring; ++dcx) {
                            if (max(abs(dcx), abs(dcy)) != ring) continue;
                            const int sc = own + dcy * kPsiSX + dcx;
                            const int nn = s_n[sc];
                            for (int q = 0; q < nn; ++q) {
                                const int32_t idq = s_id[q * nS + sc];
                                if (idq == idme) continue;
                                const P2<FIX> o = s_pos[q * nS + sc];
                                if constexpr (FIX) {
                                    const int32_t rx = (o.x + dcx * rep.W) - me.x;
                                    const int32_t ry = (o.y + dcy * rep.W) - me.y;
                                    nb.insert(int64_t(rx) * rx + int64_t(ry) * ry, idq, rx, ry);
                                } else {
                                    if (nb.n == 6) {
                                        // float pre-test: a candidate whose float estimate
                                        // of r^2 exceeds the sixth key by more than the
                                        // estimate's error bound is farther in FP64 too
                                        // (approx_f32 truncates; the product rounds up
                                        // past the key itself)
                                        const float sx = __fsub_rn(__fadd_rn(approx_f32(o.x), __fmul_rn(float(dcx), rep.wf)), mfx);
                                        const float sy = __fsub_rn(__fadd_rn(approx_f32(o.y), __fmul_rn(float(dcy), rep.wf)), mfy);
                                        const float d2f = __fadd_rn(__fmul_rn(sx, sx), __fmul_rn(sy, sy));
                                        const float k5 = __fmul_ru(approx_f32(__longlong_as_double(nb.key[5])), 1.0f + 0x1p-19f);
                                        if (d2f > __fadd_ru(k5, rep.psi_m)) continue;
                                    }
                                    const double rx = __dsub_rn(__dadd_rn(o.x, __dmul_rn(double(dcx), rep.w)), me.x);
                                    const double ry = __dsub_rn(__dadd_rn(o.y, __dmul_rn(double(dcy), rep.w)), me.y);
                                    nb.insert(__double_as_longlong(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry))), idq, rx, ry);
                                }
                            }
                        }
                    }
                }
                ok = ring_covers<FIX>(rep, nb, me, 2);
            }
            for (int RR = 3; RR <= rmax && !ok; ++RR) {
                for (int e = -RR; e <= RR; ++e) {
                    scan_cell<FIX, CAP>(rep, cnt, pos, pid, cx, cy, e, -RR, me, idme, nb);
                    scan_cell<FIX, CAP>(rep, cnt, pos, pid, cx, cy, e, RR, me, idme, nb);
                }
                for (int e = -RR + 1; e <= RR - 1; ++e) {
                    scan_cell<FIX, CAP>(rep, cnt, pos, pid, cx, cy, -RR, e, me, idme, nb);
                    scan_cell<FIX, CAP>(rep, cnt, pos, pid, cx, cy, RR, e, me, idme, nb);
                }
                ok = ring_covers<FIX>(rep, nb, me, RR);
            }
            double pre, pim;
            if (!ok) {
                atomicOr(err, 2);
                pre = pim = 0.0;
            } else if constexpr (FIX) {
                float fr = 0.0f, fi = 0.0f;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const float x = __fmul_rn(__int2float_rn(nb.rx[q]), 0x1p-24f);
                    const float y = __fmul_rn(__int2float_rn(nb.ry[q]), 0x1p-24f);
                    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y);
                    const float r2 = __fadd_rn(xx, yy);
                    const float c2 = __fsub_rn(xx, yy), s2 = __fmul_rn(__fmul_rn(x, y), 2.0f);
                    const float c4 = __fsub_rn(__fmul_rn(c2, c2), __fmul_rn(s2, s2));
                    const float s4 = __fmul_rn(__fmul_rn(c2, s2), 2.0f);
                    const float c6 = __fsub_rn(__fmul_rn(c4, c2), __fmul_rn(s4, s2));
                    const float s6 = __fadd_rn(__fmul_rn(c4, s2), __fmul_rn(s4, c2));
                    const float r6 = __fmul_rn(__fmul_rn(r2, r2), r2);
                    fr = __fadd_rn(fr, __fdiv_rn(c6, r6));
                    fi = __fadd_rn(fi, __fdiv_rn(s6, r6));
                }
                pre = double(__fdiv_rn(fr, 6.0f));
                pim = double(__fdiv_rn(fi, 6.0f));
            } else {
                double dr_ = 0.0, di = 0.0;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const double x = nb.rx[q], y = nb.ry[q];
                    const double xx = __dmul_rn(x, x), yy = __dmul_rn(y, y);
                    const double r2 = __dadd_rn(xx, yy);
                    const double c2 = __dsub_rn(xx, yy), s2 = __dmul_rn(__dmul_rn(x, y), 2.0);
                    const double c4 = __dsub_rn(__dmul_rn(c2, c2), __dmul_rn(s2, s2));
                    const double s4 = __dmul_rn(__dmul_rn(c2, s2), 2.0);
                    const double c6 = __dsub_rn(__dmul_rn(c4, c2), __dmul_rn(s4, s2));
                    const double s6 = __dadd_rn(__dmul_rn(c4, s2), __dmul_rn(s4, c2));
                    const double r6 = __dmul_rn(__dmul_rn(r2, r2), r2);
                    dr_ = __dadd_rn(dr_, __ddiv_rn(c6, r6));
                    di = __dadd_rn(di, __ddiv_rn(s6, r6));
                }
                pre = __ddiv_rn(dr_, 6.0);
                pim = __ddiv_rn(di, 6.0);
            }
            if (local) local[rep.id_off + idme] = make_double2(pre, pim);
            exact_add(sr, pre);
            exact_add(si, pim);
        }
    }
    // block sum: exact, so its value does not depend on the order of the disks
    const ExactPair t = exact_block_sum(sr, si);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Psi_6 of each replica: the exact sum of its block partials rounded once to
// double, then divided by N (the oracle's order of operations).
__global__ void k_psi6_reduce(const Rep* __restrict__ reps, int R, int blocks_total,
                              const ExactPair* __restrict__ partial, double* __restrict__ res) {
    pdl_begin();
    const int r = blockIdx.x;
    const Rep& rep = reps[r];
    const int b0 = rep.blk_t32;
    const int b1 = (r + 1 < R) ? reps[r + 1].blk_t32 : blocks_total;
    Exact192 sr = exact_zero(), si = exact_zero();
    for (int b = b0 + int(threadIdx.x); b < b1; b += blockDim.x) {
        exact_merge(sr, partial[b].re);
        exact_merge(si, partial[b].im);
    }
    const ExactPair t = exact_block_sum(sr, si);
    if (threadIdx.x == 0) {
        res[2 * r] = __ddiv_rn(exact_round(t.re), double(rep.N));
        res[2 * r + 1] = __ddiv_rn(exact_round(t.im), double(rep.N));
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <bool FIX, int CAP>
static cudaError_t hist_t(const LaunchCfg& c, const HistCfg& h, CellBufs cells, unsigned long long* hist) {
    if (h.halo <= kHistMaxHalo) {
        static std::once_flag attr_once;
        std::call_once(attr_once, [] {
            cudaFuncSetAttribute(k_hist_tile<FIX, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(hist_stage_bytes<FIX, CAP>(8, kHistMaxHalo, kMaxFitBins)));
        });
        return launch_k(k_hist_tile<FIX, CAP>, dim3(c.blocks_t32), dim3(c.threads),
                        hist_stage_bytes<FIX, CAP>(c.threads / 32, h.halo, h.K), c.stream, c.reps, c.R, h.K, h.edges,
                        h.edgesF, (const uint8_t*)cells.cnt, (const P2<FIX>*)cells.pos, (const int32_t*)cells.pid,
                        hist, h.halo);
    }
    return launch_k(k_hist_global<FIX, CAP>, dim3(c.blocks_cell), dim3(c.threads), size_t(h.K) * sizeof(unsigned int),
                    c.stream, c.reps, c.R, h.K, h.edges, h.edgesF, (const uint8_t*)cells.cnt,
                    (const P2<FIX>*)cells.pos, (const int32_t*)cells.pid, hist);
}

cudaError_t launch_hist(const LaunchCfg& c, const HistCfg& h, CellBufs cells, unsigned long long* hist) {
    if (c.fixed) return c.cap == 4 ? hist_t<true, 4>(c, h, cells, hist) : hist_t<true, 9>(c, h, cells, hist);
    return c.cap == 4 ? hist_t<false, 4>(c, h, cells, hist) : hist_t<false, 9>(c, h, cells, hist);
}

size_t fit_factor_len(int K) { return size_t(5 * K + 10); }

cudaError_t launch_fit_factor(cudaStream_t s, int K, double* qr) {
    if (K < 5 || K > kMaxFitBins) return cudaErrorInvalidValue;
    k_fit_factor<<<1, 32, 0, s>>>(K, qr);
    return cudaGetLastError();
}

cudaError_t launch_fit(const LaunchCfg& c, int K, const double* qr, const unsigned long long* hist, double* res) {
    if (K < 5 || K > kMaxFitBins) return cudaErrorInvalidValue;
    return launch_k(k_fit, dim3(c.R), dim3(32), 0, c.stream, c.reps, K, qr, hist, res);
}

template <bool FIX, int CAP>
static cudaError_t psi6_t(const LaunchCfg& c, CellBufs cells, double2* local, ExactPair* partial, int* err) {
    const size_t smem = psi6_stage_bytes<FIX, CAP>(c.threads / 32);
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_psi6<FIX, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(psi6_stage_bytes<FIX, CAP>(8)));
    });
    return launch_k(k_psi6<FIX, CAP>, dim3(c.blocks_t32), dim3(c.threads), smem, c.stream, c.reps, c.R,
                    (const uint8_t*)cells.cnt, (const P2<FIX>*)cells.pos, (const int32_t*)cells.pid, local, partial,
                    err);
}

cudaError_t launch_psi6(const LaunchCfg& c, CellBufs cells, double2* local, ExactPair* partial, int* err) {
    if (c.fixed) return c.cap == 4 ? psi6_t<true, 4>(c, cells, local, partial, err) : psi6_t<true, 9>(c, cells, local, partial, err);
    return c.cap == 4 ? psi6_t<false, 4>(c, cells, local, partial, err) : psi6_t<false, 9>(c, cells, local, partial, err);
}

__global__ void k_record(int R, const double* __restrict__ fit, const double* __restrict__ psi,
                         double* __restrict__ series, int64_t* __restrict__ len, int64_t cap, int* __restrict__ err) {
    pdl_begin();
    const int64_t idx = *len;
    const int r = threadIdx.x;
    if (r < R && idx < cap) {
        double* row = series + (size_t(idx) * R + r) * 4;
        row[0] = fit[4 * r];
        row[1] = fit[4 * r + 1];
        row[2] = psi[2 * r];
        row[3] = psi[2 * r + 1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (idx < cap) *len = idx + 1;
        else atomicOr(err, 4);
    }
}

cudaError_t launch_record(const LaunchCfg& c, const double* fit, const double* psi, double* series, int64_t* len,
                          int64_t cap, int* err) {
    return launch_k(k_record, dim3(1), dim3(((c.R + 31) / 32) * 32), 0, c.stream, c.R, fit, psi, series, len, cap, err);
}

cudaError_t launch_psi6_reduce(const LaunchCfg& c, const ExactPair* partial, double* res) {
    return launch_k(k_psi6_reduce, dim3(c.R), dim3(1024), 0, c.stream, c.reps, c.R, c.blocks_t32, partial, res);
}

}  // namespace hd
