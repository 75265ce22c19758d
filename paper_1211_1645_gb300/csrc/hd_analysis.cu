// hd_analysis.cu -- analysis of the measured chain (Engel et al.,
// arXiv:1211.1645): the autocorrelation of the global orientational order
// Psi_6 over the recorded measurement series and the correlation time of its
// exponential part (Sec. III, Eq. 9, Table II), and the coarse-grained psi_6
// field, the mean of psi_j over square sampling areas (Sec. IV, Figs. 5-6).
#include <math_constants.h>

#include "hd_kernels.h"

namespace hd {

// Series row layout: series[(t * R + r) * 4 + {0: beta P / rho, 1: g(2 sigma+), 2: Re Psi_6, 3: Im Psi_6}].
//
// S[r][d] = sum_{t < T - d} Psi(t) conj(Psi(t + d)), one thread per lag d.
__global__ void __launch_bounds__(256)
k_acf_sums(const double* __restrict__ series, int R, int64_t T, int64_t max_lag, double2* __restrict__ S) {
    pdl_begin();
    const int r = blockIdx.y;
    const int64_t d = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (d > max_lag) return;
    double sr = 0.0, si = 0.0;
    for (int64_t t = 0; t + d < T; ++t) {
        const double a = series[(size_t(t) * R + r) * 4 + 2], b = series[(size_t(t) * R + r) * 4 + 3];
        const double c = series[(size_t(t + d) * R + r) * 4 + 2], e = series[(size_t(t + d) * R + r) * 4 + 3];
        // (a + i b)(c - i e) = (a c + b e) + i (b c - a e)
        sr = __dadd_rn(sr, __dadd_rn(__dmul_rn(a, c), __dmul_rn(b, e)));
        si = __dadd_rn(si, __dsub_rn(__dmul_rn(b, c), __dmul_rn(a, e)));
    }
    S[size_t(r) * size_t(max_lag + 1) + size_t(d)] = make_double2(sr, si);
}

// Eq. 9: C(d) = (S(d) / (T - d)) / (S(0) / T), in place; one block per
// replica, so S(0) is read by every thread before any thread overwrites it.
__global__ void __launch_bounds__(256)
k_acf_norm(int R, int64_t T, int64_t max_lag, double2* __restrict__ S) {
    pdl_begin();
    double2* row = S + size_t(blockIdx.x) * size_t(max_lag + 1);
    const double den = __ddiv_rn(row[0].x, double(T));
    __syncthreads();
    for (int64_t d = threadIdx.x; d <= max_lag; d += blockDim.x) {
        const double2 s = row[d];
        const double n = double(T - d);
        row[d] = make_double2(__ddiv_rn(__ddiv_rn(s.x, n), den), __ddiv_rn(__ddiv_rn(s.y, n), den));
    }
}

// Correlation time of the exponential part: least-squares line through
// (d, ln Re C(d)) over lag_lo <= d <= lag_hi with Re C > 0, tau = -1 / slope
// (NaN with fewer than two such lags or a slope >= 0).  One thread per replica.
__global__ void k_acf_tau(int R, int64_t max_lag, int64_t lag_lo, int64_t lag_hi, const double2* __restrict__ C,
                          double* __restrict__ tau) {
    pdl_begin();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double2* row = C + size_t(r) * size_t(max_lag + 1);
    double sx = 0.0, sy = 0.0;
    int64_t n = 0;
    for (int64_t d = lag_lo; d <= lag_hi; ++d) {
        if (row[d].x > 0.0) {
            sx = __dadd_rn(sx, double(d));
            sy = __dadd_rn(sy, log(row[d].x));
            ++n;
        }
    }
    double out = CUDART_NAN;
    if (n >= 2) {
        const double mx = __ddiv_rn(sx, double(n)), my = __ddiv_rn(sy, double(n));
        double sxy = 0.0, sxx = 0.0;
        for (int64_t d = lag_lo; d <= lag_hi; ++d) {
            if (row[d].x > 0.0) {
                const double dx = __dsub_rn(double(d), mx);
                sxy = __dadd_rn(sxy, __dmul_rn(dx, __dsub_rn(log(row[d].x), my)));
                sxx = __dadd_rn(sxx, __dmul_rn(dx, dx));
            }
        }
        const double slope = __ddiv_rn(sxy, sxx);
        if (slope < 0.0) out = __ddiv_rn(-1.0, slope);
    }
    tau[r] = out;
}

// Coarse field, accumulation: one thread per disk (global id order), from
// the global positions and the local psi_6 of the same state.  Area index
// floor(x bins / L) per axis (FP64), or floor(X bins / LF) of the exact
// integer coordinate X = x 2^24 (fixed form); acc[r][area] = (sum Re, sum Im, count).
__global__ void __launch_bounds__(256)
k_field_accum(const Rep* __restrict__ reps, int R, int64_t Ntot, bool fixed, int bins, const double* __restrict__ xy,
              const double2* __restrict__ psi, double* __restrict__ acc) {
    pdl_begin();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= Ntot) return;
    int lo = 0, hi = R - 1;  // replica of global id i: last one with id_off <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reps[mid].id_off <= i) lo = mid; else hi = mid - 1;
    }
    const Rep& rep = reps[lo];
    const double x = xy[2 * i], y = xy[2 * i + 1];
    int64_t ix, iy;
    if (fixed) {
        const int64_t X = llrint(__dmul_rn(x, 16777216.0)), Y = llrint(__dmul_rn(y, 16777216.0));
        ix = (X * bins) / rep.LF;
        iy = (Y * bins) / rep.LF;
    } else {
        ix = int64_t(floor(__ddiv_rn(__dmul_rn(x, double(bins)), rep.L)));
        iy = int64_t(floor(__ddiv_rn(__dmul_rn(y, double(bins)), rep.L)));
    }
    ix = ix < bins ? ix : bins - 1;
    iy = iy < bins ? iy : bins - 1;
    double* a = acc + (size_t(lo) * size_t(bins) * size_t(bins) + size_t(iy) * bins + size_t(ix)) * 3;
    const double2 v = psi[i];
    atomicAdd(a + 0, v.x);
    atomicAdd(a + 1, v.y);
    atomicAdd(a + 2, 1.0);
}

// Coarse field, means: out[r][iy][ix] = (sum Re, sum Im) / count, NaN if empty.
__global__ void __launch_bounds__(256)
k_field_norm(int64_t cells, const double* __restrict__ acc, double2* __restrict__ out) {
    pdl_begin();
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double n = acc[3 * c + 2];
    out[c] = n > 0.0 ? make_double2(__ddiv_rn(acc[3 * c], n), __ddiv_rn(acc[3 * c + 1], n))
                     : make_double2(CUDART_NAN, CUDART_NAN);
}

cudaError_t launch_acf(const LaunchCfg& c, const double* series, int64_t T, int64_t max_lag, double2* C) {
    const dim3 grid(unsigned((max_lag + 256) / 256), unsigned(c.R));
    const cudaError_t e = launch_k(k_acf_sums, grid, dim3(256), 0, c.stream, series, c.R, T, max_lag, C);
    if (e != cudaSuccess) return e;
    return launch_k(k_acf_norm, dim3(unsigned(c.R)), dim3(256), 0, c.stream, c.R, T, max_lag, C);
}

cudaError_t launch_acf_tau(const LaunchCfg& c, int64_t max_lag, int64_t lag_lo, int64_t lag_hi, const double2* C,
                           double* tau) {
    return launch_k(k_acf_tau, dim3(unsigned((c.R + 31) / 32)), dim3(32), 0, c.stream, c.R, max_lag, lag_lo, lag_hi,
                    C, tau);
}

cudaError_t launch_field(const LaunchCfg& c, int64_t Ntot, int bins, const double* xy, const double2* psi,
                         double* acc, double2* out) {
    const int64_t cells = int64_t(c.R) * bins * bins;
    cudaError_t e = cudaMemsetAsync(acc, 0, size_t(cells) * 3 * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    e = launch_k(k_field_accum, dim3(unsigned((Ntot + 255) / 256)), dim3(256), 0, c.stream, c.reps, c.R, Ntot,
                 c.fixed, bins, xy, psi, acc);
    if (e != cudaSuccess) return e;
    return launch_k(k_field_norm, dim3(unsigned((cells + 255) / 256)), dim3(256), 0, c.stream, cells,
                    (const double*)acc, out);
}

}  // namespace hd
