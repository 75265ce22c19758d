// hd_analysis.cu -- analysis of the measured chain (Engel et al.,
// arXiv:1211.1645): the autocorrelation of the global orientational order
// Psi_6 over the recorded measurement series and the correlation time of its
// exponential part (Sec. III, Eq. 9, Table II), and the coarse-grained psi_6
// field, the mean of psi_j over square sampling areas (Sec. IV, Figs. 5-6);
// the structure factor, the choice of q_0 at its maximum, the positional
// order chi_j and the positional correlation function (Sec. IV.C, Eqs. 10-12).
#include <math_constants.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hd_kernels.h"
#include "hd_analysis.h"

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
    // xy holds caller units (sigma times the internal ones)
    const double x = __ddiv_rn(xy[2 * i], rep.sigma), y = __ddiv_rn(xy[2 * i + 1], rep.sigma);
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

// ---------------------------------------------------------------------------
// Positional order.  Wave vectors are the box-periodic q = 2 pi (h, k) / L;
// the phase q . x is taken as the turn fraction t = (h x + k y) / L mod 1 --
// exact in the fixed-point form, where x = X 2^-24 and L = LF 2^-24 -- and
// exp(i q . x) = (cospi(2t), sinpi(2t)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 plane_wave(const Rep& rep, bool fixed, int h, int k, double x, double y) {
    double t;
    if (fixed) {
        const int64_t X = llrint(__dmul_rn(x, 16777216.0)), Y = llrint(__dmul_rn(y, 16777216.0));
        int64_t a = (int64_t(h) * X + int64_t(k) * Y) % rep.LF;  // |h X| < 2^17 2^38
        if (a < 0) a += rep.LF;
        t = __ddiv_rn(double(a), double(rep.LF));
    } else {
        t = __ddiv_rn(__dadd_rn(__dmul_rn(double(h), x), __dmul_rn(double(k), y)), rep.Lm);
        t = __dsub_rn(t, floor(t));
    }
    double s, c;
    sincospi(__dmul_rn(2.0, t), &s, &c);
    return make_double2(c, s);
}

// Replica of global disk id i: the last one with id_off <= i.
__device__ __forceinline__ int rep_of_id(const Rep* __restrict__ reps, int R, int64_t i) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reps[mid].id_off <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kSqChunk = 16;  // wave vectors per block of the amplitude kernel

// Amplitudes A_r(q) = sum_n exp(i q . x_n): blockIdx.z = replica, blockIdx.y =
// chunk of wave vectors, blockIdx.x = block of the replica's disks; one
// partial sum per (replica, disk block, q), reduced in a fixed order later.
__global__ void __launch_bounds__(256)
k_sq_amp(const Rep* __restrict__ reps, bool fixed, int nq, const int2* __restrict__ hk, const double* __restrict__ xy,
         int nbx, double2* __restrict__ part) {
    pdl_begin();
    const int r = blockIdx.z;
    const Rep& rep = reps[r];
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool live = i < rep.N;
    const double x = live ? __ddiv_rn(xy[2 * (rep.id_off + i)], rep.sigma) : 0.0;
    const double y = live ? __ddiv_rn(xy[2 * (rep.id_off + i) + 1], rep.sigma) : 0.0;
    __shared__ double s_re[kSqChunk][8], s_im[kSqChunk][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q0 = blockIdx.y * kSqChunk;
    for (int j = 0; j < kSqChunk; ++j) {
        const int q = q0 + j;
        double2 v = make_double2(0.0, 0.0);
        if (live && q < nq) {
            const int2 m = hk[size_t(r) * nq + q];
            v = plane_wave(rep, fixed, m.x, m.y, x, y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
        if (lane == 0) {
            s_re[j][warp] = v.x;
            s_im[j][warp] = v.y;
        }
    }
    __syncthreads();
    if (threadIdx.x < kSqChunk && q0 + int(threadIdx.x) < nq) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            a += s_re[threadIdx.x][w];
            b += s_im[threadIdx.x][w];
        }
        part[(size_t(r) * nbx + blockIdx.x) * nq + q0 + threadIdx.x] = make_double2(a, b);
    }
}

// S_r(q) = |A_r(q)|^2 / N_r (Eq. 10); best[r] = first q of largest S.  One block per replica.
__global__ void __launch_bounds__(256)
k_sq_reduce(const Rep* __restrict__ reps, int nq, int nbx, const double2* __restrict__ part, double* __restrict__ S,
            int* __restrict__ best) {
    pdl_begin();
    const int r = blockIdx.x;
    const Rep& rep = reps[r];
    const int nb = int((rep.N + 255) / 256);
    __shared__ double s_v[256];
    __shared__ int s_i[256];
    double bv = -1.0;
    int bi = 0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int x = 0; x < nb; ++x) {
            const double2 p = part[(size_t(r) * nbx + x) * nq + q];
            a += p.x;
            b += p.y;
        }
        const double v = __ddiv_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), double(rep.N));
        S[size_t(r) * nq + q] = v;
        if (v > bv) {
            bv = v;
            bi = q;
        }
    }
    s_v[threadIdx.x] = bv;
    s_i[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (int(threadIdx.x) < st) {
            const double ov = s_v[threadIdx.x + st];
            const int oi = s_i[threadIdx.x + st];
            if (ov > s_v[threadIdx.x] || (ov == s_v[threadIdx.x] && oi < s_i[threadIdx.x])) {
                s_v[threadIdx.x] = ov;
                s_i[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) best[r] = s_i[0];
}

// Candidate window for q_0 per replica: the (2 hw + 1)^2 box-grid points
// around the first-shell reciprocal vector of a triangular lattice of the
// same density (|q| = 4 pi / (a sqrt 3), area per disk sqrt(3) a^2 / 2) at
// the angle arg(Psi_6) / 6 + 30 degrees.  psi[2r], psi[2r + 1] = Psi_6.
__global__ void k_q0_window(const Rep* __restrict__ reps, int R, int hw, const double* __restrict__ psi,
                            int2* __restrict__ hk) {
    pdl_begin();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const Rep& rep = reps[r];
    const double L = rep.Lm;
    const double eta = __ddiv_rn(__dmul_rn(double(rep.N), CUDART_PI), __dmul_rn(L, L));
    const double rho = __ddiv_rn(eta, CUDART_PI);
    const double a = sqrt(__ddiv_rn(2.0, __dmul_rn(sqrt(3.0), rho)));
    const double qmag = __ddiv_rn(__dmul_rn(4.0, CUDART_PI), __dmul_rn(a, sqrt(3.0)));
    const double th = __dadd_rn(__ddiv_rn(atan2(psi[2 * r + 1], psi[2 * r]), 6.0), __ddiv_rn(CUDART_PI, 6.0));
    const double scale = __ddiv_rn(L, __dmul_rn(2.0, CUDART_PI));
    const int hc = int(rint(__dmul_rn(__dmul_rn(qmag, cos(th)), scale)));
    const int kc = int(rint(__dmul_rn(__dmul_rn(qmag, sin(th)), scale)));
    const int w = 2 * hw + 1;
    for (int dh = 0; dh < w; ++dh)
        for (int dk = 0; dk < w; ++dk) hk[size_t(r) * w * w + dh * w + dk] = make_int2(hc - hw + dh, kc - hw + dk);
}

// chi_j = exp(i q_0 . x_j) (Eq. 11), by global disk id.
__global__ void __launch_bounds__(256)
k_chi(const Rep* __restrict__ reps, int R, int64_t Ntot, bool fixed, const int2* __restrict__ hk0,
      const double* __restrict__ xy, double2* __restrict__ chi) {
    pdl_begin();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= Ntot) return;
    const int r = rep_of_id(reps, R, i);
    chi[i] = plane_wave(reps[r], fixed, hk0[r].x, hk0[r].y, __ddiv_rn(xy[2 * i], reps[r].sigma),
                        __ddiv_rn(xy[2 * i + 1], reps[r].sigma));
}

// Positional correlation (Eq. 12): for each ordered pair n != m found through
// the cell grid within reach, with d = x_m - x_n - L rint((x_m - x_n) / L)
// from the global positions and d^2 = dx dx + dy dy, add chi_n conj(chi_m)
// to every window k (r_k = (k + 1) dr) with max(r_k - 1, 0)^2 <= d^2 <=
// (r_k + 1)^2.  acc[r][k] = (sum Re, sum Im, pairs), accumulated per block in
// shared memory (nr <= kMaxCorrWindows).
constexpr int kMaxCorrWindows = 1024;

template <int CAP>
__global__ void __launch_bounds__(256)
k_poscorr(const Rep* __restrict__ reps, int R, const uint8_t* __restrict__ cnt, const int32_t* __restrict__ pid,
          const double* __restrict__ xy, const double2* __restrict__ chi, int nr, double dr, int reach,
          double* __restrict__ acc) {
    extern __shared__ double s_acc[];  // [nr][3]
    pdl_begin();
    for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x) s_acc[k] = 0.0;
    __syncthreads();
    const int r = find_rep<kGridCell>(reps, R, blockIdx.x);
    const Rep& rep = reps[r];
    const int m = rep.m;
    const int64_t a = int64_t(blockIdx.x - rep.blk_cell) * blockDim.x + threadIdx.x;
    if (a < int64_t(m) * m) {
        int cx, cy;
        cell_coords(rep, a, cx, cy);
        const uint32_t cell = rep.coff + uint32_t(a);
        const int n = min(int(cnt[cell]), CAP);
        const double L = rep.Lm;
        for (int s = 0; s < n; ++s) {
            const int64_t in = rep.id_off + pid[size_t(s) * rep.stride32 + cell];
            const double xn = __ddiv_rn(xy[2 * in], rep.sigma), yn = __ddiv_rn(xy[2 * in + 1], rep.sigma);
            const double2 cn = chi[in];
            for (int dcy = -reach; dcy <= reach; ++dcy) {
                for (int dcx = -reach; dcx <= reach; ++dcx) {
                    const uint32_t nc = rep.coff + row_part(rep, wrap_cell(cy + dcy, m)) + col_part(rep, wrap_cell(cx + dcx, m));
                    const int nn = min(int(cnt[nc]), CAP);
                    for (int q = 0; q < nn; ++q) {
                        const int64_t im = rep.id_off + pid[size_t(q) * rep.stride32 + nc];
                        if (im == in) continue;
                        double dx = __dsub_rn(__ddiv_rn(xy[2 * im], rep.sigma), xn);
                        double dy = __dsub_rn(__ddiv_rn(xy[2 * im + 1], rep.sigma), yn);
                        dx = __dsub_rn(dx, __dmul_rn(L, rint(__ddiv_rn(dx, L))));
                        dy = __dsub_rn(dy, __dmul_rn(L, rint(__ddiv_rn(dy, L))));
                        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                        const double d = sqrt(d2);
                        const int klo = max(0, int(floor(__ddiv_rn(__dsub_rn(d, 1.0), dr))) - 2);
                        const int khi = min(nr - 1, int(floor(__ddiv_rn(__dadd_rn(d, 1.0), dr))) + 1);
                        if (klo > khi) continue;
                        const double2 cm = chi[im];
                        // chi_n conj(chi_m)
                        const double pr = __dadd_rn(__dmul_rn(cn.x, cm.x), __dmul_rn(cn.y, cm.y));
                        const double pi_ = __dsub_rn(__dmul_rn(cn.y, cm.x), __dmul_rn(cn.x, cm.y));
                        for (int k = klo; k <= khi; ++k) {
                            const double rk = __dmul_rn(double(k + 1), dr);
                            const double lo = rk > 1.0 ? __dsub_rn(rk, 1.0) : 0.0;
                            const double hi = __dadd_rn(rk, 1.0);
                            if (d2 >= __dmul_rn(lo, lo) && d2 <= __dmul_rn(hi, hi)) {
                                atomicAdd(&s_acc[3 * k], pr);
                                atomicAdd(&s_acc[3 * k + 1], pi_);
                                atomicAdd(&s_acc[3 * k + 2], 1.0);
                            }
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x)
        if (s_acc[k] != 0.0) atomicAdd(&acc[size_t(r) * 3 * nr + k], s_acc[k]);
}

__global__ void __launch_bounds__(256)
k_corr_norm(int64_t n, const double* __restrict__ acc, double2* __restrict__ out) {
    pdl_begin();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = acc[3 * i + 2];
    out[i] = c > 0.0 ? make_double2(__ddiv_rn(acc[3 * i], c), __ddiv_rn(acc[3 * i + 1], c))
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

int sq_disk_blocks(const std::vector<int64_t>& N) {
    int64_t b = 1;
    for (int64_t n : N) b = std::max<int64_t>(b, (n + 255) / 256);
    return int(b);
}

cudaError_t launch_sq(const LaunchCfg& c, int nq, const int2* hk, const double* xy, int nbx, double2* part, double* S,
                      int* best) {
    const dim3 grid(unsigned(nbx), unsigned((nq + kSqChunk - 1) / kSqChunk), unsigned(c.R));
    const cudaError_t e = launch_k(k_sq_amp, grid, dim3(256), 0, c.stream, c.reps, c.fixed, nq, hk, xy, nbx, part);
    if (e != cudaSuccess) return e;
    return launch_k(k_sq_reduce, dim3(unsigned(c.R)), dim3(256), 0, c.stream, c.reps, nq, nbx, (const double2*)part, S,
                    best);
}

cudaError_t launch_q0_window(const LaunchCfg& c, int hw, const double* psi, int2* hk) {
    return launch_k(k_q0_window, dim3(unsigned((c.R + 31) / 32)), dim3(32), 0, c.stream, c.reps, c.R, hw, psi, hk);
}

cudaError_t launch_chi(const LaunchCfg& c, int64_t Ntot, const int2* hk0, const double* xy, double2* chi) {
    return launch_k(k_chi, dim3(unsigned((Ntot + 255) / 256)), dim3(256), 0, c.stream, c.reps, c.R, Ntot, c.fixed, hk0,
                    xy, chi);
}

template <int CAP>
static cudaError_t poscorr_t(const LaunchCfg& c, CellBufs cells, const double* xy, const double2* chi, int nr,
                             double dr, int reach, double* acc) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_poscorr<CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(3 * kMaxCorrWindows * sizeof(double)));
    });
    return launch_k(k_poscorr<CAP>, dim3(c.blocks_cell), dim3(c.threads), size_t(3 * nr) * sizeof(double), c.stream,
                    c.reps, c.R, (const uint8_t*)cells.cnt, (const int32_t*)cells.pid, xy, chi, nr, dr, reach, acc);
}

cudaError_t launch_poscorr(const LaunchCfg& c, CellBufs cells, const double* xy, const double2* chi, int nr, double dr,
                           int reach, double* acc, double2* out) {
    cudaError_t e = cudaMemsetAsync(acc, 0, size_t(c.R) * 3 * nr * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    e = c.cap == 4 ? poscorr_t<4>(c, cells, xy, chi, nr, dr, reach, acc) : poscorr_t<9>(c, cells, xy, chi, nr, dr, reach, acc);
    if (e != cudaSuccess) return e;
    const int64_t n = int64_t(c.R) * nr;
    return launch_k(k_corr_norm, dim3(unsigned((n + 255) / 256)), dim3(256), 0, c.stream, n, (const double*)acc, out);
}

}  // namespace hd
