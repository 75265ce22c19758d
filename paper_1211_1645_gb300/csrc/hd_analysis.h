// hd_analysis.h -- launchers of the positional-order analysis (Sec. IV.C,
// Eqs. 10-12): the structure factor S[R][nq] at box-periodic wave vectors
// hk[R][nq] (best[R] = index of the largest), the q_0 candidate window around
// the first reciprocal shell, chi_j = exp(i q_0 . x_j), and the positional
// correlation C[R][nr] at r_k = (k + 1) dr.
#pragma once

#include <vector>

#include "hd_kernels.h"

namespace hd {

int sq_disk_blocks(const std::vector<int64_t>& N);
cudaError_t launch_sq(const LaunchCfg& c, int nq, const int2* hk, const double* xy, int nbx, double2* part, double* S,
                      int* best);
cudaError_t launch_q0_window(const LaunchCfg& c, int hw, const double* psi, int2* hk);
cudaError_t launch_chi(const LaunchCfg& c, int64_t Ntot, const int2* hk0, const double* xy, double2* chi);
cudaError_t launch_poscorr(const LaunchCfg& c, CellBufs cells, const double* xy, const double2* chi, int nr, double dr,
                           int reach, double* acc, double2* out);

}  // namespace hd
