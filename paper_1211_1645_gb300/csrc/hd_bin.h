// hd_bin.h -- device binning of caller positions (hd_set_positions).
#pragma once

#include "hd_kernels.h"

namespace hd {
// Bin positions xy[2 Ntot] (device) into the unshifted frame of `to`, whose
// occupancy must be zero; input errors set kErrBinOverflow / kErrBinInput.
constexpr int kErrBinOverflow = 16;
constexpr int kErrBinInput = 32;
cudaError_t launch_bin(const LaunchCfg& c, int64_t Ntot, double sigma, const double* xy, CellBufs to, int* err);

}  // namespace hd
