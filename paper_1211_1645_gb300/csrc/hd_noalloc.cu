// hd_noalloc.cu -- global Psi_6 from a caller-provided psi_j field without
// any memory allocation.
//
// Some callers cannot allocate device memory at the point where they need
// this reduction: code running inside a CUDA stream capture, code driven by a
// host framework that owns every allocation and forbids others (a fixed
// memory pool), or a real-time loop where an allocation could block or fail.
// For them this file provides a variant of the library's Psi_6 reduction whose
// scratch space -- the per-block partial sums -- lives in one statically sized
// device array that exists for as long as the library is loaded, so the call
// allocates and frees nothing.
//
// The sums are exact (hd_exact.cuh), so the result is the same as the
// library's own hd_psi6 on the same field, bit for bit: the total of each part
// rounded once to double, then divided by N.
//
// The scratch is shared by every call in the process on a given device: calls
// that overlap on the GPU (concurrent streams, or host threads issuing calls
// without ordering them) race on it and must be serialised by the caller.
// Each call writes every partial it later reads, so nothing needs clearing
// between calls.
#include <cstdint>

#include "hd.h"
#include "hd_exact.cuh"

namespace {

using hd::Exact192;
using hd::ExactPair;

constexpr int kThreads = 256;
constexpr int kItems = 16;                            // psi_j per thread per block
constexpr int kMaxBlocks = 4096;                      // partial sums held in the scratch array
constexpr int64_t kPerBlock = int64_t(kThreads) * kItems;

// Per-block exact partial sums (Re, Im) of one call: 4096 x 64 bytes = 256 KiB.
static __device__ __align__(256) ExactPair g_psi6_partials[kMaxBlocks];

// Stage 1: block b sums psi_j for j in [b * kPerBlock, (b + 1) * kPerBlock).
// The field is read as separate doubles, so 8-byte alignment suffices.
__global__ void __launch_bounds__(kThreads)
k_psi6_partials(const double* __restrict__ psi, int64_t N, ExactPair* __restrict__ partials) {
    const int64_t base = int64_t(blockIdx.x) * kPerBlock;
    Exact192 sr = hd::exact_zero(), si = hd::exact_zero();
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = base + int64_t(i) * kThreads + threadIdx.x;
        if (j < N) {
            hd::exact_add(sr, psi[2 * j]);
            hd::exact_add(si, psi[2 * j + 1]);
        }
    }
    const ExactPair t = hd::exact_block_sum(sr, si);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Stage 2: one block adds the partials, rounds each part once and divides by N.
__global__ void __launch_bounds__(kThreads)
k_psi6_finish(const ExactPair* __restrict__ partials, int blocks, int64_t N, double* __restrict__ out) {
    Exact192 sr = hd::exact_zero(), si = hd::exact_zero();
    for (int b = threadIdx.x; b < blocks; b += kThreads) {
        hd::exact_merge(sr, partials[b].re);
        hd::exact_merge(si, partials[b].im);
    }
    const ExactPair t = hd::exact_block_sum(sr, si);
    if (threadIdx.x == 0) {
        out[0] = __ddiv_rn(hd::exact_round(t.re), double(N));
        out[1] = __ddiv_rn(hd::exact_round(t.im), double(N));
    }
}

}  // namespace

extern "C" hd_status hd_psi6_mean_noalloc(const double* psi_local_device, int64_t N, double* out_device,
                                          void* stream) {
    if (!psi_local_device || !out_device || N < 1 || N > int64_t(kMaxBlocks) * kPerBlock) return HD_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(psi_local_device) & 7u) != 0u ||
        (reinterpret_cast<uintptr_t>(out_device) & 7u) != 0u)
        return HD_ERR_ARG;
    // The array's name is a host-side stand-in in host code: its device address
    // on the current device comes from the runtime.  Looked up on every call
    // (no allocation), so it stays valid across a cudaDeviceReset.
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_psi6_partials) != cudaSuccess || !scratch) return HD_ERR_CUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = int((N + kPerBlock - 1) / kPerBlock);
    k_psi6_partials<<<blocks, kThreads, 0, st>>>(psi_local_device, N, static_cast<ExactPair*>(scratch));
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    k_psi6_finish<<<1, kThreads, 0, st>>>(static_cast<const ExactPair*>(scratch), blocks, N, out_device);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}
