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
// The scratch is shared by every call in the process on a given device: calls
// that overlap on the GPU (concurrent streams, or host threads issuing calls
// without ordering them) race on it and must be serialised by the caller.
// Each call writes every partial it later reads, so nothing needs clearing
// between calls.
#include <mutex>

#include "hd.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                            // psi_j per thread per block
constexpr int kMaxBlocks = 4096;                      // partial sums held in the scratch array
constexpr int64_t kPerBlock = int64_t(kThreads) * kItems;
constexpr int kMaxDevices = 64;

// Per-block partial sums (Re, Im) of one call.  4096 x 16 bytes = 64 KiB.
static __device__ __align__(256) double2 g_psi6_partials[kMaxBlocks];

// Stage 1: block b sums psi_j for j in [b * kPerBlock, (b + 1) * kPerBlock)
// in a fixed order (per-thread strided sums, then a fixed shuffle tree).
__global__ void __launch_bounds__(kThreads)
k_psi6_partials(const double2* __restrict__ psi, int64_t N, double2* __restrict__ partials) {
    const int64_t base = int64_t(blockIdx.x) * kPerBlock;
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = base + int64_t(i) * kThreads + threadIdx.x;
        if (j < N) {
            const double2 v = psi[j];
            sr += v.x;
            si += v.y;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, off);
        si += __shfl_down_sync(0xffffffffu, si, off);
    }
    __shared__ double s_re[kThreads / 32], s_im[kThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        s_re[threadIdx.x >> 5] = sr;
        s_im[threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            tr += s_re[w];
            ti += s_im[w];
        }
        partials[blockIdx.x] = make_double2(tr, ti);
    }
}

// Stage 2: one block sums the partials in a fixed order and divides by N.
__global__ void __launch_bounds__(kThreads)
k_psi6_finish(const double2* __restrict__ partials, int blocks, int64_t N, double* __restrict__ out) {
    double sr = 0.0, si = 0.0;
    for (int b = threadIdx.x; b < blocks; b += kThreads) {
        sr += partials[b].x;
        si += partials[b].y;
    }
    __shared__ double s_re[kThreads], s_im[kThreads];
    s_re[threadIdx.x] = sr;
    s_im[threadIdx.x] = si;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) {
            s_re[threadIdx.x] += s_re[threadIdx.x + s];
            s_im[threadIdx.x] += s_im[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s_re[0] / double(N);
        out[1] = s_im[0] / double(N);
    }
}

// Device address of the scratch array, looked up once per device (host code
// cannot use the array's name as a device pointer).
std::mutex g_setup_mutex;
double2* g_scratch_addr[kMaxDevices] = {};

hd_status scratch_for_current_device(double2** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_psi6_partials) != cudaSuccess || !p) return HD_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<double2*>(p);
    }
    *out = g_scratch_addr[dev];
    return HD_OK;
}

}  // namespace

extern "C" hd_status hd_psi6_mean_noalloc(const double* psi_local_device, int64_t N, double* out_device,
                                          void* stream) {
    if (!psi_local_device || !out_device || N < 1 || N > int64_t(kMaxBlocks) * kPerBlock) return HD_ERR_ARG;
    double2* scratch = nullptr;
    const hd_status s = scratch_for_current_device(&scratch);
    if (s != HD_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = int((N + kPerBlock - 1) / kPerBlock);
    k_psi6_partials<<<blocks, kThreads, 0, st>>>(reinterpret_cast<const double2*>(psi_local_device), N, scratch);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    k_psi6_finish<<<1, kThreads, 0, st>>>(scratch, blocks, N, out_device);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}
