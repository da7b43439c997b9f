// Allocation-free variant of the energy reduction (mtp_energy_noalloc, see include/mtp.h).
//
// mtp_energy reduces through a per-mesh partials buffer that the library cudaMallocs the
// first time the mesh is used on a device.  Some callers cannot allocate device memory at
// the point where they need the energy: a host framework that owns every byte of device
// memory through its own caching allocator and budget, or a loop that must not allocate
// after start-up.  This variant takes every array it reads or writes from the caller and
// keeps its reduction scratch in a fixed file-scope device array instead.
#include <string>

#include <cuda_runtime.h>

#include "mtp_internal.h"

namespace mtp {

constexpr int kNoAllocBlocks = 304;     // 2 blocks per SM on 152 SMs
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxRhs = 64;      // scratch: 304 x 64 doubles = 152 KiB per device

// Reduction scratch shared by every call on a device; it lives (on every GPU that loads
// this library) until the process exits.  Each call writes every slot that it later reads,
// so nothing has to be cleared between calls.
static __device__ __align__(256) double g_energy_scratch[kNoAllocBlocks * kNoAllocMaxRhs];

template <typename Real>
__global__ void energy_partial_noalloc_kernel(const Real* state, const double* eps, const double* mu, int64_t ne,
                                              int nf, int nb, double* scratch) {
    __shared__ double red[kNoAllocThreads];
    const int rhs = blockIdx.y;
    const int64_t n = ne * nf * nb;
    const Real* s = state + (int64_t)rhs * n;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / (nf * nb);
        const int f = (int)((i / nb) % nf);
        const bool isE = nf == 6 ? f < 3 : f < 2;   // E fields first (2D: Ex, Ey | Hz)
        const double y = (double)s[i];
        acc += y * y / (isE ? eps[e] : mu[e]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[rhs * kNoAllocBlocks + blockIdx.x] = red[0];
}

__global__ void energy_final_noalloc_kernel(const double* scratch, double* out) {
    __shared__ double red[kNoAllocThreads];
    const int rhs = blockIdx.x;
    double acc = 0;
    for (int i = threadIdx.x; i < kNoAllocBlocks; i += blockDim.x) acc += scratch[rhs * kNoAllocBlocks + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[rhs] = 0.5 * red[0];
}

// Device address of g_energy_scratch on the current device.  In host code the symbol's
// name is only a host-side handle, never a device address, so it is looked up with
// cudaGetSymbolAddress (with the device current) on every call: nothing is cached, so an
// address that a device reset made stale is never reused.  The first lookup on a device
// may load this file's device code, which is why the first call belongs before any stream
// capture.
static int scratch_address(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || !p)
        return set_error(MTP_ECUDA, std::string("cudaGetSymbolAddress(g_energy_scratch): ") + cudaGetErrorString(e));
    *out = (double*)p;
    return MTP_OK;
}

}  // namespace mtp

using namespace mtp;

extern "C" int mtp_energy_noalloc(const void* state_dev, const double* eps_dev, const double* mu_dev, int dim,
                                  int64_t n_elems, int p, int precision, int n_rhs, double* out_dev,
                                  void* stream) {
    if (!state_dev || !eps_dev || !mu_dev || !out_dev) return set_error(MTP_EINVAL, "NULL argument");
    if (dim != 2 && dim != 3) return set_error(MTP_EINVAL, "dim must be 2 or 3");
    if (p < 1 || p > kMaxDegree) return set_error(MTP_EINVAL, "p must be in 1..5");
    if (n_elems < 1) return set_error(MTP_EINVAL, "n_elems must be positive");
    if (precision < MTP_FP64 || precision > MTP_FP32_SPLIT) return set_error(MTP_EINVAL, "unknown precision");
    if (n_rhs < 1 || n_rhs > kNoAllocMaxRhs)
        return set_error(MTP_EINVAL, "n_rhs must be in 1.." + std::to_string(kNoAllocMaxRhs) +
                                         " (size of the static scratch of mtp_energy_noalloc)");
    cudaStream_t st = (cudaStream_t)stream;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != MTP_OK) return rc;
    const int nf = n_fields(dim), nb = n_basis(dim, p);
    dim3 grid(kNoAllocBlocks, n_rhs);
    if (precision == MTP_FP64 || precision == MTP_FP32_SPLIT)   // double states
        energy_partial_noalloc_kernel<double><<<grid, kNoAllocThreads, 0, st>>>(
            (const double*)state_dev, eps_dev, mu_dev, n_elems, nf, nb, scratch);
    else   // MTP_FP32, MTP_TF32, MTP_TF32X3: float states
        energy_partial_noalloc_kernel<float><<<grid, kNoAllocThreads, 0, st>>>(
            (const float*)state_dev, eps_dev, mu_dev, n_elems, nf, nb, scratch);
    energy_final_noalloc_kernel<<<n_rhs, kNoAllocThreads, 0, st>>>(scratch, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MTP_ECUDA, std::string("energy_noalloc launch: ") + cudaGetErrorString(e));
    return MTP_OK;
}
