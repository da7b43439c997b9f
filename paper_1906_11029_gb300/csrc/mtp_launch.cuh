// Launch wrappers for the tent kernels; instantiated per state precision in
// mtp_k64.cu / mtp_k32.cu so the two halves compile in parallel.
#pragma once

#include "mtp_kernels.cuh"

namespace mtp {

using LaunchFn = cudaError_t (*)(const KArgs&, int64_t t0, int n_tents, int n_rhs, cudaStream_t st);
using PrepareFn = cudaError_t (*)(int max_patch, size_t* smem_bytes);
using PersistentFn = cudaError_t (*)(const KArgs&, const PArgs&, int grid, cudaStream_t st);
using PersistentPrepFn = cudaError_t (*)(int max_patch, int* blocks_per_sm);

// true when `bytes` of dynamic shared memory fit one block on the current device
inline bool smem_fits(size_t bytes) {
    int dev = 0, mx = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return bytes <= (size_t)mx;
}

// The prepare functions report the block's shared-memory size and, only when it fits the
// device, raise the kernel's dynamic shared-memory limit (a refused attribute call would leave
// an error behind for the next launch); the caller turns a size that does not fit into
// MTP_EUNSUPPORTED.
template <typename Real, int DIM, int P, int MODE = 0>
cudaError_t prepare_tent_kernel(int max_patch, size_t* smem_bytes) {
    SmemLayout<Real, DIM, P> lay(max_patch, MODE);
    *smem_bytes = lay.bytes;
    if (!smem_fits(lay.bytes)) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(tent_layer_kernel<Real, DIM, P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lay.bytes);
}

template <typename Real, int DIM, int P, int MODE = 0>
cudaError_t launch_tent_kernel(const KArgs& a, int64_t t0, int n_tents, int n_rhs, cudaStream_t st) {
    SmemLayout<Real, DIM, P> lay(a.max_patch, MODE);
    dim3 grid(n_tents, n_rhs);
    tent_layer_kernel<Real, DIM, P, MODE><<<grid, Shape<DIM, P>::NT, lay.bytes, st>>>(a, t0);
    return cudaGetLastError();
}

template <typename Real, int DIM, int P, int MODE = 0>
cudaError_t prepare_persistent_kernel(int max_patch, int* blocks_per_sm) {
    SmemLayout<Real, DIM, P> lay(max_patch, MODE);
    if (!smem_fits(lay.bytes)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tent_persistent_kernel<Real, DIM, P, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tent_persistent_kernel<Real, DIM, P, MODE>,
                                                         Shape<DIM, P>::NT, lay.bytes);
}

template <typename Real, int DIM, int P, int MODE = 0>
cudaError_t launch_persistent_kernel(const KArgs& a, const PArgs& pa, int grid, cudaStream_t st) {
    SmemLayout<Real, DIM, P> lay(a.max_patch, MODE);
    tent_persistent_kernel<Real, DIM, P, MODE><<<grid, Shape<DIM, P>::NT, lay.bytes, st>>>(a, pa);
    return cudaGetLastError();
}

struct KernelEntry {
    LaunchFn launch;
    PrepareFn prepare;
    PersistentFn persistent;
    PersistentPrepFn persistent_prepare;
};

// entries[dim - 2][p - 1]
void kernel_table_f64(KernelEntry entries[2][5]);
void kernel_table_f32(KernelEntry entries[2][5]);
// tensor-core modes (3D only): entries[mode - 1][p - 1]
void kernel_table_tc(KernelEntry entries[2][5]);
// FP32 arithmetic with the split (hi + lo) Taylor accumulator and an FP64 state: entries[dim - 2][p - 1]
void kernel_table_split(KernelEntry entries[2][5]);
// FP64, classical RK4 on the substituted tent ODE instead of SAT (MTP_FLAG_SUBSTITUTED_RK4)
void kernel_table_rk4(KernelEntry entries[2][5]);
// FP32, kernel shape variants 1 (one element per stage item) and 2 (one element and one row
// per item, 512 threads); see Shape
void kernel_table_f32_v1(KernelEntry entries[2][5]);
void kernel_table_f32_v2(KernelEntry entries[2][5]);
// FP32 3D, volume term on tcgen05 (variants 3 and 4, p = 2..4): entries[variant - 3][p - 1]
void kernel_table_f32_tc5(KernelEntry entries[2][5]);

struct AdjArgs;
using AdjLaunchFn = cudaError_t (*)(const AdjArgs&, int64_t t0, int n_tents, int n_rhs, cudaStream_t st);
using TapeStrideFn = int64_t (*)(int max_patch, int m, int q);
struct AdjEntry {
    AdjLaunchFn launch;
    PrepareFn prepare;
    TapeStrideFn tape_stride;
};
// entries[precision][dim - 2][p - 1]
void adjoint_table(AdjEntry entries[2][2][5]);

using BatchLaunchFn = cudaError_t (*)(const BatchArgs&, int grid, size_t smem, cudaStream_t st);
using BatchPrepFn = cudaError_t (*)(size_t smem, int* blocks_per_sm);
using BatchSmemFn = size_t (*)(int p, int max_patch);
struct BatchEntry {
    BatchLaunchFn launch;
    BatchPrepFn prepare;
    BatchSmemFn smem_bytes;
};
// entries[precision][dim - 2]
void batch_table(BatchEntry entries[2][2]);

#define MTP_KERNEL_ENTRY(REAL, D, P, MODE)                                                      \
    KernelEntry{launch_tent_kernel<REAL, D, P, MODE>, prepare_tent_kernel<REAL, D, P, MODE>,     \
                launch_persistent_kernel<REAL, D, P, MODE>, prepare_persistent_kernel<REAL, D, P, MODE>}
#define MTP_KERNEL_TABLE(NAME, REAL, MODE)                                                      \
    void NAME(KernelEntry e[2][5]) {                                                            \
        e[0][0] = MTP_KERNEL_ENTRY(REAL, 2, 1, MODE);                              \
        e[0][1] = MTP_KERNEL_ENTRY(REAL, 2, 2, MODE);                              \
        e[0][2] = MTP_KERNEL_ENTRY(REAL, 2, 3, MODE);                              \
        e[0][3] = MTP_KERNEL_ENTRY(REAL, 2, 4, MODE);                              \
        e[0][4] = MTP_KERNEL_ENTRY(REAL, 2, 5, MODE);                              \
        e[1][0] = MTP_KERNEL_ENTRY(REAL, 3, 1, MODE);                              \
        e[1][1] = MTP_KERNEL_ENTRY(REAL, 3, 2, MODE);                              \
        e[1][2] = MTP_KERNEL_ENTRY(REAL, 3, 3, MODE);                              \
        e[1][3] = MTP_KERNEL_ENTRY(REAL, 3, 4, MODE);                              \
        e[1][4] = MTP_KERNEL_ENTRY(REAL, 3, 5, MODE);                              \
    }

}  // namespace mtp
