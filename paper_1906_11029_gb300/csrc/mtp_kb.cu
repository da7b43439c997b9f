// Instantiations of the many-instance persistent kernel (all degrees in one kernel).
#include "mtp_launch.cuh"

namespace mtp {

template <typename Real, int DIM>
cudaError_t prepare_batch_kernel(size_t smem, int* blocks_per_sm) {
    if (!smem_fits(smem)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tent_batch_kernel<Real, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tent_batch_kernel<Real, DIM>,
                                                         Shape<DIM, 4>::NT, smem);
}

template <typename Real, int DIM>
cudaError_t launch_batch_kernel(const BatchArgs& b, int grid, size_t smem, cudaStream_t st) {
    tent_batch_kernel<Real, DIM><<<grid, Shape<DIM, 4>::NT, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename Real, int DIM>
size_t batch_smem_bytes(int p, int max_patch) {
    switch (p) {
        case 1: return SmemLayout<Real, DIM, 1>(max_patch).bytes;
        case 2: return SmemLayout<Real, DIM, 2>(max_patch).bytes;
        case 3: return SmemLayout<Real, DIM, 3>(max_patch).bytes;
        case 4: return SmemLayout<Real, DIM, 4>(max_patch).bytes;
        default: return SmemLayout<Real, DIM, 5>(max_patch).bytes;
    }
}

void batch_table(BatchEntry e[2][2]) {
    e[0][0] = {launch_batch_kernel<double, 2>, prepare_batch_kernel<double, 2>, batch_smem_bytes<double, 2>};
    e[0][1] = {launch_batch_kernel<double, 3>, prepare_batch_kernel<double, 3>, batch_smem_bytes<double, 3>};
    e[1][0] = {launch_batch_kernel<float, 2>, prepare_batch_kernel<float, 2>, batch_smem_bytes<float, 2>};
    e[1][1] = {launch_batch_kernel<float, 3>, prepare_batch_kernel<float, 3>, batch_smem_bytes<float, 3>};
}

}  // namespace mtp
