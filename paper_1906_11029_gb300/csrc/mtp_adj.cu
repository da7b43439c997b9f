// Instantiations and launch wrappers of the adjoint tent kernel.
#include "mtp_adjoint.cuh"
#include "mtp_launch.cuh"

namespace mtp {

template <typename Real, int DIM, int P>
cudaError_t prepare_adjoint_kernel(int max_patch, size_t* smem_bytes) {
    AdjLayout<Real, DIM, P> lay(max_patch);
    *smem_bytes = lay.bytes;
    if (!smem_fits(lay.bytes)) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(tent_adjoint_kernel<Real, DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lay.bytes);
}

template <typename Real, int DIM, int P>
cudaError_t launch_adjoint_kernel(const AdjArgs& a, int64_t t0, int n_tents, int n_rhs, cudaStream_t st) {
    AdjLayout<Real, DIM, P> lay(a.k.max_patch);
    dim3 grid(n_tents, n_rhs);
    tent_adjoint_kernel<Real, DIM, P><<<grid, Shape<DIM, P>::NT, lay.bytes, st>>>(a, t0);
    return cudaGetLastError();
}

template <typename Real, int DIM, int P>
int64_t adjoint_tape_stride(int max_patch, int m, int q) {
    using Sh = Shape<DIM, P>;
    return (int64_t)(m + m * q) * max_patch * Sh::NF * Sh::NBP;
}

#define ADJ_ENTRY(REAL, D, P) {launch_adjoint_kernel<REAL, D, P>, prepare_adjoint_kernel<REAL, D, P>, adjoint_tape_stride<REAL, D, P>}

void adjoint_table(AdjEntry e[2][2][5]) {
    AdjEntry t[2][2][5] = {
        {{ADJ_ENTRY(double, 2, 1), ADJ_ENTRY(double, 2, 2), ADJ_ENTRY(double, 2, 3), ADJ_ENTRY(double, 2, 4), ADJ_ENTRY(double, 2, 5)},
         {ADJ_ENTRY(double, 3, 1), ADJ_ENTRY(double, 3, 2), ADJ_ENTRY(double, 3, 3), ADJ_ENTRY(double, 3, 4), ADJ_ENTRY(double, 3, 5)}},
        {{ADJ_ENTRY(float, 2, 1), ADJ_ENTRY(float, 2, 2), ADJ_ENTRY(float, 2, 3), ADJ_ENTRY(float, 2, 4), ADJ_ENTRY(float, 2, 5)},
         {ADJ_ENTRY(float, 3, 1), ADJ_ENTRY(float, 3, 2), ADJ_ENTRY(float, 3, 3), ADJ_ENTRY(float, 3, 4), ADJ_ENTRY(float, 3, 5)}}};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 5; ++c) e[a][b][c] = t[a][b][c];
}

}  // namespace mtp
