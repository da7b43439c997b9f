// Tensor-core (warp-level TF32 MMA) instantiations of the tent kernels, 3D, FP32 state:
// mode 1 = TF32 operands, mode 2 = 3-term hi + lo split.
#include "mtp_launch.cuh"
namespace mtp {

#define TC_ENTRY(P, M) {launch_tent_kernel<float, 3, P, M>, prepare_tent_kernel<float, 3, P, M>, \
                        launch_persistent_kernel<float, 3, P, M>, prepare_persistent_kernel<float, 3, P, M>}

void kernel_table_tc(KernelEntry e[2][5]) {
    e[0][0] = TC_ENTRY(1, 1); e[0][1] = TC_ENTRY(2, 1); e[0][2] = TC_ENTRY(3, 1); e[0][3] = TC_ENTRY(4, 1);
    e[1][0] = TC_ENTRY(1, 2); e[1][1] = TC_ENTRY(2, 2); e[1][2] = TC_ENTRY(3, 2); e[1][3] = TC_ENTRY(4, 2);
    e[0][4] = e[1][4] = KernelEntry{nullptr, nullptr, nullptr, nullptr};   // p = 5: facet modes exceed one m16 tile
}

}  // namespace mtp
