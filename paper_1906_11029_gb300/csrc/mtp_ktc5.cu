// FP32 instantiations of the tent kernels with the volume term on the tcgen05 tensor cores (3D,
// p = 2..4): shape variant 3 (item shape of variant 1, degree argument p + 48) and 4 (item
// shape of variant 2, p + 64); entries[variant - 3][p - 1].
#include "mtp_launch.cuh"
namespace mtp {
void kernel_table_f32_tc5(KernelEntry e[2][5]) {
    for (int v = 0; v < 2; ++v)
        for (int p = 0; p < 5; ++p) e[v][p] = KernelEntry{nullptr, nullptr, nullptr, nullptr};
    e[0][1] = MTP_KERNEL_ENTRY(float, 3, 50, 0);
    e[0][2] = MTP_KERNEL_ENTRY(float, 3, 51, 0);
    e[0][3] = MTP_KERNEL_ENTRY(float, 3, 52, 0);
    e[1][1] = MTP_KERNEL_ENTRY(float, 3, 66, 0);
    e[1][2] = MTP_KERNEL_ENTRY(float, 3, 67, 0);
    e[1][3] = MTP_KERNEL_ENTRY(float, 3, 68, 0);
}
}  // namespace mtp
