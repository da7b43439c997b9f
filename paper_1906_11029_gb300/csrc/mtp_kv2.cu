// FP32 instantiations of the tent kernels in shape variant 2: one patch element and one basis
// function (or facet mode) per item, 512 threads per CTA in 3D, for the shortest tents on
// layers that hold fewer tents than the GPU has CTA slots; the degree argument carries the
// variant as p + 32.
#include "mtp_launch.cuh"
namespace mtp {
void kernel_table_f32_v2(KernelEntry e[2][5]) {
    e[0][0] = MTP_KERNEL_ENTRY(float, 2, 33, 0);
    e[0][1] = MTP_KERNEL_ENTRY(float, 2, 34, 0);
    e[0][2] = MTP_KERNEL_ENTRY(float, 2, 35, 0);
    e[0][3] = MTP_KERNEL_ENTRY(float, 2, 36, 0);
    e[0][4] = MTP_KERNEL_ENTRY(float, 2, 37, 0);
    e[1][0] = MTP_KERNEL_ENTRY(float, 3, 33, 0);
    e[1][1] = MTP_KERNEL_ENTRY(float, 3, 34, 0);
    e[1][2] = MTP_KERNEL_ENTRY(float, 3, 35, 0);
    e[1][3] = MTP_KERNEL_ENTRY(float, 3, 36, 0);
    e[1][4] = MTP_KERNEL_ENTRY(float, 3, 37, 0);
}
}  // namespace mtp
