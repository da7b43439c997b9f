// FP32 instantiations of the tent kernels in shape variant 1: one patch element per stage item
// (twice the items of the paired default at half the work each) for layers that hold fewer
// tents than the GPU has CTA slots; the degree argument carries the variant as p + 16.
#include "mtp_launch.cuh"
namespace mtp {
void kernel_table_f32_v1(KernelEntry e[2][5]) {
    e[0][0] = MTP_KERNEL_ENTRY(float, 2, 17, 0);
    e[0][1] = MTP_KERNEL_ENTRY(float, 2, 18, 0);
    e[0][2] = MTP_KERNEL_ENTRY(float, 2, 19, 0);
    e[0][3] = MTP_KERNEL_ENTRY(float, 2, 20, 0);
    e[0][4] = MTP_KERNEL_ENTRY(float, 2, 21, 0);
    e[1][0] = MTP_KERNEL_ENTRY(float, 3, 17, 0);
    e[1][1] = MTP_KERNEL_ENTRY(float, 3, 18, 0);
    e[1][2] = MTP_KERNEL_ENTRY(float, 3, 19, 0);
    e[1][3] = MTP_KERNEL_ENTRY(float, 3, 20, 0);
    e[1][4] = MTP_KERNEL_ENTRY(float, 3, 21, 0);
}
}  // namespace mtp
