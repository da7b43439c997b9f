// FP32 instantiations of the tent kernels (geometry and the causality test in FP64).
#include "mtp_launch.cuh"
namespace mtp {
MTP_KERNEL_TABLE(kernel_table_f32, float, 0)
}
