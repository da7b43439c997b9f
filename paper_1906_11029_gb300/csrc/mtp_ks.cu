// Instantiations of the tent kernels with FP32 arithmetic, the Taylor sum of each tent carried
// as an FP32 pair hi + lo (two-sum) and the state between tents stored in FP64 (MTP_FP32_SPLIT).
#include "mtp_launch.cuh"
namespace mtp {
MTP_KERNEL_TABLE(kernel_table_split, float, 3)
}
