// FP64 instantiations of the tent kernels.
#include "mtp_launch.cuh"
namespace mtp {
MTP_KERNEL_TABLE(kernel_table_f64, double, 0)
}
