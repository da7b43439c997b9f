// FP64 instantiations of the tent kernels that advance each tent with the classical Runge-Kutta
// method on the substituted equation d/dt Y = A M^-1 Y (MTP_FLAG_SUBSTITUTED_RK4), the
// approach that structure-aware Taylor stepping replaces (Sec. 3 and Sec. 5.1).
#include "mtp_launch.cuh"
namespace mtp {
MTP_KERNEL_TABLE(kernel_table_rk4, double, 4)
}
