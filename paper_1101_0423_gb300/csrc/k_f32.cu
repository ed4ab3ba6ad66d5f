// FP32 instantiations of the kernel launchers (the inner CG of the mixed-precision solver).
#define DWF_KERNEL_TU
#include "dwf_launch.cuh"

namespace dwf {
DWF_INSTANTIATE_PREC(P_F32)
}  // namespace dwf
