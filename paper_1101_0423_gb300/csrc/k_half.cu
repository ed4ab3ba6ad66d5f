// fp16 / bf16 storage instantiations (FP32 arithmetic, per-(site, s) norm, 12-real links).
#define DWF_KERNEL_TU
#include "dwf_launch.cuh"

namespace dwf {
DWF_INSTANTIATE_PREC(P_F16)
DWF_INSTANTIATE_PREC(P_BF16)
}  // namespace dwf
