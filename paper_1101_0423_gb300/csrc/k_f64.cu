// FP64 instantiations of the kernel launchers (restart operator, source preparation,
// reconstruction, FP64 operator applications).
#define DWF_KERNEL_TU
#define DWF_DEFINE_PLAIN_KERNELS
#include "dwf_launch.cuh"

namespace dwf {
DWF_INSTANTIATE_PREC(P_F64)

cudaError_t neighbours_launch(int *nbr, Geom g, int parity, int sm_count, cudaStream_t st) {
  k_neighbours<<<vec_grid(g.h, sm_count), 256, 0, st>>>(nbr, g, parity);
  return cudaGetLastError();
}

cudaError_t diff_norm2_launch(const VecArgs &v, int sm_count, cudaStream_t st) {
  k_diff_norm2<<<vec_grid(v.n, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}
}  // namespace dwf
