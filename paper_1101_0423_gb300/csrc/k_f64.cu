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

cudaError_t point_sources_launch(double *rhs, long x0site, long V4, int Ns, cudaStream_t st) {
  k_point_sources<<<1, 32, 0, st>>>(rhs, x0site, V4, Ns);
  return cudaGetLastError();
}

cudaError_t prop_extract_launch(const double *sol, double *prop, long V4, int Ns, int sm_count, cudaStream_t st) {
  k_prop_extract<<<vec_grid(V4 * 144, sm_count), 256, 0, st>>>(sol, prop, V4, Ns);
  return cudaGetLastError();
}

cudaError_t diff_norm2_launch(const VecArgs &v, int sm_count, cudaStream_t st) {
  k_diff_norm2<<<vec_grid(v.n, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}
cudaError_t host_axpy_launch(const HostAxpyArgs &v, int sm_count, cudaStream_t st) {
  k_host_axpy<<<vec_grid(2 * v.g.h * v.g.Ns * 24, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}
}  // namespace dwf
