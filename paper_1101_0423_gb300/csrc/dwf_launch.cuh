// dwf_launch.cuh -- host-side launchers of the kernel templates, instantiated once per
// precision in k_f64.cu / k_f32.cu / k_half.cu so the three compile in parallel.
#pragma once

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "dwf_kernels.cuh"

namespace dwf {

// threads per CTA of the per-site kernels: the Ns slices of spb sites
// (at most 64 sites, which bounds the shared memory of small-Ns CTAs)
inline int sites_per_block(int P, int Ns) {
  const int target = (P == P_F64) ? 128 : 256;
  int spb = target / Ns;
  if (spb > 64) spb = 64;
  return spb < 1 ? 1 : spb;
}

// sites per CTA of k_hop, whose CTA is (Ns, spb): 128 threads measured best at Ns = 16
// (against 256 and 512 threads, and 64 and 96, for the FP32 hop kernels)
inline int hop_sites_per_block(int P, int Ns) {
  const int target = 128;
  (void)P;
  int spb = target / Ns;
  if (spb > 64) spb = 64;
  return spb < 1 ? 1 : spb;
}

inline int vec_grid(long n, int sm_count) {
  long g = (n + 255) / 256;
  long cap = (long)sm_count * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <int P, int EPI, int NSC>
cudaError_t hop_go(const HopArgs &a, cudaStream_t st) {
  // the shape the host chose (autotuner), else 128-thread CTAs, persistent without M5
  int spb = hop_sites_per_block(P, a.Ns);
  bool persistent = hop_persistent<EPI>();
  if (a.shape_threads > 0) {
    spb = std::max(1, std::min(64, a.shape_threads / a.Ns));
    persistent = a.shape_persistent != 0;
  }
  if (spb * a.Ns > 256) return cudaErrorInvalidConfiguration;
  const size_t smem = hop_smem_bytes<P, EPI>(spb, a.Ns);
  if (smem > 48 * 1024) {  // launches may come from several host threads
    static std::mutex cmu;
    static size_t configured = 0;
    std::lock_guard<std::mutex> lock(cmu);
    if (configured < smem) {
      cudaError_t e =
          cudaFuncSetAttribute(k_hop<P, EPI, NSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
  }
  const int nrhs = a.nrhs > 1 ? a.nrhs : 1;
  const long ntile = (a.h + spb - 1) / spb;
  long nblk = ntile;  // one tile per CTA
  if (persistent) {
    // persistent grid: as many CTAs per right-hand side as are resident at once, each taking
    // an equal number of tiles (the rows of a batch follow one another through the GPU, and
    // a finished right-hand side's row returns at once)
    const int nthr = a.Ns * spb;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // resident CTAs per GPU for this kernel, CTA size and shared memory (cached)
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, long> resident;
    const auto key = std::make_tuple(dev, nthr, smem);
    long res = 0;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = resident.find(key);
      if (it != resident.end()) res = it->second;
    }
    if (res <= 0) {
      int sms = 0, per = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hop<P, EPI, NSC>, nthr, smem);
      if (e != cudaSuccess) return e;
      res = (long)std::max(per, 1) * sms;
      std::lock_guard<std::mutex> lock(mu);
      resident[key] = res;
    }
    const long per_cta = (ntile + res - 1) / res;
    nblk = (ntile + per_cta - 1) / per_cta;
  }
  k_hop<P, EPI, NSC><<<dim3((unsigned)nblk, nrhs), dim3(a.Ns, spb), smem, st>>>(a);
  return cudaGetLastError();
}

// the inner-CG kernels get a compile-time Ns for the fifth-dimension extents in use
template <int P, int EPI>
cudaError_t hop_ns(const HopArgs &a, cudaStream_t st) {
  if constexpr (P != P_F64 && (EPI == E_M || EPI == E_XPAY_G5 || EPI == E_CG_UPDATE)) {
    switch (a.Ns) {
      case 8: return hop_go<P, EPI, 8>(a, st);
      case 12: return hop_go<P, EPI, 12>(a, st);
      case 16: return hop_go<P, EPI, 16>(a, st);
      case 20: return hop_go<P, EPI, 20>(a, st);
      case 24: return hop_go<P, EPI, 24>(a, st);
      case 32: return hop_go<P, EPI, 32>(a, st);
      default: break;
    }
  }
  return hop_go<P, EPI, 0>(a, st);
}

template <int P>
cudaError_t hop_launch(int epi, const HopArgs &a, cudaStream_t st) {
  switch (epi) {
    case E_PLAIN: return hop_ns<P, E_PLAIN>(a, st);
    case E_M: return hop_ns<P, E_M>(a, st);
    case E_XPAY_G5: return hop_ns<P, E_XPAY_G5>(a, st);
    case E_XPAY: return hop_ns<P, E_XPAY>(a, st);
    case E_M_XPAY: return hop_ns<P, E_M_XPAY>(a, st);
    case E_CG_UPDATE: return hop_ns<P, E_CG_UPDATE>(a, st);
    case E_RESID: return hop_ns<P, E_RESID>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <int P, int MODE>
cudaError_t smix_go(const SmixArgs &a, cudaStream_t st) {
  const int spb = sites_per_block(P, a.Ns);
  const size_t smem = smix_smem_bytes<P>(spb, a.Ns, MODE == S_DUAL);
  if (smem > 48 * 1024) {
    static std::mutex cmu;
    static size_t configured = 0;
    std::lock_guard<std::mutex> lock(cmu);
    if (configured < smem) {
      cudaError_t e = cudaFuncSetAttribute(k_smix<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
  }
  const long nblk = (a.h + spb - 1) / spb;
  k_smix<P, MODE><<<dim3((unsigned)nblk, a.nrhs > 1 ? a.nrhs : 1), dim3(a.Ns, spb), smem, st>>>(a);
  return cudaGetLastError();
}

template <int P>
cudaError_t smix_launch(int mode, const SmixArgs &a, cudaStream_t st) {
  switch (mode) {
    case S_PLAIN: return smix_go<P, S_PLAIN>(a, st);
    case S_G5: return smix_go<P, S_G5>(a, st);
    case S_CGP: return smix_go<P, S_CGP>(a, st);
    case S_DUAL: return smix_go<P, S_DUAL>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <int P>
cudaError_t norm2_launch(const VecArgs &v, int sm_count, cudaStream_t st) {
  k_norm2<P><<<vec_grid(v.n, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}

template <int PA, int PB>
cudaError_t convert_go(const VecArgs &v, int sm_count, cudaStream_t st) {
  k_convert<PA, PB><<<vec_grid(v.n, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}

// conversions between FP64 and precision P, both directions
template <int P>
cudaError_t convert_launch(int to_p, const VecArgs &v, int sm_count, cudaStream_t st) {
  if (to_p) return convert_go<P_F64, P>(v, sm_count, st);
  return convert_go<P, P_F64>(v, sm_count, st);
}

template <int P>
cudaError_t accum_launch(const VecArgs &v, int sm_count, cudaStream_t st) {
  k_accum<P><<<vec_grid(v.n, sm_count), 256, 0, st>>>(v);
  return cudaGetLastError();
}

template <int P>
cudaError_t pack_launch(const double *host, Field out, Geom g, int parity, int sm_count, cudaStream_t st) {
  k_pack<P><<<vec_grid(g.h * g.Ns, sm_count), 256, 0, st>>>(host, out, g, parity);
  return cudaGetLastError();
}

template <int P>
cudaError_t unpack_launch(Field in, double *host, Geom g, int parity, int sm_count, cudaStream_t st) {
  k_unpack<P><<<vec_grid(g.h * g.Ns, sm_count), 256, 0, st>>>(in, host, g, parity);
  return cudaGetLastError();
}

template <int P>
cudaError_t gauge_launch(const double *U, void *G, Geom g, int parity, int sm_count, cudaStream_t st) {
  k_gauge<P><<<vec_grid(g.h * 8, sm_count), 256, 0, st>>>(U, static_cast<typename PT<P>::lreal *>(G), g,
                                                            parity);
  return cudaGetLastError();
}

// one set of entry points per precision
#define DWF_DECLARE_PREC(P)                                                                           \
  extern template cudaError_t hop_launch<P>(int, const HopArgs &, cudaStream_t);                     \
  extern template cudaError_t smix_launch<P>(int, const SmixArgs &, cudaStream_t);                   \
  extern template cudaError_t norm2_launch<P>(const VecArgs &, int, cudaStream_t);                   \
  extern template cudaError_t convert_launch<P>(int, const VecArgs &, int, cudaStream_t);            \
  extern template cudaError_t accum_launch<P>(const VecArgs &, int, cudaStream_t);                   \
  extern template cudaError_t pack_launch<P>(const double *, Field, Geom, int, int, cudaStream_t);    \
  extern template cudaError_t unpack_launch<P>(Field, double *, Geom, int, int, cudaStream_t);       \
  extern template cudaError_t gauge_launch<P>(const double *, void *, Geom, int, int, cudaStream_t);

#define DWF_INSTANTIATE_PREC(P)                                                                \
  template cudaError_t hop_launch<P>(int, const HopArgs &, cudaStream_t);                     \
  template cudaError_t smix_launch<P>(int, const SmixArgs &, cudaStream_t);                   \
  template cudaError_t norm2_launch<P>(const VecArgs &, int, cudaStream_t);                   \
  template cudaError_t convert_launch<P>(int, const VecArgs &, int, cudaStream_t);            \
  template cudaError_t accum_launch<P>(const VecArgs &, int, cudaStream_t);                   \
  template cudaError_t pack_launch<P>(const double *, Field, Geom, int, int, cudaStream_t);    \
  template cudaError_t unpack_launch<P>(Field, double *, Geom, int, int, cudaStream_t);       \
  template cudaError_t gauge_launch<P>(const double *, void *, Geom, int, int, cudaStream_t);

#ifndef DWF_KERNEL_TU
DWF_DECLARE_PREC(P_F64)
DWF_DECLARE_PREC(P_F32)
DWF_DECLARE_PREC(P_F16)
DWF_DECLARE_PREC(P_BF16)
#endif

cudaError_t neighbours_launch(int *nbr, Geom g, int parity, int sm_count, cudaStream_t st);
cudaError_t diff_norm2_launch(const VecArgs &v, int sm_count, cudaStream_t st);
cudaError_t host_axpy_launch(const HostAxpyArgs &v, int sm_count, cudaStream_t st);
cudaError_t point_sources_launch(double *rhs, long x0site, long V4, int Ns, cudaStream_t st);
cudaError_t prop_extract_launch(const double *sol, double *prop, long V4, int Ns, int sm_count, cudaStream_t st);

}  // namespace dwf
