// dwf_internal.h -- host-side state of a dwf_ctx (library-internal).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dwf.h"
#include "dwf_launch.cuh"
#include "dwf_part.cuh"
#include "dwf_tune.h"

namespace dwf {

// matrices along s held per context (kernel order K[chi][t][s] on the device)
enum MatKind { MK_M5 = 0, MK_M5T, MK_S1, MK_S2, MK_W, MK_Z, MK_ID, MK_MASS, MK_COUNT };

struct Buf {
  void *v = nullptr;
  float *nrm = nullptr;
  size_t bytes = 0;
};

// one profiled launch: kernel class and its event pair
struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

// Device memory of contexts and shared gauge fields comes from one library-owned,
// stream-ordered pool per device (cudaMallocFromPoolAsync / cudaFreeAsync on the owner's
// stream): releasing it does not synchronise the device, so a context destroyed while
// other solves run does not stall them, and freed blocks stay in the pool for the next
// context.  Pinned host mirrors come from a process-wide free list and are never handed
// back to the driver (cudaFreeHost synchronises).
cudaError_t dmalloc(void **p, size_t bytes, int device, cudaStream_t st);
void dfree(void *p, cudaStream_t st);
void *pinned_get(size_t bytes);
void pinned_put(void *p, size_t bytes);

}  // namespace dwf

// a device-resident gauge field shared by handle among the contexts of one lattice: the
// FP64 host-layout copy and the doubled per-parity forms of each precision, built on first
// use by whichever context needs them; freed with its last reference
struct dwf_gauge {
  int dims[4];
  long V4 = 0, h = 0;
  int device = 0;
  int sm_count = 0;
  double *d_U = nullptr;
  void *d_gauge[4][2] = {};
  bool ready[4] = {false, false, false, false};
  cudaStream_t stream = nullptr;  // allocation and build stream
  std::mutex mu;
  int refs = 1;  // the creator's reference plus one per attached context
};

struct dwf_ctx {
  int dims[4];
  int Ns;
  long V4, h;
  double m0, mq;
  std::vector<double> omega, sigma;
  // host FP64 matrices, row-major [chi][s][t]
  std::vector<double> mat[dwf::MK_COUNT];
  // device matrices per arithmetic precision (0: double, 1: float), kernel order
  void *dmat[2][dwf::MK_COUNT] = {};
  // M5 (0) and M5^T (1) as recurrence tables along s (host FP64; device per precision)
  std::vector<double> rec[2];
  void *drec[2][2] = {};
  int *d_nbr[2] = {nullptr, nullptr};
  double *d_U = nullptr;  // FP64 host-layout copy of the gauge field
  void *d_gauge[4][2] = {};
  dwf_gauge *shared = nullptr;  // when attached: d_U and d_gauge point into it
  bool gauge_loaded = false;
  bool gauge_ready[4] = {false, false, false, false};
  std::map<std::string, dwf::Buf> bufs;
  dwf::CGScalars *d_sc = nullptr;
  dwf::CGScalars *h_sc = nullptr;  // pinned mirror
  dwf::CGScalars *h_scb = nullptr; // pinned mirror of the scalars of a batch
  int h_scb_cap = 0;
  double *d_part = nullptr;
  unsigned *d_ticket = nullptr;
  size_t part_len = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int device = 0;
  long long launches = 0;
  // failure-detection hook (dwf_debug_set_wait): bound of the hop kernels' waits for their
  // TMA copies, and whether the copies are left out so that the waits run out
  unsigned wait_tries = dwf::kWaitTries;
  int skip_copies = 0;
  // device address of the allocation-free entry point's static array (looked up by the
  // first dwf_apply_eo_dev_static call on this context)
  void *static_scratch = nullptr;
  // the launches of the current call take the autotuner's shapes (off for a solve with
  // no_autotune, which keeps the default shapes)
  bool use_tuned = true;
  // one part of a 4D domain decomposition (dwf_create_part): halo layout, the global gauge
  // field its local links are read from
  bool part = false;
  dwf::PartGeom pg{};
  double *d_Ug = nullptr;
  // pinned host staging of the packed faces for a caller's transport (dwf_part_*_comm):
  // the eight send faces, then the eight receive faces
  void *h_face = nullptr;
  size_t h_face_bytes = 0;
  // profiling of the current call
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<dwf::ProfRec> prof;
  std::string err;
};
