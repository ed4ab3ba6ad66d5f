// dwf_host.cu -- C-ABI entry points: context, gauge, operator applications, solver.
//
// As in Sec. 3, the host only steers: it decides what runs next, owns the allocations and
// drives the device; every vector operation, reduction and operator application runs in
// the kernels of dwf_kernels.cuh.  The CG scalars
// (alpha, beta, |r|^2, restart flag) stay on the device; the host reads them once per
// batch of inner iterations, and a batch is replayed from a CUDA graph.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cmath>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dwf_internal.h"

using namespace dwf;

// ------------------------------------------------------------------ memory

namespace dwf {

namespace {
constexpr int kMaxPoolDevices = 256;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};
std::mutex g_pinned_mu;
std::multimap<size_t, void *> g_pinned_free;  // size class -> free pinned block
size_t pinned_class(size_t bytes) { return (bytes + 4095) & ~(size_t)4095; }
}  // namespace

cudaError_t dmalloc(void **p, size_t bytes, int device, cudaStream_t st) {
  *p = nullptr;
  if (device < 0 || device >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[device]) {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      cudaMemPool_t np;
      cudaError_t e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return e;
      // keep freed blocks in the pool (they serve the next context) instead of returning
      // them to the driver at the next synchronisation
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      g_pools[device] = np;
    }
    pool = g_pools[device];
  }
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
}

void dfree(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

void *pinned_get(size_t bytes) {
  const size_t cls = pinned_class(bytes);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    auto it = g_pinned_free.find(cls);
    if (it != g_pinned_free.end()) {
      void *p = it->second;
      g_pinned_free.erase(it);
      return p;
    }
  }
  void *p = nullptr;
  if (cudaMallocHost(&p, cls) != cudaSuccess) return nullptr;
  return p;
}

void pinned_put(void *p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.emplace(pinned_class(bytes), p);
}

}  // namespace dwf

namespace {

constexpr double kD = 4.0;  // space-time dimension d of Eq. 2

const char *status_name(dwf_status s) {
  switch (s) {
    case DWF_OK: return "DWF_OK";
    case DWF_EINVAL: return "DWF_EINVAL";
    case DWF_ENOMEM: return "DWF_ENOMEM";
    case DWF_ENOCONV: return "DWF_ENOCONV";
    case DWF_EBUSY: return "DWF_EBUSY";
    case DWF_EAGAIN: return "DWF_EAGAIN";
    case DWF_ETIMEOUT: return "DWF_ETIMEOUT";
    case DWF_ECUDA: return "DWF_ECUDA";
    case DWF_ENOGAUGE: return "DWF_ENOGAUGE";
    case DWF_ECOMM: return "DWF_ECOMM";
  }
  return "DWF_UNKNOWN";
}

dwf_status fail(dwf_ctx *c, dwf_status st, const std::string &msg) {
  if (c) c->err = std::string(status_name(st)) + ": " + msg;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(c, e_ == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA,          \
                  std::string(#call) + " -> " + cudaGetErrorString(e_));                \
  } while (0)

#define TRY(expr)                        \
  do {                                   \
    dwf_status s_ = (expr);              \
    if (s_ != DWF_OK) return s_;         \
  } while (0)

size_t site_bytes(int prec) { return prec == P_F64 ? 192 : prec == P_F32 ? 96 : 48; }
// precision of the inner CG's x (FP32 when the inner fields are 16-bit, see k_smix)
int xprec(int prec) { return prec >= P_F16 ? P_F32 : prec; }
int mat_index(int prec) { return prec == P_F64 ? 0 : 1; }
bool valid_prec(int p) { return p >= DWF_PREC_F64 && p <= DWF_PREC_BF16; }

// ------------------------------------------------------------------ fifth-dimension matrices
//
// M5 of Eq. 8 is applied as a dense Ns x Ns matrix per chirality (Sec. 3.3).  Its entries
// are computed here column by column from the structure of Eq. 8: with y = omega^{-1/2} u
// and z = (1 + cL)^{-1} y, M5^{-1} u = v becomes the cyclic bidiagonal system
//   [(d - m0) sqrt(omega) + 1/sqrt(omega)] z + [(d - m0) sigma/sqrt(omega) - 1/sqrt(omega)] L z = v,
// then u = sqrt(omega) (z + c L z).  L = L+ (chirality +) or L- (chirality -), Eq. 4.

// (A + B L) z = v for the cyclic shift L of Eq. 4: chirality 0 uses L+ ((L z)_s = z_{s-1},
// (L z)_0 = kappa z_{Ns-1}), chirality 1 uses L- = L+^T.  Returns false on a zero pivot.
bool cyclic_solve(int Ns, const double *A, const double *B, double kappa, int chi, const double *v,
                  double *z) {
  std::vector<double> al(Ns), be(Ns);
  auto at = [&](int k) { return chi == 0 ? k : Ns - 1 - k; };
  const int s0 = at(0), last = at(Ns - 1);
  al[s0] = 0.0;
  be[s0] = 1.0;
  for (int k = 1; k < Ns; ++k) {
    const int s = at(k), sp = at(k - 1);
    if (A[s] == 0.0) return false;
    al[s] = (v[s] - B[s] * al[sp]) / A[s];
    be[s] = -B[s] * be[sp] / A[s];
  }
  const double den = A[s0] + B[s0] * kappa * be[last];
  if (den == 0.0) return false;
  const double zeta = (v[s0] - B[s0] * kappa * al[last]) / den;
  for (int s = 0; s < Ns; ++s) z[s] = al[s] + be[s] * zeta;
  return true;
}

// (L z)_s for chirality chi
double lshift(int Ns, double kappa, int chi, const double *z, int s) {
  if (chi == 0) return s > 0 ? z[s - 1] : kappa * z[Ns - 1];
  return s < Ns - 1 ? z[s + 1] : kappa * z[0];
}

bool build_matrices(dwf_ctx *c) {
  const int Ns = c->Ns;
  const double kappa = -c->mq / (2.0 * c->m0);
  const double dm = kD - c->m0;
  for (auto &m : c->mat) m.assign((size_t)2 * Ns * Ns, 0.0);
  std::vector<double> A(Ns), B(Ns), A1(Ns), Bc(Ns), v(Ns), z(Ns);
  for (int s = 0; s < Ns; ++s) {
    const double rw = sqrt(c->omega[s]);
    A[s] = dm * rw + 1.0 / rw;
    B[s] = dm * c->sigma[s] / rw - 1.0 / rw;
    A1[s] = 1.0;
    Bc[s] = c->sigma[s] / c->omega[s];
  }
  for (int chi = 0; chi < 2; ++chi) {
    double *M5 = c->mat[MK_M5].data() + (size_t)chi * Ns * Ns;
    double *M5T = c->mat[MK_M5T].data() + (size_t)chi * Ns * Ns;
    double *S1 = c->mat[MK_S1].data() + (size_t)chi * Ns * Ns;
    double *S2 = c->mat[MK_S2].data() + (size_t)chi * Ns * Ns;
    double *W = c->mat[MK_W].data() + (size_t)chi * Ns * Ns;
    double *Z = c->mat[MK_Z].data() + (size_t)chi * Ns * Ns;
    double *ID = c->mat[MK_ID].data() + (size_t)chi * Ns * Ns;
    double *MS = c->mat[MK_MASS].data() + (size_t)chi * Ns * Ns;
    for (int j = 0; j < Ns; ++j) {
      std::fill(v.begin(), v.end(), 0.0);
      v[j] = 1.0;
      // column j of M5
      if (!cyclic_solve(Ns, A.data(), B.data(), kappa, chi, v.data(), z.data())) return false;
      for (int s = 0; s < Ns; ++s)
        M5[s * Ns + j] = sqrt(c->omega[s]) * (z[s] + Bc[s] * lshift(Ns, kappa, chi, z.data(), s));
      // column j of (1 + cL)^{-1}, for S2 = Y^{-1} sqrt(omega) = (1 + cL)^{-1} omega^{-1/2} (Eq. 9)
      if (!cyclic_solve(Ns, A1.data(), Bc.data(), kappa, chi, v.data(), z.data())) return false;
      for (int s = 0; s < Ns; ++s) S2[s * Ns + j] = z[s] / sqrt(c->omega[j]);
    }
    for (int s = 0; s < Ns; ++s)
      for (int t = 0; t < Ns; ++t) {
        M5T[s * Ns + t] = M5[t * Ns + s];
        S1[s * Ns + t] = M5[s * Ns + t] / sqrt(c->omega[t]);  // S1 = M5 omega^{-1/2}
        // L_{st} of Eq. 4 for this chirality
        double Lst;
        if (chi == 0) Lst = (s > 0 ? (t == s - 1) : (t == Ns - 1) * kappa);
        else Lst = (s < Ns - 1 ? (t == s + 1) : (t == 0) * kappa);
        if (Ns == 1) Lst = kappa;
        const double diag = (s == t) ? 1.0 : 0.0;
        W[s * Ns + t] = c->omega[s] * diag + c->sigma[s] * Lst;  // omega + sigma L
        Z[s * Ns + t] = dm * W[s * Ns + t] + diag - Lst;          // (d - m0) W + 1 - L
        ID[s * Ns + t] = diag;
        MS[s * Ns + t] = dm * diag;
      }
  }
  for (auto &m : c->mat)
    for (double x : m)
      if (!std::isfinite(x)) return false;
  return true;
}

// M5 and M5^T of Eq. 8 as recurrences along s, for the hop epilogues.  With
// A = (d - m0) sqrt(omega) (1 + cL) + omega^{-1/2} (1 - L) (cyclic bidiagonal through the
// corner kappa of L, Eq. 4) and P = sqrt(omega) (1 + cL): M5 = P A^{-1}, M5^T = A^{-T} P^T.
// A chirality's recurrence visits s in one direction (step j at s = j, or Ns - 1 - j when
// backward: chirality - for M5, chirality + for M5^T); every step uses the values of the
// step before it, and step 0 those of the last step scaled by kappa:
//   g_j = PS_j v_j + PN_j vp,  z_j = (g_j - BB_j zp) AI_j,  u_j = QS_j z_j + QN_j zp,
// with the first zp = kappa z_last from the closure z_last = sum_j W_j v_j and the first
// vp = kappa v_last.  Table: per chirality, RC_N reals per step.
enum { RC_PS, RC_PN, RC_BB, RC_AI, RC_QS, RC_QN, RC_W, RC_N = 8 };

void apply_recurrence(const double *T, int Ns, bool bwd, double kappa, const double *v, double *u) {
  auto sg = [&](int j) { return bwd ? Ns - 1 - j : j; };
  double zc = 0.0;
  for (int j = 0; j < Ns; ++j) zc += T[j * RC_N + RC_W] * v[sg(j)];
  double zp = kappa * zc, vp = kappa * v[sg(Ns - 1)];
  for (int j = 0; j < Ns; ++j) {
    const double *t = T + j * RC_N;
    const int s = sg(j);
    const double g = t[RC_PS] * v[s] + t[RC_PN] * vp;
    const double z = (g - t[RC_BB] * zp) * t[RC_AI];
    u[s] = t[RC_QS] * z + t[RC_QN] * zp;
    zp = z;
    vp = v[s];
  }
}

// builds the tables and checks each against the dense M5 / M5^T column by column
bool build_recurrences(dwf_ctx *c) {
  const int Ns = c->Ns;
  const double kappa = -c->mq / (2.0 * c->m0);
  const double dm = kD - c->m0;
  std::vector<double> a(Ns), beta(Ns), sw(Ns), cc(Ns), lam(Ns), u(Ns), v(Ns);
  for (int s = 0; s < Ns; ++s) {
    sw[s] = sqrt(c->omega[s]);
    a[s] = dm * sw[s] + 1.0 / sw[s];
    beta[s] = dm * c->sigma[s] / sw[s] - 1.0 / sw[s];
    cc[s] = c->sigma[s] / c->omega[s];
  }
  for (int tr = 0; tr < 2; ++tr) {
    c->rec[tr].assign((size_t)2 * Ns * RC_N, 0.0);
    for (int chi = 0; chi < 2; ++chi) {
      const bool bwd = (chi ^ tr) != 0;
      auto sg = [&](int j) { return bwd ? Ns - 1 - j : j; };
      double *T = c->rec[tr].data() + (size_t)chi * Ns * RC_N;
      for (int j = 0; j < Ns; ++j) {
        const int s = sg(j), n = sg((j + Ns - 1) % Ns);  // this step's s and the step before's
        double *t = T + j * RC_N;
        if (a[s] == 0.0) return false;
        t[RC_AI] = 1.0 / a[s];
        if (tr == 0) {  // M5 = P A^{-1}: solve, then u = sqrt(omega) (z + c L z)
          t[RC_PS] = 1.0;
          t[RC_PN] = 0.0;
          t[RC_BB] = beta[s];
          t[RC_QS] = sw[s];
          t[RC_QN] = sw[s] * cc[s];
        } else {  // M5^T = A^{-T} P^T: g = P^T v, then solve with A^T
          t[RC_PS] = sw[s];
          t[RC_PN] = sw[n] * cc[n];
          t[RC_BB] = beta[n];
          t[RC_QS] = 1.0;
          t[RC_QN] = 0.0;
        }
      }
      // closure: z_last = sum_j lam_j g_j (forward substitution with z depending linearly on
      // z_last through step 0), and g_j = PS_j v_j + PN_j vp_j gives the weights on v
      double q = -T[RC_BB] * kappa * T[RC_AI];
      for (int j = 1; j < Ns; ++j) q = -T[j * RC_N + RC_BB] * q * T[j * RC_N + RC_AI];
      const double den = 1.0 - q;
      if (den == 0.0) return false;
      double r = 1.0;
      for (int j = Ns - 1; j >= 0; --j) {
        lam[j] = T[j * RC_N + RC_AI] * r / den;
        r *= -T[j * RC_N + RC_BB] * T[j * RC_N + RC_AI];
      }
      for (int j = 0; j < Ns; ++j) {
        double w = lam[j] * T[j * RC_N + RC_PS];
        if (j + 1 < Ns) w += lam[j + 1] * T[(j + 1) * RC_N + RC_PN];
        if (j == Ns - 1) w += kappa * lam[0] * T[RC_PN];
        T[j * RC_N + RC_W] = w;
      }
      // check: the recurrence reproduces every column of the dense matrix
      const double *M = c->mat[tr ? MK_M5T : MK_M5].data() + (size_t)chi * Ns * Ns;
      double mmax = 0.0;
      for (int i = 0; i < Ns * Ns; ++i) mmax = std::max(mmax, fabs(M[i]));
      for (int t0 = 0; t0 < Ns; ++t0) {
        std::fill(v.begin(), v.end(), 0.0);
        v[t0] = 1.0;
        apply_recurrence(T, Ns, bwd, kappa, v.data(), u.data());
        for (int s = 0; s < Ns; ++s)
          if (!(fabs(u[s] - M[s * Ns + t0]) <= 1e-11 * mmax)) return false;
      }
    }
  }
  return true;
}

// ------------------------------------------------------------------ buffers

dwf_status get_buf(dwf_ctx *c, const std::string &name, int prec, Field *f) {
  const size_t n = (size_t)c->h * c->Ns;
  const size_t bytes = n * site_bytes(prec);
  const std::string key = name + "#" + std::to_string(prec);
  Buf &b = c->bufs[key];
  if (!b.v) {
    CK(dmalloc(&b.v, bytes, c->device, c->stream));
    b.bytes = bytes;
    if (prec >= P_F16) CK(dmalloc((void **)&b.nrm, n * sizeof(float), c->device, c->stream));
    CK(cudaMemsetAsync(b.v, 0, bytes, c->stream));
    if (b.nrm) CK(cudaMemsetAsync(b.nrm, 0, n * sizeof(float), c->stream));
    CK(cudaStreamSynchronize(c->stream));  // ordered before any use on another stream
  }
  f->v = b.v;
  f->nrm = b.nrm;
  return DWF_OK;
}

dwf_status get_raw(dwf_ctx *c, const std::string &name, size_t bytes, void **p) {
  Buf &b = c->bufs["raw:" + name];
  if (b.v && b.bytes < bytes) {
    dfree(b.v, c->stream);
    b.v = nullptr;
  }
  if (!b.v) {
    CK(dmalloc(&b.v, bytes, c->device, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // ordered before any use on another stream
    b.bytes = bytes;
  }
  *p = b.v;
  return DWF_OK;
}

Geom geom(const dwf_ctx *c) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.d[i] = c->dims[i];
  g.h = c->h;
  g.Ns = c->Ns;
  return g;
}

// ------------------------------------------------------------------ launches (counted, optionally timed)

cudaEvent_t next_event(dwf_ctx *c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

struct Timed {
  dwf_ctx *c;
  cudaStream_t st;
  int cls;
  cudaEvent_t a = nullptr;
  Timed(dwf_ctx *c_, cudaStream_t st_, int cls_) : c(c_), st(st_), cls(cls_) {
    if (c->profiling) {
      a = next_event(c);
      cudaEventRecord(a, st);
    }
    c->launches++;
  }
  ~Timed() {
    if (c->profiling) {
      cudaEvent_t b = next_event(c);
      cudaEventRecord(b, st);
      c->prof.push_back({cls, a, b});
    }
  }
};

cudaError_t hop_any(int prec, int epi, const HopArgs &a, cudaStream_t st) {
  switch (prec) {
    case P_F64: return hop_launch<P_F64>(epi, a, st);
    case P_F32: return hop_launch<P_F32>(epi, a, st);
    case P_F16: return hop_launch<P_F16>(epi, a, st);
    case P_BF16: return hop_launch<P_BF16>(epi, a, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t smix_any(int prec, int mode, const SmixArgs &a, cudaStream_t st) {
  switch (prec) {
    case P_F64: return smix_launch<P_F64>(mode, a, st);
    case P_F32: return smix_launch<P_F32>(mode, a, st);
    case P_F16: return smix_launch<P_F16>(mode, a, st);
    case P_BF16: return smix_launch<P_BF16>(mode, a, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t norm2_any(int prec, const VecArgs &v, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return norm2_launch<P_F64>(v, sm, st);
    case P_F32: return norm2_launch<P_F32>(v, sm, st);
    case P_F16: return norm2_launch<P_F16>(v, sm, st);
    case P_BF16: return norm2_launch<P_BF16>(v, sm, st);
  }
  return cudaErrorInvalidValue;
}
// to_p != 0: FP64 -> prec, else prec -> FP64
cudaError_t convert_any(int prec, int to_p, const VecArgs &v, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return convert_launch<P_F64>(to_p, v, sm, st);
    case P_F32: return convert_launch<P_F32>(to_p, v, sm, st);
    case P_F16: return convert_launch<P_F16>(to_p, v, sm, st);
    case P_BF16: return convert_launch<P_BF16>(to_p, v, sm, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t accum_any(int prec, const VecArgs &v, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return accum_launch<P_F64>(v, sm, st);
    case P_F32: return accum_launch<P_F32>(v, sm, st);
    case P_F16: return accum_launch<P_F16>(v, sm, st);
    case P_BF16: return accum_launch<P_BF16>(v, sm, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t pack_any(int prec, const double *host, Field f, Geom g, int par, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return pack_launch<P_F64>(host, f, g, par, sm, st);
    case P_F32: return pack_launch<P_F32>(host, f, g, par, sm, st);
    case P_F16: return pack_launch<P_F16>(host, f, g, par, sm, st);
    case P_BF16: return pack_launch<P_BF16>(host, f, g, par, sm, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t unpack_any(int prec, Field f, double *host, Geom g, int par, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return unpack_launch<P_F64>(f, host, g, par, sm, st);
    case P_F32: return unpack_launch<P_F32>(f, host, g, par, sm, st);
    case P_F16: return unpack_launch<P_F16>(f, host, g, par, sm, st);
    case P_BF16: return unpack_launch<P_BF16>(f, host, g, par, sm, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t gauge_any(int prec, const double *U, void *G, Geom g, int par, int sm, cudaStream_t st) {
  switch (prec) {
    case P_F64: return gauge_launch<P_F64>(U, G, g, par, sm, st);
    case P_F32: return gauge_launch<P_F32>(U, G, g, par, sm, st);
    case P_F16: return gauge_launch<P_F16>(U, G, g, par, sm, st);
    case P_BF16: return gauge_launch<P_BF16>(U, G, g, par, sm, st);
  }
  return cudaErrorInvalidValue;
}

size_t link_bytes_per_site(int prec) {
  switch (prec) {
    case P_F64: return PT<P_F64>::SITE_LREALS * sizeof(double);
    case P_F32: return PT<P_F32>::SITE_LREALS * sizeof(float);
    default: return PT<P_F16>::SITE_LREALS * 2;
  }
}

// doubled gauge field of precision prec, built on first use (in the shared gauge object
// when the context is attached to one, once for all its contexts)
dwf_status ensure_gauge(dwf_ctx *c, int prec, cudaStream_t st) {
  if (!c->gauge_loaded) return fail(c, DWF_ENOGAUGE, "dwf_load_gauge has not been called");
  if (c->gauge_ready[prec]) return DWF_OK;
  if (dwf_gauge *G = c->shared) {
    std::lock_guard<std::mutex> lock(G->mu);
    if (!G->ready[prec]) {
      for (int p = 0; p < 2; ++p) {
        if (!G->d_gauge[prec][p])
          CK(dmalloc(&G->d_gauge[prec][p], (size_t)G->h * link_bytes_per_site(prec), G->device, G->stream));
        CK(gauge_any(prec, G->d_U, G->d_gauge[prec][p], geom(c), p, c->sm_count, G->stream));
      }
      CK(cudaStreamSynchronize(G->stream));  // complete before any context's stream uses it
      G->ready[prec] = true;
    }
    for (int p = 0; p < 2; ++p) c->d_gauge[prec][p] = G->d_gauge[prec][p];
    c->gauge_ready[prec] = true;
    return DWF_OK;
  }
  for (int p = 0; p < 2; ++p) {
    if (!c->d_gauge[prec][p])
      CK(dmalloc(&c->d_gauge[prec][p], (size_t)c->h * link_bytes_per_site(prec), c->device, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    Timed t(c, st, DWF_KC_OTHER);
    CK(gauge_any(prec, c->d_U, c->d_gauge[prec][p], geom(c), p, c->sm_count, st));
  }
  c->gauge_ready[prec] = true;
  return DWF_OK;
}

// drops the context's gauge: its private copies, or its reference to a shared gauge
void release_gauge(dwf_ctx *c);

HopArgs hop_args(dwf_ctx *c, int prec, int outpar) {
  HopArgs a;
  memset(&a, 0, sizeof(a));
  a.gauge = c->d_gauge[prec][outpar];
  a.nbr = c->d_nbr[outpar];
  a.h = c->h;
  a.Ns = c->Ns;
  a.fin = FIN_RED2;
  a.sc = c->d_sc;
  a.partials = c->d_part;
  a.ticket = c->d_ticket;
  a.wait_tries = c->wait_tries;
  a.skip_copies = c->skip_copies;
  return a;
}

// launch shapes picked by the autotuner, per (device, precision, epilogue, Ns, volume class)
TuneCache g_tune;

TuneCache::Key tune_key(const dwf_ctx *c, int prec, int epi) {
  return TuneCache::Key(c->device, prec, epi, c->Ns, volume_class(c->h));
}

dwf_status hop(dwf_ctx *c, cudaStream_t st, int prec, int epi, HopArgs a, int cls) {
  HopShape shape;
  if (prec != P_F64 && c->use_tuned && g_tune.get(tune_key(c, prec, epi), &shape)) {
    a.shape_threads = shape.threads;
    a.shape_persistent = shape.persistent ? 1 : 0;
  }
  Timed t(c, st, cls);
  CK(hop_any(prec, epi, a, st));
  return DWF_OK;
}

const void *dmat(dwf_ctx *c, int prec, int kind) { return c->dmat[mat_index(prec)][kind]; }

// the hop epilogue's matrix along s, M5 or M5^T: dense (FP32 arithmetic) and as a
// recurrence table (FP64)
void set_m5(HopArgs &a, dwf_ctx *c, int prec, bool trans) {
  a.K = dmat(c, prec, trans ? MK_M5T : MK_M5);
  a.rec = c->drec[mat_index(prec)][trans ? 1 : 0];
  a.mtrans = trans ? 1 : 0;
  a.kappa = -c->mq / (2.0 * c->m0);
}

dwf_status smix(dwf_ctx *c, cudaStream_t st, int prec, int mode, Field in, Field out, int kind,
                double coef, int cls, Field out2 = Field{nullptr, nullptr}, int kind2 = MK_ID,
                Field r = Field{nullptr, nullptr}, Field p = Field{nullptr, nullptr}, int use_flag = 0) {
  SmixArgs a;
  memset(&a, 0, sizeof(a));
  a.in = in;
  a.out = out;
  a.out2 = out2;
  a.r = r;
  a.p = p;
  a.K = dmat(c, prec, kind);
  a.K2 = dmat(c, prec, kind2);
  a.coef = coef;
  a.h = c->h;
  a.Ns = c->Ns;
  a.use_flag = use_flag;
  a.sc = c->d_sc;
  Timed t(c, st, cls);
  CK(smix_any(prec, mode, a, st));
  return DWF_OK;
}

dwf_status norm2(dwf_ctx *c, cudaStream_t st, int prec, Field f, int fin) {
  VecArgs v;
  memset(&v, 0, sizeof(v));
  v.a = f;
  v.n = c->h * c->Ns;
  v.Ns = c->Ns;
  v.fin = fin;
  v.sc = c->d_sc;
  v.partials = c->d_part;
  v.ticket = c->d_ticket;
  Timed t(c, st, DWF_KC_OTHER);
  CK(norm2_any(prec, v, c->sm_count, st));
  return DWF_OK;
}

// dst (prec_dst) = src (prec_src); one side must be FP64 unless both are equal
dwf_status convert(dwf_ctx *c, cudaStream_t st, int prec_src, Field src, int prec_dst, Field dst, int cls) {
  VecArgs v;
  memset(&v, 0, sizeof(v));
  v.a = src;
  v.b = dst;
  v.n = c->h * c->Ns;
  v.Ns = c->Ns;
  Timed t(c, st, cls);
  if (prec_src == P_F64) {
    CK(convert_any(prec_dst, 1, v, c->sm_count, st));
  } else if (prec_dst == P_F64) {
    CK(convert_any(prec_src, 0, v, c->sm_count, st));
  } else {
    return fail(c, DWF_EINVAL, "conversion between two reduced precisions");
  }
  return DWF_OK;
}

dwf_status pull_scalars(dwf_ctx *c, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (c->h_sc->error) {
    // a bounded wait gave up: clear the error word and the reduction ticket
    cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), st);
    c->h_sc->error = 0;
    cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CGScalars), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    return fail(c, DWF_ETIMEOUT, "a device-side wait for the TMA link copy timed out");
  }
  return DWF_OK;
}

dwf_status push_scalars(dwf_ctx *c, cudaStream_t st) {
  CK(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CGScalars), cudaMemcpyHostToDevice, st));
  return DWF_OK;
}

// ------------------------------------------------------------------ operator compositions

// q = C^dag v on Schur parity sp (Eq. 11, adjoint via gamma5-hermiticity of D_w):
// C^dag v = g5 (1 - D^{sp,op} M5^T D^{op,sp} M5^T) g5 v
//   w = M5^T g5 v;  t = M5^T D^{op,sp} w = -1/2 M5^T H w;  q = v + 1/2 g5 H t
dwf_status op_cdag(dwf_ctx *c, cudaStream_t st, int prec, int sp, Field v, Field q, Field w, Field t,
                   int cls) {
  const int op = 1 - sp;
  TRY(smix(c, st, prec, S_G5, v, w, MK_M5T, 1.0, cls));
  HopArgs a = hop_args(c, prec, op);
  a.in = w;
  a.out = t;
  set_m5(a, c, prec, true);
  a.coef = -0.5;
  TRY(hop(c, st, prec, E_M, a, cls));
  HopArgs b = hop_args(c, prec, sp);
  b.in = t;
  b.y = v;
  b.out = q;
  b.coef = 0.5;
  TRY(hop(c, st, prec, E_XPAY_G5, b, cls));
  return DWF_OK;
}

// out = C v = v - M5 D^{sp,op} M5 D^{op,sp} v:  u = -1/2 M5 H v;  out = v + 1/2 M5 H u
dwf_status op_c(dwf_ctx *c, cudaStream_t st, int prec, int sp, Field v, Field out, Field u, int cls) {
  const int op = 1 - sp;
  HopArgs a = hop_args(c, prec, op);
  a.in = v;
  a.out = u;
  set_m5(a, c, prec, false);
  a.coef = -0.5;
  TRY(hop(c, st, prec, E_M, a, cls));
  HopArgs b = hop_args(c, prec, sp);
  b.in = u;
  b.y = v;
  b.out = out;
  set_m5(b, c, prec, false);
  b.coef = 0.5;
  TRY(hop(c, st, prec, E_M_XPAY, b, cls));
  return DWF_OK;
}

// full-lattice operator on both parities: out_p = Z in_p - 1/2 H (W in)_{1-p}
// (kindW, kindZ) = (MK_W, MK_Z) gives D(mq) of Eq. 5; (MK_ID, MK_MASS) gives D_w of Eq. 2.
dwf_status op_full(dwf_ctx *c, cudaStream_t st, int prec, const Field in[2], Field out[2], int kindW,
                   int kindZ, int cls) {
  Field t[2], z[2];
  for (int p = 0; p < 2; ++p) {
    TRY(get_buf(c, "full_t" + std::to_string(p), prec, &t[p]));
    TRY(get_buf(c, "full_z" + std::to_string(p), prec, &z[p]));
    TRY(smix(c, st, prec, S_DUAL, in[p], t[p], kindW, 1.0, cls, z[p], kindZ));
  }
  for (int p = 0; p < 2; ++p) {
    HopArgs a = hop_args(c, prec, p);
    a.in = t[1 - p];
    a.y = z[p];
    a.out = out[p];
    a.coef = -0.5;
    TRY(hop(c, st, prec, E_XPAY, a, cls));
  }
  return DWF_OK;
}

dwf_status check_ctx(dwf_ctx *c) {
  if (!c) return DWF_EINVAL;
  c->err.clear();
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, DWF_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return DWF_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// a context of one part of a domain decomposition only works through dwf_part_apply
dwf_status not_part(dwf_ctx *c) {
  if (c->part) return fail(c, DWF_EINVAL, "a partitioned context is applied with dwf_part_apply");
  return DWF_OK;
}

void begin_profile(dwf_ctx *c, bool on) {
  c->profiling = on;
  c->ev_used = 0;
  c->prof.clear();
}

void end_profile(dwf_ctx *c, dwf_solve_stats *stats) {
  if (!c->profiling) return;
  if (stats)
    for (auto &r : c->prof) {
      float ms = 0;
      cudaEventElapsedTime(&ms, r.a, r.b);
      stats->class_ms[r.cls] += ms;
      stats->class_launches[r.cls] += 1;
    }
  c->profiling = false;
}

}  // namespace

// ====================================================================== C-ABI

extern "C" {

const char *dwf_status_string(dwf_status st) { return status_name(st); }

const char *dwf_last_error(const dwf_ctx *c) { return c ? c->err.c_str() : "null context"; }

dwf_status dwf_debug_set_wait(dwf_ctx *c, unsigned wait_tries, int skip_copies) {
  if (!c) return DWF_EINVAL;
  c->wait_tries = wait_tries ? wait_tries : kWaitTries;
  c->skip_copies = skip_copies ? 1 : 0;
  return DWF_OK;
}

void dwf_solve_params_default(dwf_solve_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-10;
  p->delta = 0.0;
  p->max_iter = 100000;
  p->inner_prec = DWF_PREC_F32;
  p->mode = DWF_MODE_AUTO;
  p->system = DWF_SYS_FULL;
  p->schur_parity = 1;
  p->check_every = 8;
  p->use_graph = 1;
  p->profile = 0;
  p->schur_target_pct = 50;
}

dwf_status dwf_create(const int dims[4], int Ns, double m0, double mq, const double *omega,
                      const double *sigma, dwf_ctx **out) {
  if (!dims || !omega || !sigma || !out) return DWF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1)) return DWF_EINVAL;
  if (Ns < 1 || Ns > 64 || !(m0 > 0.0 && m0 < 2.0) || !(mq >= 0.0)) return DWF_EINVAL;
  for (int s = 0; s < Ns; ++s)
    if (!(omega[s] > 0.0) || !std::isfinite(sigma[s])) return DWF_EINVAL;
  const long V4 = (long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V4 / 2 > (1L << 30)) return DWF_EINVAL;

  dwf_ctx *c = new dwf_ctx();
  for (int i = 0; i < 4; ++i) c->dims[i] = dims[i];
  c->Ns = Ns;
  c->V4 = V4;
  c->h = V4 / 2;
  c->m0 = m0;
  c->mq = mq;
  c->omega.assign(omega, omega + Ns);
  c->sigma.assign(sigma, sigma + Ns);
  if (!build_matrices(c) || !build_recurrences(c)) {
    delete c;
    return DWF_EINVAL;
  }
  auto bail = [&](cudaError_t e) {
    dwf_destroy(c);
    return e == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail(e);
  if ((e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess)
    return bail(e);
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
  // matrices in both arithmetic precisions, kernel order K[chi][t][s]
  const size_t nm = (size_t)2 * Ns * Ns;
  std::vector<double> kd(nm);
  std::vector<float> kf(nm);
  for (int k = 0; k < MK_COUNT; ++k) {
    for (int chi = 0; chi < 2; ++chi)
      for (int s = 0; s < Ns; ++s)
        for (int t = 0; t < Ns; ++t) {
          const double v = c->mat[k][(size_t)chi * Ns * Ns + (size_t)s * Ns + t];
          kd[(size_t)chi * Ns * Ns + (size_t)t * Ns + s] = v;
          kf[(size_t)chi * Ns * Ns + (size_t)t * Ns + s] = (float)v;
        }
    if ((e = dmalloc(&c->dmat[0][k], nm * sizeof(double), c->device, c->stream)) != cudaSuccess) return bail(e);
    if ((e = dmalloc(&c->dmat[1][k], nm * sizeof(float), c->device, c->stream)) != cudaSuccess) return bail(e);
    if ((e = cudaMemcpyAsync(c->dmat[0][k], kd.data(), nm * sizeof(double), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
      return bail(e);
    if ((e = cudaMemcpyAsync(c->dmat[1][k], kf.data(), nm * sizeof(float), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
      return bail(e);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e);  // kd, kf are reused
  }
  for (int tr = 0; tr < 2; ++tr) {
    const size_t nr = c->rec[tr].size();
    std::vector<float> rf(c->rec[tr].begin(), c->rec[tr].end());
    if ((e = dmalloc(&c->drec[0][tr], nr * sizeof(double), c->device, c->stream)) != cudaSuccess) return bail(e);
    if ((e = dmalloc(&c->drec[1][tr], nr * sizeof(float), c->device, c->stream)) != cudaSuccess) return bail(e);
    if ((e = cudaMemcpyAsync(c->drec[0][tr], c->rec[tr].data(), nr * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return bail(e);
    if ((e = cudaMemcpyAsync(c->drec[1][tr], rf.data(), nr * sizeof(float), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
      return bail(e);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e);  // rf is a temporary
  }
  Geom g = geom(c);
  for (int p = 0; p < 2; ++p) {
    if ((e = dmalloc((void **)&c->d_nbr[p], (size_t)c->h * 8 * sizeof(int), c->device, c->stream)) != cudaSuccess)
      return bail(e);
    if ((e = neighbours_launch(c->d_nbr[p], g, p, c->sm_count, c->stream)) != cudaSuccess) return bail(e);
  }
  if ((e = dmalloc((void **)&c->d_sc, sizeof(CGScalars), c->device, c->stream)) != cudaSuccess) return bail(e);
  if (!(c->h_sc = static_cast<CGScalars *>(pinned_get(sizeof(CGScalars))))) return bail(cudaErrorMemoryAllocation);
  memset(c->h_sc, 0, sizeof(CGScalars));
  c->part_len = std::max<size_t>((size_t)c->h, 8192);
  if ((e = dmalloc((void **)&c->d_part, c->part_len * sizeof(double), c->device, c->stream)) != cudaSuccess)
    return bail(e);
  if ((e = dmalloc((void **)&c->d_ticket, sizeof(unsigned), c->device, c->stream)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), c->stream)) != cudaSuccess) return bail(e);
  if ((e = cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(CGScalars), cudaMemcpyHostToDevice, c->stream)) !=
      cudaSuccess)
    return bail(e);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(e);
  *out = c;
  return DWF_OK;
}

dwf_status dwf_destroy(dwf_ctx *c) {
  if (!c) return DWF_OK;
  cudaSetDevice(c->device);
  // every call on the context has finished its work (each waits for its stream), so the
  // buffers go back to the pool in the context stream's order: nothing synchronises the
  // device, and solves of other contexts keep running
  if (c->stream) {
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->bufs) {
      dfree(kv.second.v, c->stream);
      dfree(kv.second.nrm, c->stream);
    }
    for (auto &row : c->dmat)
      for (void *p : row) dfree(p, c->stream);
    for (auto &row : c->drec)
      for (void *p : row) dfree(p, c->stream);
    release_gauge(c);
    dfree(c->d_Ug, c->stream);
    for (int *p : c->d_nbr) dfree(p, c->stream);
    dfree(c->d_sc, c->stream);
    dfree(c->d_part, c->stream);
    dfree(c->d_ticket, c->stream);
    cudaStreamSynchronize(c->stream);
  }
  pinned_put(c->h_sc, sizeof(CGScalars));
  pinned_put(c->h_scb, c->h_scb_cap * sizeof(CGScalars));
  pinned_put(c->h_face, c->h_face_bytes);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return DWF_OK;
}

dwf_status dwf_load_gauge_dev(dwf_ctx *c, const double *d_U, void *stream) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!d_U) return fail(c, DWF_EINVAL, "null gauge pointer");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  const size_t bytes = (size_t)c->V4 * 72 * sizeof(double);
  if (c->shared) release_gauge(c);  // back to a private copy
  if (!c->d_U) {
    CK(dmalloc((void **)&c->d_U, bytes, c->device, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaMemcpyAsync(c->d_U, d_U, bytes, cudaMemcpyDeviceToDevice, st));
  c->gauge_loaded = true;
  for (int p = 0; p < 4; ++p) c->gauge_ready[p] = false;
  // the FP64 and FP32 forms are always needed (restart operator, inner CG)
  TRY(ensure_gauge(c, P_F64, st));
  TRY(ensure_gauge(c, P_F32, st));
  CK(cudaStreamSynchronize(st));
  return DWF_OK;
}

dwf_status dwf_load_gauge(dwf_ctx *c, const double *U) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!U) return fail(c, DWF_EINVAL, "null gauge pointer");
  const size_t bytes = (size_t)c->V4 * 72 * sizeof(double);
  if (c->shared) release_gauge(c);  // back to a private copy
  if (!c->d_U) CK(dmalloc((void **)&c->d_U, bytes, c->device, c->stream));
  CK(cudaMemcpyAsync(c->d_U, U, bytes, cudaMemcpyHostToDevice, c->stream));
  c->gauge_loaded = true;
  for (int p = 0; p < 4; ++p) c->gauge_ready[p] = false;
  TRY(ensure_gauge(c, P_F64, c->stream));
  TRY(ensure_gauge(c, P_F32, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

}  // extern "C"

namespace {

void gauge_unref(dwf_gauge *G) {
  bool last;
  {
    std::lock_guard<std::mutex> lock(G->mu);
    last = --G->refs == 0;
  }
  if (!last) return;
  cudaSetDevice(G->device);
  dfree(G->d_U, G->stream);
  for (auto &row : G->d_gauge)
    for (void *p : row) dfree(p, G->stream);
  cudaStreamSynchronize(G->stream);
  cudaStreamDestroy(G->stream);
  delete G;
}

void release_gauge(dwf_ctx *c) {
  if (c->shared) {
    // the context's stream has finished its work with the shared arrays
    gauge_unref(c->shared);
    c->shared = nullptr;
    c->d_U = nullptr;
    for (auto &row : c->d_gauge)
      for (auto &p : row) p = nullptr;
  } else {
    dfree(c->d_U, c->stream);
    c->d_U = nullptr;
    for (auto &row : c->d_gauge)
      for (auto &p : row) {
        dfree(p, c->stream);
        p = nullptr;
      }
  }
  c->gauge_loaded = false;
  for (bool &r : c->gauge_ready) r = false;
}

dwf_status gauge_create_impl(const int dims[4], const double *U, bool on_device, void *stream, dwf_gauge **out) {
  if (!dims || !U || !out) return DWF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2 || (dims[i] & 1)) return DWF_EINVAL;
  dwf_gauge *G = new dwf_gauge();
  memcpy(G->dims, dims, sizeof(G->dims));
  G->V4 = (long)dims[0] * dims[1] * dims[2] * dims[3];
  G->h = G->V4 / 2;
  const size_t bytes = (size_t)G->V4 * 72 * sizeof(double);
  cudaError_t e = cudaGetDevice(&G->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&G->sm_count, cudaDevAttrMultiProcessorCount, G->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dmalloc((void **)&G->d_U, bytes, G->device, G->stream);
  if (e == cudaSuccess && on_device && stream) {
    // the copy waits for the caller's stream, where d_U may still be being written
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      e = cudaEventRecord(ev, (cudaStream_t)stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(G->stream, ev, 0);
      cudaEventDestroy(ev);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_U, U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  if (e != cudaSuccess) {
    if (G->stream) {
      dfree(G->d_U, G->stream);
      cudaStreamSynchronize(G->stream);
      cudaStreamDestroy(G->stream);
    }
    delete G;
    return e == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
  }
  *out = G;
  return DWF_OK;
}

}  // namespace

extern "C" {

dwf_status dwf_gauge_create(const int dims[4], const double *U, dwf_gauge **out) {
  return gauge_create_impl(dims, U, false, nullptr, out);
}

dwf_status dwf_gauge_create_dev(const int dims[4], const double *d_U, void *stream, dwf_gauge **out) {
  return gauge_create_impl(dims, d_U, true, stream, out);
}

dwf_status dwf_gauge_release(dwf_gauge *g) {
  if (g) gauge_unref(g);
  return DWF_OK;
}

dwf_status dwf_attach_gauge(dwf_ctx *c, dwf_gauge *g) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!g) return fail(c, DWF_EINVAL, "null gauge handle");
  if (memcmp(g->dims, c->dims, sizeof(c->dims)) != 0) return fail(c, DWF_EINVAL, "gauge lattice differs from the context's");
  if (g->device != c->device) return fail(c, DWF_EINVAL, "gauge field lives on another device");
  if (c->shared == g) return DWF_OK;
  CK(cudaStreamSynchronize(c->stream));
  release_gauge(c);
  {
    std::lock_guard<std::mutex> lock(g->mu);
    ++g->refs;
  }
  c->shared = g;
  c->d_U = g->d_U;
  c->gauge_loaded = true;
  // the FP64 and FP32 forms are always needed (restart operator, inner CG)
  TRY(ensure_gauge(c, P_F64, c->stream));
  TRY(ensure_gauge(c, P_F32, c->stream));
  return DWF_OK;
}

dwf_status dwf_apply_eo_dev(dwf_ctx *c, int op, int prec, int parity, const double *d_in, double *d_out,
                            void *stream) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!d_in || !d_out || !aligned16(d_in) || !aligned16(d_out))
    return fail(c, DWF_EINVAL, "null or non-16-byte-aligned field pointer");
  if (!valid_prec(prec)) return fail(c, DWF_EINVAL, "unknown precision");
  if (op < DWF_OP_DEO || op > DWF_OP_DW) return fail(c, DWF_EINVAL, "unknown operator");
  const bool needs_parity = op >= DWF_OP_M5 && op <= DWF_OP_CCDAG;
  if (needs_parity && parity != 0 && parity != 1) return fail(c, DWF_EINVAL, "parity must be 0 or 1");
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double);
  if ((const char *)d_in < (const char *)d_out + full && (const char *)d_out < (const char *)d_in + full)
    return fail(c, DWF_EINVAL, "in and out overlap");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  TRY(ensure_gauge(c, prec, st));
  const Geom g = geom(c);
  const int cls = DWF_KC_OTHER;
  CK(cudaMemsetAsync(d_out, 0, full, st));

  Field in[2], out[2], tA, tB, tC;
  for (int p = 0; p < 2; ++p) {
    TRY(get_buf(c, "ap_in" + std::to_string(p), prec, &in[p]));
    TRY(get_buf(c, "ap_out" + std::to_string(p), prec, &out[p]));
  }
  TRY(get_buf(c, "ap_tA", prec, &tA));
  TRY(get_buf(c, "ap_tB", prec, &tB));
  TRY(get_buf(c, "ap_tC", prec, &tC));
  auto pack = [&](int p) -> dwf_status {
    Timed t(c, st, cls);
    CK(pack_any(prec, d_in, in[p], g, p, c->sm_count, st));
    return DWF_OK;
  };
  auto unpack = [&](int p) -> dwf_status {
    Timed t(c, st, cls);
    CK(unpack_any(prec, out[p], d_out, g, p, c->sm_count, st));
    return DWF_OK;
  };
  switch (op) {
    case DWF_OP_DEO:
    case DWF_OP_DOE: {
      const int outp = op == DWF_OP_DEO ? 0 : 1;
      TRY(pack(1 - outp));
      HopArgs a = hop_args(c, prec, outp);
      a.in = in[1 - outp];
      a.out = out[outp];
      a.coef = -0.5;
      TRY(hop(c, st, prec, E_PLAIN, a, cls));
      TRY(unpack(outp));
      break;
    }
    case DWF_OP_M5:
    case DWF_OP_M5T:
      TRY(pack(parity));
      TRY(smix(c, st, prec, S_PLAIN, in[parity], out[parity], op == DWF_OP_M5 ? MK_M5 : MK_M5T, 1.0, cls));
      TRY(unpack(parity));
      break;
    case DWF_OP_C:
      TRY(pack(parity));
      TRY(op_c(c, st, prec, parity, in[parity], out[parity], tA, cls));
      TRY(unpack(parity));
      break;
    case DWF_OP_CDAG:
      TRY(pack(parity));
      TRY(op_cdag(c, st, prec, parity, in[parity], out[parity], tA, tB, cls));
      TRY(unpack(parity));
      break;
    case DWF_OP_CCDAG:
      TRY(pack(parity));
      TRY(op_cdag(c, st, prec, parity, in[parity], tC, tA, tB, cls));
      TRY(op_c(c, st, prec, parity, tC, out[parity], tA, cls));
      TRY(unpack(parity));
      break;
    case DWF_OP_DFULL:
    case DWF_OP_DW:
      TRY(pack(0));
      TRY(pack(1));
      TRY(op_full(c, st, prec, in, out, op == DWF_OP_DFULL ? MK_W : MK_ID, op == DWF_OP_DFULL ? MK_Z : MK_MASS,
                  cls));
      TRY(unpack(0));
      TRY(unpack(1));
      break;
  }
  CK(cudaStreamSynchronize(st));
  return pull_scalars(c, st);
}

dwf_status dwf_apply_eo(dwf_ctx *c, int op, int prec, int parity, const double *in, double *out) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!in || !out) return fail(c, DWF_EINVAL, "null field pointer");
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double);
  void *din, *dout;
  TRY(get_raw(c, "host_in", full, &din));
  TRY(get_raw(c, "host_out", full, &dout));
  CK(cudaMemcpyAsync(din, in, full, cudaMemcpyHostToDevice, c->stream));
  TRY(dwf_apply_eo_dev(c, op, prec, parity, (const double *)din, (double *)dout, c->stream));
  CK(cudaMemcpyAsync(out, dout, full, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

}  // extern "C"

// ====================================================================== solver

namespace {

struct SolveState {
  int prec, sp, op, K;
  Field b, xh, rh;            // FP64 on the Schur parity, one field per right-hand side
  Field w64, t64, q64, u64;   // FP64 temporaries of the restart operator (t64, u64: other parity)
  Field x, r, p, q, w, t, u;  // inner precision, one field per right-hand side (t, u: other parity)
};

size_t field_bytes(const dwf_ctx *c, int prec) { return (size_t)c->h * c->Ns * site_bytes(prec); }

// field k of a batch of fields
Field at(const dwf_ctx *c, Field f, int k, int prec) {
  Field g = f;
  if (g.v) g.v = static_cast<char *>(g.v) + (size_t)k * field_bytes(c, prec);
  if (g.nrm) g.nrm += (size_t)k * c->h * c->Ns;
  return g;
}

// K consecutive fields under one name (reallocated when a larger batch needs more)
dwf_status get_buf_k(dwf_ctx *c, const std::string &name, int prec, int K, Field *f) {
  if (K == 1) return get_buf(c, name, prec, f);
  const size_t n = (size_t)c->h * c->Ns * K;
  const size_t bytes = n * site_bytes(prec);
  Buf &b = c->bufs["batch:" + name + "#" + std::to_string(prec)];
  if (b.v && b.bytes < bytes) {
    dfree(b.v, c->stream);
    dfree(b.nrm, c->stream);
    b.v = nullptr;
    b.nrm = nullptr;
  }
  if (!b.v) {
    CK(dmalloc(&b.v, bytes, c->device, c->stream));
    b.bytes = bytes;
    if (prec >= P_F16) CK(dmalloc((void **)&b.nrm, n * sizeof(float), c->device, c->stream));
    CK(cudaMemsetAsync(b.v, 0, bytes, c->stream));
    if (b.nrm) CK(cudaMemsetAsync(b.nrm, 0, n * sizeof(float), c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  f->v = b.v;
  f->nrm = b.nrm;
  return DWF_OK;
}

// scalars, partial sums and tickets of a batch (slot k at base + k)
struct Slots {
  CGScalars *d_sc, *h_sc;
  double *d_part;
  unsigned *d_ticket;
};

dwf_status batch_slots(dwf_ctx *c, int K, Slots *sl) {
  if (K == 1) {
    *sl = Slots{c->d_sc, c->h_sc, c->d_part, c->d_ticket};
    return DWF_OK;
  }
  void *p;
  TRY(get_raw(c, "batch_sc", K * sizeof(CGScalars), &p));
  sl->d_sc = static_cast<CGScalars *>(p);
  TRY(get_raw(c, "batch_part", (size_t)K * c->part_len * sizeof(double), &p));
  sl->d_part = static_cast<double *>(p);
  TRY(get_raw(c, "batch_ticket", K * sizeof(unsigned), &p));
  sl->d_ticket = static_cast<unsigned *>(p);
  if (c->h_scb_cap < K) {
    pinned_put(c->h_scb, c->h_scb_cap * sizeof(CGScalars));
    c->h_scb = static_cast<CGScalars *>(pinned_get(K * sizeof(CGScalars)));
    c->h_scb_cap = c->h_scb ? K : 0;
    if (!c->h_scb) return fail(c, DWF_ENOMEM, "pinned host memory for the batch scalars");
  }
  sl->h_sc = c->h_scb;
  memset(sl->h_sc, 0, K * sizeof(CGScalars));
  CK(cudaMemsetAsync(sl->d_ticket, 0, K * sizeof(unsigned), c->stream));
  CK(cudaMemcpyAsync(sl->d_sc, sl->h_sc, K * sizeof(CGScalars), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

// points the context's scalar/partials/ticket at one slot (or at the batch base) for a scope
struct UseSlot {
  dwf_ctx *c;
  CGScalars *dsc, *hsc;
  double *part;
  unsigned *tick;
  UseSlot(dwf_ctx *c_, const Slots &sl, int k)
      : c(c_), dsc(c_->d_sc), hsc(c_->h_sc), part(c_->d_part), tick(c_->d_ticket) {
    c->d_sc = sl.d_sc + k;
    c->h_sc = sl.h_sc + k;
    c->d_part = sl.d_part + (size_t)k * c->part_len;
    c->d_ticket = sl.d_ticket + k;
  }
  ~UseSlot() {
    c->d_sc = dsc;
    c->h_sc = hsc;
    c->d_part = part;
    c->d_ticket = tick;
  }
};

// one inner CG iteration on A = C C^dag (Algorithm 1) for every right-hand side, five kernels:
//   p = r + beta p, w = M5^T g5 p | t = -1/2 M5^T H w | q = p + 1/2 g5 H t, |q|^2
//   u = -1/2 M5 H q | Ap = q + 1/2 M5 H u, r -= alpha Ap, x += alpha p, |r|^2, beta
dwf_status cg_iteration(dwf_ctx *c, cudaStream_t st, const SolveState &S, const Slots &sl) {
  const int P = S.prec;
  const size_t fs = field_bytes(c, P), ns = (size_t)c->h * c->Ns;
  auto batch = [&](HopArgs &a) {
    a.nrhs = S.K;
    a.fstride = fs;
    a.nstride = ns;
    a.part_stride = c->part_len;
    a.sc = sl.d_sc;
    a.partials = sl.d_part;
    a.ticket = sl.d_ticket;
  };
  {
    SmixArgs m;
    memset(&m, 0, sizeof(m));
    m.out = S.w;
    m.r = S.r;
    m.p = S.p;
    m.x = S.x;
    m.xfstride = field_bytes(c, xprec(P));
    m.K = dmat(c, P, MK_M5T);
    m.K2 = dmat(c, P, MK_ID);
    m.coef = 1.0;
    m.h = c->h;
    m.Ns = c->Ns;
    m.use_flag = 1;
    m.sc = sl.d_sc;
    m.nrhs = S.K;
    m.fstride = fs;
    m.nstride = ns;
    Timed t(c, st, DWF_KC_SMIX_P);
    CK(smix_any(P, S_CGP, m, st));
  }
  HopArgs a = hop_args(c, P, S.op);
  a.in = S.w;
  a.out = S.t;
  set_m5(a, c, P, true);
  a.coef = -0.5;
  a.use_flag = 1;
  batch(a);
  TRY(hop(c, st, P, E_M, a, DWF_KC_HOP_M5));
  HopArgs b = hop_args(c, P, S.sp);
  b.in = S.t;
  b.y = S.p;
  b.out = S.q;
  b.coef = 0.5;
  b.fin = FIN_QQ;
  b.use_flag = 1;
  batch(b);
  TRY(hop(c, st, P, E_XPAY_G5, b, DWF_KC_HOP_XPAY));
  HopArgs d = hop_args(c, P, S.op);
  d.in = S.q;
  d.out = S.u;
  set_m5(d, c, P, false);
  d.coef = -0.5;
  d.use_flag = 1;
  batch(d);
  TRY(hop(c, st, P, E_M, d, DWF_KC_HOP_M5));
  HopArgs e = hop_args(c, P, S.sp);
  e.in = S.u;
  e.y = S.q;
  e.r = S.r;
  set_m5(e, c, P, false);
  e.coef = 0.5;
  e.fin = FIN_CG;
  e.use_flag = 1;
  batch(e);
  TRY(hop(c, st, P, E_CG_UPDATE, e, DWF_KC_HOP_UPDATE));
  return DWF_OK;
}

// The autotuner: for each of the inner CG's three hop kernels (hop + M5, hop + g5 xpay and
// norm, hop + M5 + CG update and norm) not yet tuned for this device, precision, Ns and
// volume class, time every candidate launch shape (dwf_tune.h) on this solve's own fields
// -- before they hold any state: the source preparation and the arming of the scalars
// overwrite everything these launches write -- and keep the fastest for the process.  Runs
// outside any stream capture; a candidate that fails to launch is skipped.
dwf_status tune_inner(dwf_ctx *c, cudaStream_t st, const SolveState &S) {
  const int P = S.prec;
  if (P == P_F64) return DWF_OK;
  HopArgs m = hop_args(c, P, S.op);
  m.in = S.w;
  m.out = S.t;
  set_m5(m, c, P, true);
  m.coef = -0.5;
  HopArgs x = hop_args(c, P, S.sp);
  x.in = S.t;
  x.y = S.p;
  x.out = S.q;
  x.coef = 0.5;
  x.fin = FIN_NONE;
  HopArgs u = hop_args(c, P, S.sp);
  u.in = S.u;
  u.y = S.q;
  u.r = S.r;
  set_m5(u, c, P, false);
  u.coef = 0.5;
  u.fin = FIN_NONE;
  const std::pair<int, HopArgs *> classes[3] = {{E_M, &m}, {E_XPAY_G5, &x}, {E_CG_UPDATE, &u}};
  cudaEvent_t e0 = next_event(c), e1 = next_event(c);
  for (const auto &cl : classes) {
    HopShape have;
    if (g_tune.get(tune_key(c, P, cl.first), &have)) continue;
    std::vector<std::pair<HopShape, double>> timed;
    for (const HopShape &cand : hop_candidates(c->Ns)) {
      HopArgs a = *cl.second;
      a.shape_threads = cand.threads;
      a.shape_persistent = cand.persistent ? 1 : 0;
      if (hop_any(P, cl.first, a, st) != cudaSuccess) {  // warm-up; skip shapes that cannot launch
        cudaGetLastError();
        continue;
      }
      constexpr int REPS = 3;
      CK(cudaEventRecord(e0, st));
      for (int r = 0; r < REPS; ++r) CK(hop_any(P, cl.first, a, st));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      timed.emplace_back(cand, ms / REPS);
    }
    g_tune.put(tune_key(c, P, cl.first), pick_fastest(timed, HopShape{}));
  }
  return DWF_OK;
}

// FP64 restart of right-hand side k (Algorithm 2), with the context pointed at its slot:
// x_hat += x + alpha p (the last inner step, which the skipped p-update did not add), x = 0,
// r_hat = b - C C^dag x_hat, |r_hat|^2 -> red, r = r_hat in the inner precision, |r|^2 -> red2
dwf_status fp64_restart(dwf_ctx *c, cudaStream_t st, const SolveState &S, int k) {
  const Field xh = at(c, S.xh, k, P_F64), rh = at(c, S.rh, k, P_F64), bk = at(c, S.b, k, P_F64);
  const Field x = at(c, S.x, k, xprec(S.prec)), r = at(c, S.r, k, S.prec);
  {
    VecArgs v;
    memset(&v, 0, sizeof(v));
    v.a = xh;
    v.b = x;
    v.c = at(c, S.p, k, S.prec);
    v.sc = c->d_sc;
    v.n = c->h * c->Ns;
    v.Ns = c->Ns;
    Timed t(c, st, DWF_KC_F64);
    CK(accum_any(S.prec, v, c->sm_count, st));
  }
  TRY(smix(c, st, P_F64, S_G5, xh, S.w64, MK_M5T, 1.0, DWF_KC_F64));
  HopArgs a = hop_args(c, P_F64, S.op);
  a.in = S.w64;
  a.out = S.t64;
  set_m5(a, c, P_F64, true);
  a.coef = -0.5;
  TRY(hop(c, st, P_F64, E_M, a, DWF_KC_F64));
  HopArgs b = hop_args(c, P_F64, S.sp);
  b.in = S.t64;
  b.y = xh;
  b.out = S.q64;
  b.coef = 0.5;
  b.fin = FIN_NONE;
  TRY(hop(c, st, P_F64, E_XPAY_G5, b, DWF_KC_F64));
  HopArgs d = hop_args(c, P_F64, S.op);
  d.in = S.q64;
  d.out = S.u64;
  set_m5(d, c, P_F64, false);
  d.coef = -0.5;
  TRY(hop(c, st, P_F64, E_M, d, DWF_KC_F64));
  HopArgs e = hop_args(c, P_F64, S.sp);
  e.in = S.u64;
  e.y = S.q64;
  e.b = bk;
  e.out = rh;
  set_m5(e, c, P_F64, false);
  e.coef = 0.5;
  e.fin = FIN_RED;
  TRY(hop(c, st, P_F64, E_RESID, e, DWF_KC_F64));
  TRY(convert(c, st, P_F64, rh, S.prec, r, DWF_KC_F64));
  TRY(norm2(c, st, S.prec, r, FIN_RED2));
  return DWF_OK;
}

// counted flops per 5D half-site (fixed convention; hop 1320, dense M5 24 (2 Ns - 1))
double flops_cg_iter(int Ns) { return 5472.0 + 192.0 * Ns; }
double flops_restart(int Ns) { return 5328.0 + 192.0 * Ns; }
double flops_prep_recon(int Ns) { return 5160.0 + 384.0 * Ns; }

constexpr int RS_DONE = 6;  // restart flag of a right-hand side that is finished

// reliable-update trigger when the caller leaves delta to the library: fp16 inner iterations
// lose their way in long cycles (measured at 16^3x32x16: 5.7k-12.9k iterations at 0.01,
// 1.8k-1.9k at 0.3 over four sources), so they take the true residual after every fall of
// |r| by 0.3; FP32 and bf16 are fastest at 0.01
double default_delta(int prec) { return prec == P_F16 ? 0.3 : 0.01; }

// per right-hand-side bookkeeping of the host loop
struct RhsState {
  double bnorm2 = 0, rhat2 = 0, prev_rhat2 = 0, rr_last = 0, res_full = 0;
  double tol = 0;  // relative Schur residual this right-hand side is solved to
  int restarts = 0, iters = 0, mode = DWF_MODE_RELIABLE;
  bool done = false, converged = false;
  dwf_status status = DWF_OK;
};

// One solve of K systems with the same operator (rhs/sol hold K full-lattice arrays one after
// another), taken in steps by its driver: begin() forms the sources and arms the inner CG;
// while !all_done(), one interval of check_every inner iterations is enqueued
// (enqueue_interval keeps this run's own CUDA graph; record_interval only enqueues, for a
// driver that captures several runs into one graph), the batch scalars are read back
// (fetch_scalars) and process_interval() takes the FP64 restarts that fell due; then
// after_loop() reconstructs the solutions (and re-arms the systems that need a tightened
// pass) and finish() fills the stats.  solve_core drives one run; dwf_solve_ragged drives
// one per context, with the intervals of all of them in one graph.
struct SolveRun {
  dwf_ctx *c;
  int K;
  const double *d_rhs;
  double *d_sol;
  dwf_solve_params prm;
  dwf_solve_stats *S_out;
  cudaStream_t st;

  double delta = 0.01;
  bool full = false;
  int stall_iters = 500;
  bool trace = false;
  long long launches0 = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SolveState S;
  Field eta[2], etap[2], phi[2], psi[2], dpsi[2];
  int eta_of = -1;  // the right-hand side whose eta and eta' the shared fields hold
  Slots sl;
  Geom g;
  size_t full_doubles = 0, nbytes64 = 0;
  double tol_schur = 0;
  std::vector<RhsState> R;
  int escalations = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  bool use_graph = false;
  bool first_batch = true;
  bool graph_dirty = false;  // a record_interval capture of this run is out of date
  int pass = 0;              // after_loop calls so far
  std::vector<int> again;    // systems of the tightened pass
  bool tuned_saved = false, prev_tuned = true;

  SolveRun(dwf_ctx *c_, int K_, const double *rhs, double *sol, const dwf_solve_params &p, dwf_solve_stats *out,
           cudaStream_t s)
      : c(c_), K(K_), d_rhs(rhs), d_sol(sol), prm(p), S_out(out), st(s) {}
  ~SolveRun() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (tuned_saved) c->use_tuned = prev_tuned;  // the solve's own choice, not the context's
  }

  dwf_status inner_bufs() {
    TRY(get_buf_k(c, "cg_x", xprec(S.prec), K, &S.x));
    TRY(get_buf_k(c, "cg_r", S.prec, K, &S.r));
    TRY(get_buf_k(c, "cg_p", S.prec, K, &S.p));
    TRY(get_buf_k(c, "cg_q", S.prec, K, &S.q));
    TRY(get_buf_k(c, "cg_w", S.prec, K, &S.w));
    TRY(get_buf_k(c, "cg_t", S.prec, K, &S.t));
    TRY(get_buf_k(c, "cg_u", S.prec, K, &S.u));
    return DWF_OK;
  }

  // eta'_k = S1 eta_k on both parities (the shared temporaries eta, etap; nothing else
  // writes them during the solve, so a single system's are formed once)
  dwf_status prep_eta(int k) {
    if (eta_of == k) return DWF_OK;
    eta_of = k;
    for (int p = 0; p < 2; ++p) {
      {
        Timed t(c, st, DWF_KC_F64);
        CK(pack_any(P_F64, d_rhs + (size_t)k * full_doubles, eta[p], g, p, c->sm_count, st));
      }
      TRY(smix(c, st, P_F64, S_PLAIN, eta[p], etap[p], MK_S1, 1.0, DWF_KC_F64));
    }
    return DWF_OK;
  }

  // (re)arm the inner CG of right-hand side k after a restart: r_k holds r_hat in the inner
  // precision with |r|^2 = rr_conv.  Reliable updates keep p (beta from the recomputed
  // residual), defect correction restarts from p = r (beta = 0).
  dwf_status arm(int k, double tol_now, bool first, bool reset_p, double rr_conv) {
    UseSlot use(c, sl, k);
    CGScalars &h = *c->h_sc;
    if (first) {
      h.rr_old = rr_conv;
      h.qq = 1.0;
      h.iter = 0;
      h.iter_cap = prm.max_iter;
      h.error = 0;
      h.beta = 0.0;
    } else {
      h.beta = reset_p ? 0.0 : rr_conv / h.rr_old;
    }
    h.delta2 = delta * delta;
    h.beta_f = (float)h.beta;
    h.alpha = 0.0;  // no inner step pending: x = 0 (the restart added the last one)
    h.alpha_f = 0.0f;
    h.rr = rr_conv;
    h.rmax2 = rr_conv;
    h.rr_start = rr_conv;
    h.rr_min = rr_conv;
    h.iter_min = h.iter;
    h.stall_iters = stall_iters;
    h.target2 = tol_now * tol_now * R[k].bnorm2;
    h.restart_flag = R[k].done ? RS_DONE : 0;
    return push_scalars(c, st);
  }

  dwf_status begin() {
    delta = prm.delta > 0.0 ? prm.delta : default_delta(prm.inner_prec);
    full = prm.system == DWF_SYS_FULL;
    stall_iters = prm.stall_iters > 0 ? prm.stall_iters : 500;
    const char *trace_env = getenv("DWF_TRACE");
    trace = trace_env && trace_env[0] == '1';
    for (int k = 0; k < K; ++k) memset(&S_out[k], 0, sizeof(dwf_solve_stats));
    begin_profile(c, prm.profile != 0);
    launches0 = c->launches;
    TRY(ensure_gauge(c, P_F64, st));
    TRY(ensure_gauge(c, prm.inner_prec, st));
    ev0 = next_event(c);
    ev1 = next_event(c);
    CK(cudaEventRecord(ev0, st));

    S.prec = prm.inner_prec;
    S.sp = prm.schur_parity;
    S.op = 1 - S.sp;
    S.K = K;
    TRY(get_buf_k(c, "b", P_F64, K, &S.b));
    TRY(get_buf_k(c, "xh", P_F64, K, &S.xh));
    TRY(get_buf_k(c, "rh", P_F64, K, &S.rh));
    TRY(get_buf(c, "w64", P_F64, &S.w64));
    TRY(get_buf(c, "t64", P_F64, &S.t64));
    TRY(get_buf(c, "q64", P_F64, &S.q64));
    TRY(get_buf(c, "u64", P_F64, &S.u64));
    TRY(inner_bufs());
    prev_tuned = c->use_tuned;
    tuned_saved = true;
    c->use_tuned = !prm.no_autotune;
    if (!prm.no_autotune) TRY(tune_inner(c, st, S));
    if (full)
      for (int p = 0; p < 2; ++p) {
        TRY(get_buf(c, "eta" + std::to_string(p), P_F64, &eta[p]));
        TRY(get_buf(c, "etap" + std::to_string(p), P_F64, &etap[p]));
        TRY(get_buf(c, "phi" + std::to_string(p), P_F64, &phi[p]));
        TRY(get_buf(c, "psi" + std::to_string(p), P_F64, &psi[p]));
        TRY(get_buf(c, "dpsi" + std::to_string(p), P_F64, &dpsi[p]));
      }
    TRY(batch_slots(c, K, &sl));
    g = geom(c);
    full_doubles = (size_t)c->V4 * c->Ns * 24;
    nbytes64 = field_bytes(c, P_F64);
    // the full-system residual runs a little above the Schur one (by at most cond(S1)): the
    // Schur system of a full solve aims at schur_target_pct of the tolerance (default 50 %),
    // and the systems that still miss it take one tightened pass below
    tol_schur = full ? 0.01 * (prm.schur_target_pct > 0 ? prm.schur_target_pct : 50) * prm.tol : prm.tol;
    R.assign(K, RhsState());

    // ---- source: b_k on the Schur parity (Eq. 10 for the full system); x_hat = 0, r_hat = b,
    // r = b in the inner precision, x = p = 0
    CK(cudaMemsetAsync(S.x.v, 0, (size_t)K * field_bytes(c, xprec(S.prec)), st));
    CK(cudaMemsetAsync(S.p.v, 0, (size_t)K * field_bytes(c, S.prec), st));
    if (S.p.nrm) CK(cudaMemsetAsync(S.p.nrm, 0, (size_t)K * c->h * c->Ns * sizeof(float), st));
    CK(cudaMemsetAsync(S.xh.v, 0, (size_t)K * nbytes64, st));
    for (int k = 0; k < K; ++k) {
      UseSlot use(c, sl, k);
      const Field bk = at(c, S.b, k, P_F64);
      if (full) {
        TRY(prep_eta(k));
        // b = eta'_sp - M5 D^{sp,op} eta'_op = eta'_sp + 1/2 M5 H eta'_op
        HopArgs a = hop_args(c, P_F64, S.sp);
        a.in = etap[S.op];
        a.y = etap[S.sp];
        a.out = bk;
        set_m5(a, c, P_F64, false);
        a.coef = 0.5;
        TRY(hop(c, st, P_F64, E_M_XPAY, a, DWF_KC_F64));
      } else {
        Timed t(c, st, DWF_KC_F64);
        CK(pack_any(P_F64, d_rhs + (size_t)k * full_doubles, bk, g, S.sp, c->sm_count, st));
      }
      TRY(norm2(c, st, P_F64, bk, FIN_RED));
      CK(cudaMemcpyAsync(at(c, S.rh, k, P_F64).v, bk.v, nbytes64, cudaMemcpyDeviceToDevice, st));
      TRY(convert(c, st, P_F64, bk, S.prec, at(c, S.r, k, S.prec), DWF_KC_OTHER));
      TRY(norm2(c, st, S.prec, at(c, S.r, k, S.prec), FIN_RED2));
      TRY(pull_scalars(c, st));
      R[k].bnorm2 = R[k].rhat2 = R[k].prev_rhat2 = c->h_sc->red;
      R[k].rr_last = c->h_sc->red2;
      R[k].mode = prm.mode == DWF_MODE_DEFECT ? DWF_MODE_DEFECT : DWF_MODE_RELIABLE;
      R[k].done = R[k].converged = R[k].bnorm2 == 0.0;
    }
    for (int k = 0; k < K; ++k) {
      R[k].tol = tol_schur;
      TRY(arm(k, tol_schur, true, true, R[k].rr_last));
    }
    use_graph = prm.use_graph && !c->profiling;
    first_batch = true;
    return DWF_OK;
  }

  bool all_done() const {
    for (auto &x : R)
      if (!x.done) return false;
    return true;
  }

  // one interval of inner iterations, enqueued on s (the device skips a right-hand side
  // once its restart is due or it is finished)
  dwf_status record_interval(cudaStream_t s) {
    for (int it = 0; it < prm.check_every; ++it) TRY(cg_iteration(c, s, S, sl));
    return DWF_OK;
  }

  // the same on st, replayed from this run's own graph after the first interval
  dwf_status enqueue_interval() {
    if (use_graph && !first_batch) {
      if (!gexec) {
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c->launches;
        dwf_status s2 = record_interval(st);
        if (s2 != DWF_OK) {
          cudaStreamEndCapture(st, &graph);
          return s2;
        }
        c->launches = l0;
        CK(cudaStreamEndCapture(st, &graph));
        CK(cudaGraphInstantiate(&gexec, graph, 0));
      }
      CK(cudaGraphLaunch(gexec, st));
      c->launches += 5LL * prm.check_every;
    } else {
      TRY(record_interval(st));
    }
    first_batch = false;
    return DWF_OK;
  }

  // the batch scalars to the host, after the work enqueued on s
  dwf_status fetch_scalars(cudaStream_t s) {
    CK(cudaMemcpyAsync(sl.h_sc, sl.d_sc, K * sizeof(CGScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DWF_OK;
  }

  // ---- after an interval: the FP64 restarts that fell due (reliable update / defect
  // correction), convergence to |b_k - A x_hat_k| <= R[k].tol |b_k| (FP64)
  dwf_status process_interval() {
    for (int k = 0; k < K; ++k) {
      if (R[k].done) continue;
      UseSlot use(c, sl, k);
      if (c->h_sc->error) TRY(pull_scalars(c, st));  // reports DWF_ETIMEOUT and resets
      const int reason = c->h_sc->restart_flag;
      if (!reason) continue;
      R[k].iters = c->h_sc->iter;
      TRY(fp64_restart(c, st, S, k));
      TRY(pull_scalars(c, st));
      ++R[k].restarts;
      R[k].rhat2 = c->h_sc->red;
      R[k].rr_last = c->h_sc->red2;
      if (trace)
        fprintf(stderr, "dwf: rhs %d restart %d iter %d reason %d |r_iter|/|b| %.3e |r_true|/|b| %.3e mode %s\n", k,
                R[k].restarts, R[k].iters, reason, sqrt(c->h_sc->rr / R[k].bnorm2), sqrt(R[k].rhat2 / R[k].bnorm2),
                R[k].mode == DWF_MODE_DEFECT ? "defect" : "reliable");
      const double tol_now = R[k].tol;
      if (!std::isfinite(R[k].rhat2)) {
        R[k].done = true;
        R[k].status = fail(c, DWF_ENOCONV, "residual is not finite");
      } else if (R[k].rhat2 <= tol_now * tol_now * R[k].bnorm2) {
        R[k].done = R[k].converged = true;
      } else if (R[k].iters >= prm.max_iter) {
        R[k].done = true;
        R[k].status = fail(c, DWF_ENOCONV, "max_iter reached");
      }
      if (R[k].done) {
        TRY(arm(k, tol_now, false, true, R[k].rr_last));  // parks the right-hand side
        continue;
      }
      // Sec. 2.3: fall back to defect correction when the reliable updates stop converging
      // (the true residual grew, or the inner recursion diverged or stalled).  A 16-bit
      // inner CG (a single solve) instead continues in FP32 with reliable updates at its
      // first such cycle: measured at 16^3x32x16, every 16-bit solve whose cycle failed
      // once failed again under 16-bit defect correction before reaching FP32 anyway
      const bool failed = R[k].rhat2 > R[k].prev_rhat2 || reason == RS_DIVERGED || reason == RS_STALLED;
      const bool to_f32 = prm.mode == DWF_MODE_AUTO && failed && S.prec >= P_F16 && K == 1;
      if (prm.mode == DWF_MODE_AUTO && R[k].mode == DWF_MODE_RELIABLE && failed && !to_f32) {
        R[k].mode = DWF_MODE_DEFECT;
      } else if (to_f32) {
        // 16-bit storage is too coarse for this system: continue from x_hat with FP32
        // inner iterations and reliable updates (the FP64 state x_hat, r_hat is untouched)
        R[k].mode = DWF_MODE_RELIABLE;
        TRY(ensure_gauge(c, P_F32, st));
        S.prec = P_F32;
        if (!(prm.delta > 0.0)) delta = default_delta(P_F32);
        TRY(inner_bufs());
        CK(cudaMemsetAsync(S.x.v, 0, field_bytes(c, xprec(S.prec)), st));
        CK(cudaMemsetAsync(S.p.v, 0, field_bytes(c, S.prec), st));
        TRY(convert(c, st, P_F64, S.rh, S.prec, S.r, DWF_KC_F64));
        TRY(norm2(c, st, S.prec, S.r, FIN_RED2));
        TRY(pull_scalars(c, st));
        R[k].rr_last = c->h_sc->red2;
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        first_batch = true;
        graph_dirty = true;
        ++escalations;
      }
      R[k].prev_rhat2 = R[k].rhat2;
      TRY(arm(k, tol_now, false, R[k].mode == DWF_MODE_DEFECT || failed, R[k].rr_last));
    }
    return DWF_OK;
  }

  // ---- solution k: phi_sp = C^dag x_hat; phi_op = eta'_op - M5 D^{op,sp} phi_sp; psi = S2 phi,
  // unpacked to sol_k; then |eta - D psi| / |eta| in FP64
  dwf_status reconstruct(int k) {
    UseSlot use(c, sl, k);
    TRY(prep_eta(k));
    TRY(op_cdag(c, st, P_F64, S.sp, at(c, S.xh, k, P_F64), phi[S.sp], S.w64, S.t64, DWF_KC_F64));
    HopArgs a = hop_args(c, P_F64, S.op);
    a.in = phi[S.sp];
    a.y = etap[S.op];
    a.out = phi[S.op];
    set_m5(a, c, P_F64, false);
    a.coef = 0.5;
    TRY(hop(c, st, P_F64, E_M_XPAY, a, DWF_KC_F64));
    for (int p = 0; p < 2; ++p) {
      TRY(smix(c, st, P_F64, S_PLAIN, phi[p], psi[p], MK_S2, 1.0, DWF_KC_F64));
      Timed t(c, st, DWF_KC_F64);
      CK(unpack_any(P_F64, psi[p], d_sol + (size_t)k * full_doubles, g, p, c->sm_count, st));
    }
    TRY(op_full(c, st, P_F64, psi, dpsi, MK_W, MK_Z, DWF_KC_F64));
    double num = 0, den = 0;
    for (int p = 0; p < 2; ++p) {
      VecArgs v;
      memset(&v, 0, sizeof(v));
      v.a = eta[p];
      v.b = dpsi[p];
      v.n = c->h * c->Ns;
      v.Ns = c->Ns;
      v.fin = FIN_RED;
      v.sc = c->d_sc;
      v.partials = c->d_part;
      v.ticket = c->d_ticket;
      {
        Timed t(c, st, DWF_KC_F64);
        CK(diff_norm2_launch(v, c->sm_count, st));
      }
      TRY(norm2(c, st, P_F64, eta[p], FIN_RED2));
      TRY(pull_scalars(c, st));
      num += c->h_sc->red;
      den += c->h_sc->red2;
    }
    R[k].res_full = den > 0 ? sqrt(num / den) : 0.0;
    return DWF_OK;
  }

  // after the inner loop has finished every system: the solutions (full system: each
  // reconstructed and its full residual taken; a system whose full residual still misses
  // the target continues from x_hat with its Schur tolerance tightened once, each row of a
  // batch as it would alone, the others parked).  *more: the tightened pass is armed and the
  // loop has to run again before the next call.
  dwf_status after_loop(bool *more) {
    *more = false;
    if (full) {
      if (pass == 0) {
        for (int k = 0; k < K; ++k) TRY(reconstruct(k));
        for (int k = 0; k < K; ++k)
          if (R[k].converged && R[k].res_full > prm.tol) again.push_back(k);
        for (int k : again) {
          R[k].tol = tol_schur * std::min(0.1, 0.5 * prm.tol / R[k].res_full);
          R[k].done = R[k].converged = false;
          TRY(arm(k, R[k].tol, false, R[k].mode == DWF_MODE_DEFECT, R[k].rr_last));
        }
        *more = !again.empty();
      } else {
        for (int k : again) TRY(reconstruct(k));
      }
    } else {
      CK(cudaMemsetAsync(d_sol, 0, (size_t)K * full_doubles * sizeof(double), st));
      for (int k = 0; k < K; ++k) {
        Timed t(c, st, DWF_KC_F64);
        CK(unpack_any(P_F64, at(c, S.xh, k, P_F64), d_sol + (size_t)k * full_doubles, g, S.sp, c->sm_count, st));
      }
    }
    ++pass;
    return DWF_OK;
  }

  dwf_status finish() {
    CK(cudaEventRecord(ev1, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(sl.h_sc, sl.d_sc, K * sizeof(CGScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    const double n = (double)c->h * c->Ns;
    end_profile(c, &S_out[0]);
    dwf_status result = DWF_OK;
    for (int k = 0; k < K; ++k) {
      dwf_solve_stats &o = S_out[k];
      if (k > 0) {
        memcpy(o.class_ms, S_out[0].class_ms, sizeof(o.class_ms));
        memcpy(o.class_launches, S_out[0].class_launches, sizeof(o.class_launches));
      }
      o.iters = sl.h_sc[k].iter;
      o.restarts = R[k].restarts;
      o.mode_used = R[k].mode;
      o.converged = R[k].converged ? 1 : 0;
      o.true_res = R[k].bnorm2 > 0 ? sqrt(R[k].rhat2 / R[k].bnorm2) : 0.0;
      o.true_res_full = full ? R[k].res_full : 0.0;
      o.flops = n * (o.iters * flops_cg_iter(c->Ns) + o.restarts * flops_restart(c->Ns) +
                     (full ? flops_prep_recon(c->Ns) : 0.0));
      o.time_ms = ms;
      // algorithmic bytes: 18 (16-bit: 12) reals per link, whatever padding the layout adds
      const double lb = S.prec == P_F64 ? 144.0 : S.prec == P_F32 ? 72.0 : 24.0;
      o.bytes_hop_m5 = n * (2.0 * site_bytes(S.prec) + 8.0 * lb / c->Ns);
      o.inner_prec_used = S.prec;
      o.escalations = escalations;
      o.kernel_launches = c->launches - launches0;
      if (R[k].status != DWF_OK && result == DWF_OK) result = R[k].status;
      if (!R[k].converged && result == DWF_OK) result = fail(c, DWF_ENOCONV, "not converged");
    }
    return result;
  }
};

// the inner loop of one run until every system is finished
dwf_status run_loop(SolveRun &r) {
  while (!r.all_done()) {
    TRY(r.enqueue_interval());
    TRY(r.fetch_scalars(r.st));
    TRY(r.process_interval());
  }
  return DWF_OK;
}

// Solve K systems with the same operator; rhs/sol hold K full-lattice arrays one after another.
dwf_status solve_core(dwf_ctx *c, int K, const double *d_rhs, double *d_sol, dwf_solve_params prm,
                      dwf_solve_stats *S_out, cudaStream_t st) {
  SolveRun r(c, K, d_rhs, d_sol, prm, S_out, st);
  TRY(r.begin());
  for (;;) {
    dwf_status loop_st = run_loop(r);
    if (loop_st != DWF_OK && loop_st != DWF_ENOCONV) return loop_st;
    bool more = false;
    TRY(r.after_loop(&more));
    if (!more) break;
  }
  return r.finish();
}

dwf_status check_solve_args(dwf_ctx *c, dwf_solve_params *prm, const dwf_solve_params *pp, const void *d_rhs,
                            const void *d_sol) {
  TRY(not_part(c));
  if (pp) *prm = *pp;
  else dwf_solve_params_default(prm);
  if (!d_rhs || !d_sol || !aligned16(d_rhs) || !aligned16(d_sol))
    return fail(c, DWF_EINVAL, "null or non-16-byte-aligned field pointer");
  if (!valid_prec(prm->inner_prec)) return fail(c, DWF_EINVAL, "unknown inner precision");
  if (prm->system != DWF_SYS_FULL && prm->system != DWF_SYS_NORMAL) return fail(c, DWF_EINVAL, "unknown system");
  if (prm->schur_parity != 0 && prm->schur_parity != 1) return fail(c, DWF_EINVAL, "schur_parity must be 0 or 1");
  if (prm->mode < DWF_MODE_AUTO || prm->mode > DWF_MODE_DEFECT) return fail(c, DWF_EINVAL, "unknown mode");
  if (!(prm->tol > 0.0) || prm->max_iter < 1) return fail(c, DWF_EINVAL, "tol must be > 0 and max_iter >= 1");
  if (prm->check_every < 1) prm->check_every = 8;
  if (prm->schur_target_pct > 100000) return fail(c, DWF_EINVAL, "schur_target_pct above 100000");
  return DWF_OK;
}

// y = a + sb b on host-layout device arrays (sites of parity keep, all if keep < 0; the
// rest set to 0) and |y|^2 into the scalar `fin`
dwf_status host_axpy(dwf_ctx *c, cudaStream_t st, double *y, const double *a, const double *b, double sb, int keep,
                     int fin) {
  HostAxpyArgs v;
  memset(&v, 0, sizeof(v));
  v.y = y;
  v.a = a;
  v.b = b;
  v.sb = sb;
  v.g = geom(c);
  v.keep = keep;
  v.fin = fin;
  v.sc = c->d_sc;
  v.partials = c->d_part;
  v.ticket = c->d_ticket;
  Timed t(c, st, DWF_KC_F64);
  CK(host_axpy_launch(v, c->sm_count, st));
  return DWF_OK;
}

// Warm start (Algorithm 2 from a given x_hat): for each right-hand side the caller's sol
// holds x0.  The FP64 residual r = rhs - A x0 of the requested system (A = D for the full
// system, C C^dag on the Schur parity for the normal one) is solved for the correction,
// A dx = r, to tol |rhs| / |r|, and sol = x0 + dx.  The residuals in the stats are then
// relative to |rhs|.
dwf_status warm_solve(dwf_ctx *c, int K, const double *d_rhs, double *d_sol, dwf_solve_params prm,
                      dwf_solve_stats *S_out, cudaStream_t st) {
  const bool full = prm.system == DWF_SYS_FULL;
  const int keep = full ? -1 : prm.schur_parity;
  const size_t nd = (size_t)c->V4 * c->Ns * 24;
  void *pr, *pt, *pd;
  TRY(get_raw(c, "warm_r", nd * sizeof(double), &pr));
  TRY(get_raw(c, "warm_t", nd * sizeof(double), &pt));
  TRY(get_raw(c, "warm_d", nd * sizeof(double), &pd));
  double *r = static_cast<double *>(pr), *t = static_cast<double *>(pt), *dx = static_cast<double *>(pd);
  dwf_solve_params inner = prm;
  inner.use_x0 = 0;
  dwf_status result = DWF_OK;
  for (int k = 0; k < K; ++k) {
    const double *rhs = d_rhs + (size_t)k * nd;
    double *x = d_sol + (size_t)k * nd;
    dwf_solve_stats &o = S_out[k];
    memset(&o, 0, sizeof(o));
    TRY(host_axpy(c, st, x, x, nullptr, 0.0, keep, FIN_NONE));  // x0 on the system's sites
    TRY(dwf_apply_eo_dev(c, full ? DWF_OP_DFULL : DWF_OP_CCDAG, DWF_PREC_F64, prm.schur_parity, x, t, st));
    TRY(host_axpy(c, st, r, rhs, nullptr, 0.0, keep, FIN_RED2));  // |rhs|^2
    TRY(host_axpy(c, st, r, r, t, -1.0, keep, FIN_RED));          // r = rhs - A x0, |r|^2
    TRY(pull_scalars(c, st));
    const double bb = c->h_sc->red2, rr = c->h_sc->red;
    if (!std::isfinite(bb) || !std::isfinite(rr)) return fail(c, DWF_EINVAL, "source or initial guess is not finite");
    o.inner_prec_used = prm.inner_prec;
    o.mode_used = prm.mode == DWF_MODE_DEFECT ? DWF_MODE_DEFECT : DWF_MODE_RELIABLE;
    if (bb == 0.0) {  // zero source: the solution is 0 (no site has parity 2)
      TRY(host_axpy(c, st, x, x, nullptr, 0.0, 2, FIN_NONE));
      o.converged = 1;
      continue;
    }
    if (rr <= prm.tol * prm.tol * bb) {  // x0 already meets the tolerance
      o.converged = 1;
      o.true_res = sqrt(rr / bb);
      o.true_res_full = full ? o.true_res : 0.0;
      continue;
    }
    inner.tol = prm.tol * sqrt(bb / rr);
    dwf_status s = solve_core(c, 1, r, dx, inner, &o, st);
    if (s != DWF_OK && s != DWF_ENOCONV) return s;
    if (s != DWF_OK && result == DWF_OK) result = s;
    TRY(host_axpy(c, st, x, x, dx, 1.0, keep, FIN_NONE));
    const double f = sqrt(rr / bb);
    o.true_res *= f;
    o.true_res_full *= f;
  }
  CK(cudaStreamSynchronize(st));
  if (result != DWF_OK) return fail(c, result, "not converged");
  return DWF_OK;
}

}  // namespace

extern "C" dwf_status dwf_solve_batch_dev(dwf_ctx *c, int nrhs, const double *d_rhs, double *d_sol,
                                          const dwf_solve_params *pp, dwf_solve_stats *stats, void *stream) {
  TRY(check_ctx(c));
  if (nrhs < 1 || nrhs > 65535) return fail(c, DWF_EINVAL, "nrhs must be in 1..65535");
  dwf_solve_params prm;
  TRY(check_solve_args(c, &prm, pp, d_rhs, d_sol));
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double);
  const char *a = (const char *)d_rhs, *b = (const char *)d_sol;
  if (a < b + nrhs * full && b < a + nrhs * full) return fail(c, DWF_EINVAL, "rhs and sol overlap");
  std::vector<dwf_solve_stats> local;
  if (!stats) {
    local.resize(nrhs);
    stats = local.data();
  }
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  if (prm.use_x0) return warm_solve(c, nrhs, d_rhs, d_sol, prm, stats, st);
  return solve_core(c, nrhs, d_rhs, d_sol, prm, stats, st);
}

extern "C" dwf_status dwf_tuned_shape(dwf_ctx *c, int prec, int kclass, int *threads, int *persistent) {
  TRY(check_ctx(c));
  if (!threads || !persistent) return fail(c, DWF_EINVAL, "null output");
  if (prec != P_F32 && prec != P_F16 && prec != P_BF16) return fail(c, DWF_EINVAL, "inner precisions only");
  int epi;
  switch (kclass) {
    case DWF_KC_HOP_M5: epi = E_M; break;
    case DWF_KC_HOP_XPAY: epi = E_XPAY_G5; break;
    case DWF_KC_HOP_UPDATE: epi = E_CG_UPDATE; break;
    default: return fail(c, DWF_EINVAL, "kernel class must be hop_m5, hop_xpay or hop_update");
  }
  HopShape s;
  const bool tuned = g_tune.get(tune_key(c, prec, epi), &s);
  if (!tuned) s.persistent = epi == E_XPAY_G5;  // the default shapes
  *threads = s.threads;
  *persistent = s.persistent ? 1 : 0;
  return tuned ? DWF_OK : DWF_EAGAIN;
}

extern "C" dwf_status dwf_solve_dev(dwf_ctx *c, const double *d_rhs, double *d_sol, const dwf_solve_params *pp,
                                    dwf_solve_stats *stats, void *stream) {
  return dwf_solve_batch_dev(c, 1, d_rhs, d_sol, pp, stats, stream);
}

extern "C" dwf_status dwf_solve_batch(dwf_ctx *c, int nrhs, const double *rhs, double *sol,
                                      const dwf_solve_params *pp, dwf_solve_stats *stats) {
  TRY(check_ctx(c));
  if (!rhs || !sol) return fail(c, DWF_EINVAL, "null field pointer");
  if (nrhs < 1 || nrhs > 65535) return fail(c, DWF_EINVAL, "nrhs must be in 1..65535");
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double) * nrhs;
  void *din, *dout;
  TRY(get_raw(c, "host_in", full, &din));
  TRY(get_raw(c, "host_out", full, &dout));
  CK(cudaMemcpyAsync(din, rhs, full, cudaMemcpyHostToDevice, c->stream));
  if (pp && pp->use_x0) CK(cudaMemcpyAsync(dout, sol, full, cudaMemcpyHostToDevice, c->stream));
  dwf_status s = dwf_solve_batch_dev(c, nrhs, (const double *)din, (double *)dout, pp, stats, c->stream);
  if (s != DWF_OK && s != DWF_ENOCONV) return s;
  CK(cudaMemcpyAsync(sol, dout, full, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return s;
}

extern "C" dwf_status dwf_solve(dwf_ctx *c, const double *rhs, double *sol, const dwf_solve_params *pp,
                                dwf_solve_stats *stats) {
  return dwf_solve_batch(c, 1, rhs, sol, pp, stats);
}

// ====================================================================== ragged sets

// A ragged set: one right-hand side on each of n contexts (their own lattice, Ns, masses and
// weights; typically one gauge field shared by handle), solved together.  Every interval of
// check_every inner iterations of all unfinished systems is one CUDA graph, a branch per
// context fork-joined on the caller's stream (the branches run concurrently); restarts,
// reconstruction and stats stay per context, on the context's own stream, between the
// graph launches.  Each system takes the same kernels in the same order as it would alone,
// so its result is the same bit for bit.
extern "C" dwf_status dwf_solve_ragged_dev(int n, dwf_ctx *const *ctxs, const double *const *d_rhs,
                                           double *const *d_sol, const dwf_solve_params *pp,
                                           dwf_solve_stats *stats, void *stream) {
  if (n < 1 || n > 256 || !ctxs) return DWF_EINVAL;
  for (int k = 0; k < n; ++k) TRY(check_ctx(ctxs[k]));
  dwf_ctx *c = ctxs[0];  // errors of the set as a whole are reported on the first context
  if (!d_rhs || !d_sol) return fail(c, DWF_EINVAL, "null rhs or sol array");
  std::vector<dwf_solve_params> prm(n);
  for (int k = 0; k < n; ++k) {
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(c, DWF_EINVAL, "a context appears twice in a ragged set");
    if (ctxs[k]->device != c->device) return fail(c, DWF_EINVAL, "the contexts of a ragged set must share a device");
    TRY(check_solve_args(ctxs[k], &prm[k], pp, d_rhs[k], d_sol[k]));
    if (prm[k].use_x0) return fail(ctxs[k], DWF_EINVAL, "a ragged set takes no initial guess");
    const size_t full = (size_t)ctxs[k]->V4 * ctxs[k]->Ns * 24 * sizeof(double);
    const char *a = (const char *)d_rhs[k], *b = (const char *)d_sol[k];
    if (a < b + full && b < a + full) return fail(ctxs[k], DWF_EINVAL, "rhs and sol overlap");
  }
  std::vector<dwf_solve_stats> local;
  if (!stats) {
    local.resize(n);
    stats = local.data();
  }
  const cudaStream_t st0 = stream ? (cudaStream_t)stream : c->stream;
  struct Owned {  // events and the combined graph of this call
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~Owned() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
    void drop_graph() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
    }
  } own;
  own.ev.assign(n + 1, nullptr);
  for (auto &e : own.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // every context's stream starts after the caller's stream (its sources)
  CK(cudaEventRecord(own.ev[0], st0));
  for (int k = 0; k < n; ++k) CK(cudaStreamWaitEvent(ctxs[k]->stream, own.ev[0], 0));

  std::vector<std::unique_ptr<SolveRun>> runs;
  for (int k = 0; k < n; ++k) {
    runs.emplace_back(new SolveRun(ctxs[k], 1, d_rhs[k], d_sol[k], prm[k], &stats[k], ctxs[k]->stream));
    TRY(runs[k]->begin());
  }
  std::vector<char> pending(n, 1);  // the run has an inner loop (or a tightened pass) to finish
  std::vector<int> gset;            // the runs the combined graph was captured for
  for (;;) {
    std::vector<int> act;
    for (int k = 0; k < n; ++k)
      if (pending[k] && !runs[k]->all_done()) act.push_back(k);
    if (act.empty()) {
      bool any = false;
      for (int k = 0; k < n; ++k)
        if (pending[k]) {
          bool more = false;
          TRY(runs[k]->after_loop(&more));
          pending[k] = more;
          any = any || more;
        }
      if (!any) break;
      continue;
    }
    bool eager = false;  // the first interval of a run (or of its new precision) runs outside a graph
    for (int k : act) eager = eager || runs[k]->first_batch || !runs[k]->use_graph;
    if (eager) {
      for (int k : act) {
        TRY(runs[k]->record_interval(runs[k]->st));
        runs[k]->first_batch = false;
      }
      for (int k : act) TRY(runs[k]->fetch_scalars(runs[k]->st));
    } else {
      bool dirty = !own.exec || act != gset;
      for (int k : act) dirty = dirty || runs[k]->graph_dirty;
      if (dirty) {
        own.drop_graph();
        CK(cudaStreamBeginCapture(st0, cudaStreamCaptureModeThreadLocal));
        dwf_status cs = DWF_OK;
        cudaError_t ce = cudaEventRecord(own.ev[0], st0);
        for (size_t i = 0; i < act.size() && cs == DWF_OK && ce == cudaSuccess; ++i) {
          SolveRun &r = *runs[act[i]];
          ce = cudaStreamWaitEvent(r.st, own.ev[0], 0);
          const long long l0 = r.c->launches;
          if (ce == cudaSuccess) cs = r.record_interval(r.st);
          r.c->launches = l0;
          if (cs == DWF_OK && ce == cudaSuccess) ce = cudaEventRecord(own.ev[1 + act[i]], r.st);
          if (cs == DWF_OK && ce == cudaSuccess) ce = cudaStreamWaitEvent(st0, own.ev[1 + act[i]], 0);
        }
        const cudaError_t ee = cudaStreamEndCapture(st0, &own.graph);
        if (cs != DWF_OK) return cs;
        CK(ce);
        CK(ee);
        CK(cudaGraphInstantiate(&own.exec, own.graph, 0));
        gset = act;
        for (int k : act) runs[k]->graph_dirty = false;
      }
      // the graph starts after each run's last restart and scalar upload on its own stream
      for (int k : act) {
        CK(cudaEventRecord(own.ev[1 + k], runs[k]->st));
        CK(cudaStreamWaitEvent(st0, own.ev[1 + k], 0));
      }
      CK(cudaGraphLaunch(own.exec, st0));
      for (int k : act) runs[k]->c->launches += 5LL * runs[k]->prm.check_every;
      for (int k : act) TRY(runs[k]->fetch_scalars(st0));
    }
    for (int k : act) TRY(runs[k]->process_interval());
  }
  dwf_status result = DWF_OK;
  for (int k = 0; k < n; ++k) {
    const dwf_status s = runs[k]->finish();
    if (s != DWF_OK && s != DWF_ENOCONV) return s;
    if (s != DWF_OK && result == DWF_OK) result = s;
  }
  // the caller's stream continues after every solution is written
  for (int k = 0; k < n; ++k) {
    CK(cudaEventRecord(own.ev[1 + k], ctxs[k]->stream));
    CK(cudaStreamWaitEvent(st0, own.ev[1 + k], 0));
  }
  return result;
}

extern "C" dwf_status dwf_solve_ragged(int n, dwf_ctx *const *ctxs, const double *const *rhs, double *const *sol,
                                       const dwf_solve_params *pp, dwf_solve_stats *stats) {
  if (n < 1 || n > 256 || !ctxs) return DWF_EINVAL;
  for (int k = 0; k < n; ++k) TRY(check_ctx(ctxs[k]));
  dwf_ctx *c = ctxs[0];
  if (!rhs || !sol) return fail(c, DWF_EINVAL, "null rhs or sol array");
  std::vector<const double *> din(n);
  std::vector<double *> dout(n);
  for (int k = 0; k < n; ++k) {
    if (!rhs[k] || !sol[k]) return fail(ctxs[k], DWF_EINVAL, "null field pointer");
    const size_t full = (size_t)ctxs[k]->V4 * ctxs[k]->Ns * 24 * sizeof(double);
    void *a, *b;
    TRY(get_raw(ctxs[k], "host_in", full, &a));
    TRY(get_raw(ctxs[k], "host_out", full, &b));
    CK(cudaMemcpyAsync(a, rhs[k], full, cudaMemcpyHostToDevice, ctxs[k]->stream));
    CK(cudaStreamSynchronize(ctxs[k]->stream));
    din[k] = (const double *)a;
    dout[k] = (double *)b;
  }
  const dwf_status s = dwf_solve_ragged_dev(n, ctxs, din.data(), dout.data(), pp, stats, c->stream);
  if (s != DWF_OK && s != DWF_ENOCONV) return s;
  for (int k = 0; k < n; ++k) {
    const size_t full = (size_t)ctxs[k]->V4 * ctxs[k]->Ns * 24 * sizeof(double);
    CK(cudaMemcpyAsync(sol[k], dout[k], full, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return s;
}

// ====================================================================== propagators

extern "C" dwf_status dwf_propagator_dev(dwf_ctx *c, const int x0[4], const dwf_solve_params *pp, double *d_prop,
                                         dwf_solve_stats *stats, void *stream) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!x0 || !d_prop || !aligned16(d_prop)) return fail(c, DWF_EINVAL, "null x0 or non-16-byte-aligned output");
  for (int mu = 0; mu < 4; ++mu)
    if (x0[mu] < 0 || x0[mu] >= c->dims[mu]) return fail(c, DWF_EINVAL, "source point outside the lattice");
  dwf_solve_params prm;
  if (pp) prm = *pp;
  else dwf_solve_params_default(&prm);
  prm.system = DWF_SYS_FULL;
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double);
  void *drhs, *dsol;
  TRY(get_raw(c, "prop_rhs", 12 * full, &drhs));
  TRY(get_raw(c, "prop_sol", 12 * full, &dsol));
  CK(cudaMemsetAsync(drhs, 0, 12 * full, st));
  const long x0site = x0[0] + (long)c->dims[0] * (x0[1] + (long)c->dims[1] * (x0[2] + (long)c->dims[2] * x0[3]));
  CK(point_sources_launch(static_cast<double *>(drhs), x0site, c->V4, c->Ns, st));
  c->launches++;
  dwf_status s = dwf_solve_batch_dev(c, 12, static_cast<const double *>(drhs), static_cast<double *>(dsol), &prm,
                                     stats, st);
  if (s != DWF_OK && s != DWF_ENOCONV) return s;
  CK(prop_extract_launch(static_cast<const double *>(dsol), d_prop, c->V4, c->Ns, c->sm_count, st));
  c->launches++;
  CK(cudaStreamSynchronize(st));
  return s;
}

extern "C" dwf_status dwf_propagator(dwf_ctx *c, const int x0[4], const dwf_solve_params *pp, double *prop,
                                     dwf_solve_stats *stats) {
  TRY(check_ctx(c));
  if (!prop) return fail(c, DWF_EINVAL, "null output");
  const size_t bytes = (size_t)c->V4 * 144 * 2 * sizeof(double);
  void *dprop;
  TRY(get_raw(c, "prop_out", bytes, &dprop));
  dwf_status s = dwf_propagator_dev(c, x0, pp, static_cast<double *>(dprop), stats, c->stream);
  if (s != DWF_OK && s != DWF_ENOCONV) return s;
  CK(cudaMemcpyAsync(prop, dprop, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return s;
}

// ====================================================================== allocation-free variant
//
// dwf_apply_eo_dev_static is dwf_apply_eo_dev for the Schur-parity operators with every
// work field (packed input and output, three intermediates), the CG scalar block and the
// reduction scratch (block partial sums and the last-block ticket) taken from one static
// device array, so a call never allocates.  It is for callers that cannot let a library
// allocate device memory: applications whose device memory is owned by their own pool
// allocator (a framework's caching allocator that already holds the GPU's memory) or held
// to a fixed budget decided at start-up, and paths that must not meet the device-wide
// synchronisation a cudaMalloc or cudaFree can bring.  The array is a file-scope
// __device__ variable, so every GPU that loads the library holds it until the process
// exits.  The call touches no mutable state of the context (its device address of the
// array aside), so other work on the same context is not redirected to the array.

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB per device
__device__ __align__(256) unsigned char g_dwf_static_scratch[kStaticScratchBytes];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" dwf_status dwf_apply_eo_dev_static(dwf_ctx *c, int op, int prec, int parity, const double *d_in,
                                              double *d_out, void *stream) {
  TRY(check_ctx(c));
  TRY(not_part(c));
  if (!d_in || !d_out || !aligned16(d_in) || !aligned16(d_out))
    return fail(c, DWF_EINVAL, "null or non-16-byte-aligned field pointer");
  if (!valid_prec(prec)) return fail(c, DWF_EINVAL, "unknown precision");
  if (op < DWF_OP_DEO || op > DWF_OP_CCDAG)
    return fail(c, DWF_EINVAL, "the allocation-free variant applies DEO, DOE, M5, M5T, C, CDAG or CCDAG");
  const bool needs_parity = op >= DWF_OP_M5;
  if (needs_parity && parity != 0 && parity != 1) return fail(c, DWF_EINVAL, "parity must be 0 or 1");
  const size_t full = (size_t)c->V4 * c->Ns * 24 * sizeof(double);
  if ((const char *)d_in < (const char *)d_out + full && (const char *)d_out < (const char *)d_in + full)
    return fail(c, DWF_EINVAL, "in and out overlap");
  if (!c->gauge_loaded) return fail(c, DWF_ENOGAUGE, "dwf_load_gauge has not been called");
  if (!c->gauge_ready[prec])
    return fail(c, DWF_EINVAL,
                "the gauge field of this precision is not built yet (dwf_load_gauge builds FP64 and FP32; "
                "one dwf_apply_eo_dev call in a 16-bit precision builds that form)");

  // carve five fields, the scalar block, the partial sums and the ticket out of the array
  const size_t n = (size_t)c->h * c->Ns;
  const size_t data_b = round256(n * site_bytes(prec));
  const size_t nrm_b = prec >= P_F16 ? round256(n * sizeof(float)) : 0;
  const long spb = std::min(hop_sites_per_block(prec, c->Ns), sites_per_block(prec, c->Ns));
  const size_t max_blocks = std::max<size_t>((size_t)((c->h + spb - 1) / spb), (size_t)c->sm_count * 8);
  const size_t need = 5 * (data_b + nrm_b) + round256(sizeof(CGScalars)) + round256(max_blocks * sizeof(double)) +
                      256;
  if (need > kStaticScratchBytes)
    return fail(c, DWF_EINVAL,
                "lattice too large for the static scratch: needs " + std::to_string(need) + " bytes, the array holds " +
                    std::to_string(kStaticScratchBytes));
  // set-up, once per context (so once per device it runs on, with that device current):
  // in host code the array's name is only a host-side stand-in, so its device address is
  // looked up here; the first call on a context should come before any stream capture
  if (!c->static_scratch) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dwf_static_scratch);
    if (e != cudaSuccess) return fail(c, DWF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    c->static_scratch = p;
  }
  unsigned char *cur = static_cast<unsigned char *>(c->static_scratch);
  Field f[5];
  for (auto &x : f) {
    x.v = cur;
    cur += data_b;
    x.nrm = nrm_b ? reinterpret_cast<float *>(cur) : nullptr;
    cur += nrm_b;
  }
  CGScalars *sc = reinterpret_cast<CGScalars *>(cur);
  cur += round256(sizeof(CGScalars));
  double *part = reinterpret_cast<double *>(cur);
  cur += round256(max_blocks * sizeof(double));
  unsigned *ticket = reinterpret_cast<unsigned *>(cur);

  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  // the array keeps the previous call's contents: the scalars (error word included) and the
  // ticket must start at zero
  CK(cudaMemsetAsync(sc, 0, sizeof(CGScalars), st));
  CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
  CK(cudaMemsetAsync(d_out, 0, full, st));
  const Geom g = geom(c);
  Field &in = f[0], &out = f[1], &tA = f[2], &tB = f[3], &tC = f[4];
  const int inpar = op == DWF_OP_DEO ? 1 : op == DWF_OP_DOE ? 0 : parity;
  const int outpar = op == DWF_OP_DEO ? 0 : op == DWF_OP_DOE ? 1 : parity;
  // the hop launches of this call, with the reduction scratch of the array
  auto hop_s = [&](int outp, int epi, Field x, Field y, Field o, bool m5, bool trans, double coef) -> cudaError_t {
    HopArgs a = hop_args(c, prec, outp);
    a.in = x;
    a.y = y;
    a.out = o;
    if (m5) set_m5(a, c, prec, trans);
    a.coef = coef;
    a.sc = sc;
    a.partials = part;
    a.ticket = ticket;
    return hop_any(prec, epi, a, st);
  };
  auto smix_s = [&](int mode, Field x, Field o, int kind) -> cudaError_t {
    SmixArgs a;
    memset(&a, 0, sizeof(a));
    a.in = x;
    a.out = o;
    a.K = dmat(c, prec, kind);
    a.K2 = dmat(c, prec, MK_ID);
    a.coef = 1.0;
    a.h = c->h;
    a.Ns = c->Ns;
    a.sc = sc;
    return smix_any(prec, mode, a, st);
  };
  // Eq. 11 on Schur parity sp: C v = v - M5 D M5 D v (u = -1/2 M5 H v, out = v + 1/2 M5 H u)
  auto apply_c = [&](int sp, Field v, Field o, Field u) -> cudaError_t {
    cudaError_t e = hop_s(1 - sp, E_M, v, Field{}, u, true, false, -0.5);
    if (e == cudaSuccess) e = hop_s(sp, E_M_XPAY, u, v, o, true, false, 0.5);
    return e;
  };
  // C^dag v = g5 (1 - D M5^T D M5^T) g5 v (w = M5^T g5 v, t = -1/2 M5^T H w, q = v + 1/2 g5 H t)
  auto apply_cdag = [&](int sp, Field v, Field q, Field w, Field t) -> cudaError_t {
    cudaError_t e = smix_s(S_G5, v, w, MK_M5T);
    if (e == cudaSuccess) e = hop_s(1 - sp, E_M, w, Field{}, t, true, true, -0.5);
    if (e == cudaSuccess) e = hop_s(sp, E_XPAY_G5, t, v, q, false, false, 0.5);
    return e;
  };
  CK(pack_any(prec, d_in, in, g, inpar, c->sm_count, st));
  switch (op) {
    case DWF_OP_DEO:
    case DWF_OP_DOE:
      CK(hop_s(outpar, E_PLAIN, in, Field{}, out, false, false, -0.5));
      break;
    case DWF_OP_M5:
    case DWF_OP_M5T:
      CK(smix_s(S_PLAIN, in, out, op == DWF_OP_M5 ? MK_M5 : MK_M5T));
      break;
    case DWF_OP_C:
      CK(apply_c(parity, in, out, tA));
      break;
    case DWF_OP_CDAG:
      CK(apply_cdag(parity, in, out, tA, tB));
      break;
    case DWF_OP_CCDAG:
      CK(apply_cdag(parity, in, tC, tA, tB));
      CK(apply_c(parity, tC, out, tA));
      break;
  }
  CK(unpack_any(prec, out, d_out, g, outpar, c->sm_count, st));
  // the call returns when its work is done: it waits for `stream` and reads the kernels'
  // error word (a bounded device-side wait that gave up) into host memory of its own
  int err = 0;
  CK(cudaMemcpyAsync(&err, &sc->error, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) return fail(c, DWF_ETIMEOUT, "a device-side wait for the TMA link copy timed out");
  return DWF_OK;
}

// ====================================================================== 4D domain decomposition
//
// One context per part of the lattice (dwf_create_part); dwf_part_apply applies an operator
// to a field spread over all parts: before every hop each part packs the spin projections of
// its cut faces (12 reals per (site, s)), the packed faces are copied to the neighbouring
// parts' receive buffers (device to device, or between devices) and unpacked into their
// halo slots, and each part's hop kernel then runs unchanged with the halo-aware neighbour
// table.  The fifth-dimension matrices act within a part.

namespace {

template <int P>
cudaError_t part_gauge_go(dwf_ctx *c, int p, cudaStream_t st) {
  k_part_gauge<P><<<vec_grid(c->h * 8, c->sm_count), 256, 0, st>>>(
      c->d_Ug, static_cast<typename PT<P>::lreal *>(c->d_gauge[P][p]), c->pg, p);
  return cudaGetLastError();
}

dwf_status ensure_part_gauge(dwf_ctx *c, int prec) {
  if (!c->d_Ug) return fail(c, DWF_ENOGAUGE, "dwf_load_gauge_part has not been called");
  if (c->gauge_ready[prec]) return DWF_OK;
  for (int p = 0; p < 2; ++p) {
    if (!c->d_gauge[prec][p])
      CK(dmalloc(&c->d_gauge[prec][p], (size_t)c->h * link_bytes_per_site(prec), c->device, c->stream));
    switch (prec) {
      case P_F64: CK(part_gauge_go<P_F64>(c, p, c->stream)); break;
      case P_F32: CK(part_gauge_go<P_F32>(c, p, c->stream)); break;
      case P_F16: CK(part_gauge_go<P_F16>(c, p, c->stream)); break;
      default: CK(part_gauge_go<P_BF16>(c, p, c->stream)); break;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  c->gauge_ready[prec] = true;
  c->gauge_loaded = true;
  return DWF_OK;
}

// a field of one parity with the halo slots after the local sites
dwf_status part_field(dwf_ctx *c, const std::string &name, int prec, Field *f) {
  const size_t n = (size_t)(c->h + c->pg.halo) * c->Ns;
  void *v = nullptr, *nrm = nullptr;
  TRY(get_raw(c, "part:" + name + "#" + std::to_string(prec), n * site_bytes(prec), &v));
  if (prec >= P_F16) TRY(get_raw(c, "part:" + name + "#nrm" + std::to_string(prec), n * sizeof(float), &nrm));
  f->v = v;
  f->nrm = static_cast<float *>(nrm);
  return DWF_OK;
}

size_t real_bytes(int prec) { return prec == P_F64 ? 8 : 4; }

template <int P>
cudaError_t part_pack_go(dwf_ctx *c, Field in, int mu, int side, int q, void *buf, cudaStream_t st) {
  const long n = c->pg.fsz[mu] * c->Ns;
  k_part_pack<P><<<vec_grid(n, c->sm_count), 256, 0, st>>>(in, c->pg, c->Ns, mu, side, q, side ? 1.0 : -1.0,
                                                          static_cast<typename PT<P>::real *>(buf));
  return cudaGetLastError();
}
template <int P>
cudaError_t part_unpack_go(dwf_ctx *c, const void *buf, Field out, long first, long nslot, cudaStream_t st) {
  k_part_unpack<P><<<vec_grid(nslot * c->Ns, c->sm_count), 256, 0, st>>>(
      static_cast<const typename PT<P>::real *>(buf), out, first, nslot, c->Ns);
  return cudaGetLastError();
}
cudaError_t part_pack_any(int prec, dwf_ctx *c, Field in, int mu, int side, int q, void *buf, cudaStream_t st) {
  switch (prec) {
    case P_F64: return part_pack_go<P_F64>(c, in, mu, side, q, buf, st);
    case P_F32: return part_pack_go<P_F32>(c, in, mu, side, q, buf, st);
    case P_F16: return part_pack_go<P_F16>(c, in, mu, side, q, buf, st);
    default: return part_pack_go<P_BF16>(c, in, mu, side, q, buf, st);
  }
}
cudaError_t part_unpack_any(int prec, dwf_ctx *c, const void *buf, Field out, long first, long nslot,
                            cudaStream_t st) {
  switch (prec) {
    case P_F64: return part_unpack_go<P_F64>(c, buf, out, first, nslot, st);
    case P_F32: return part_unpack_go<P_F32>(c, buf, out, first, nslot, st);
    case P_F16: return part_unpack_go<P_F16>(c, buf, out, first, nslot, st);
    default: return part_unpack_go<P_BF16>(c, buf, out, first, nslot, st);
  }
}

// the parts of one decomposed lattice, indexed by their grid coordinates
// the parts of one decomposed lattice that this call drives: every part, in grid order
// (at[x + gx (y + gy (z + gz t))]), or -- with a caller's transport, comm -- this process's
// one part, the others reached through comm
struct PartSet {
  std::vector<dwf_ctx *> at;
  int grid[4];
  const dwf_part_comm *comm = nullptr;
  dwf_ctx *get(const int (&c)[4]) const {
    int k[4];
    for (int mu = 0; mu < 4; ++mu) k[mu] = (c[mu] % grid[mu] + grid[mu]) % grid[mu];
    return at[k[0] + grid[0] * (k[1] + grid[1] * (k[2] + grid[2] * k[3]))];
  }
};

// part_exchange through the caller's transport: this process's part packs its cut faces
// into pinned host memory (face k = 2 mu + side), comm->exchange swaps them with the
// neighbours, and the received faces are unpacked into the halo slots
dwf_status part_exchange_comm(const PartSet &ps, const std::string &name, int prec, int q) {
  dwf_ctx *c = ps.at[0];
  Field f;
  TRY(part_field(c, name, prec, &f));
  size_t bytes[8] = {}, off[8] = {}, total = 0;
  for (int k = 0; k < 8; ++k) {
    if (c->pg.grid[k >> 1] == 1) continue;
    bytes[k] = (size_t)c->pg.fsz[k >> 1] * c->Ns * 12 * real_bytes(prec);
    off[k] = total;
    total += (bytes[k] + 15) & ~(size_t)15;
  }
  if (total == 0) return DWF_OK;  // no cut direction: a single part
  if (c->h_face_bytes < 2 * total) {
    pinned_put(c->h_face, c->h_face_bytes);
    c->h_face = pinned_get(2 * total);
    c->h_face_bytes = c->h_face ? 2 * total : 0;
    if (!c->h_face) return fail(c, DWF_ENOMEM, "pinned host memory for the faces");
  }
  char *hs = static_cast<char *>(c->h_face), *hr = hs + total;
  const void *send[8] = {};
  void *recv[8] = {};
  for (int k = 0; k < 8; ++k) {
    if (!bytes[k]) continue;
    void *d;
    TRY(get_raw(c, "part_send" + std::to_string(k), bytes[k], &d));
    CK(part_pack_any(prec, c, f, k >> 1, k & 1, q, d, c->stream));
    CK(cudaMemcpyAsync(hs + off[k], d, bytes[k], cudaMemcpyDeviceToHost, c->stream));
    send[k] = hs + off[k];
    recv[k] = hr + off[k];
  }
  CK(cudaStreamSynchronize(c->stream));
  if (ps.comm->exchange(ps.comm->user, send, recv, bytes) != 0)
    return fail(c, DWF_ECOMM, "the exchange callback failed");
  for (int k = 0; k < 8; ++k) {
    if (!bytes[k]) continue;
    // the halo slab on side k & 1 takes that neighbour's face k ^ 1
    void *d;
    TRY(get_raw(c, "part_recv" + std::to_string(k), bytes[k], &d));
    CK(cudaMemcpyAsync(d, hr + off[k], bytes[k], cudaMemcpyHostToDevice, c->stream));
    CK(part_unpack_any(prec, c, d, f, c->h + c->pg.foff[k >> 1][k & 1], c->pg.fsz[k >> 1], c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

// every part's field `name` (parity q) gets its halo slots from the neighbouring parts
dwf_status part_exchange(const PartSet &ps, const std::string &name, int prec, int q) {
  if (ps.comm) return part_exchange_comm(ps, name, prec, q);
  // 1. pack the cut faces
  for (dwf_ctx *c : ps.at) {
    Field f;
    TRY(part_field(c, name, prec, &f));
    for (int mu = 0; mu < 4; ++mu) {
      if (c->pg.grid[mu] == 1) continue;
      const size_t bytes = (size_t)c->pg.fsz[mu] * c->Ns * 12 * real_bytes(prec);
      for (int side = 0; side < 2; ++side) {
        void *send;
        TRY(get_raw(c, "part_send" + std::to_string(2 * mu + side), bytes, &send));
        CK(part_pack_any(prec, c, f, mu, side, q, send, c->stream));
      }
    }
  }
  for (dwf_ctx *c : ps.at) CK(cudaStreamSynchronize(c->stream));
  // 2. copy each neighbour's face into this part's receive buffers, 3. unpack into the halo
  for (dwf_ctx *c : ps.at) {
    Field f;
    TRY(part_field(c, name, prec, &f));
    for (int mu = 0; mu < 4; ++mu) {
      if (c->pg.grid[mu] == 1) continue;
      const size_t bytes = (size_t)c->pg.fsz[mu] * c->Ns * 12 * real_bytes(prec);
      for (int side = 0; side < 2; ++side) {
        // the upper halo (side 1) holds the upper neighbour's lower face, and vice versa
        int nc[4] = {c->pg.coord[0], c->pg.coord[1], c->pg.coord[2], c->pg.coord[3]};
        nc[mu] += side ? 1 : -1;
        dwf_ctx *n = ps.get(nc);
        void *send, *recv;
        TRY(get_raw(n, "part_send" + std::to_string(2 * mu + (1 - side)), bytes, &send));
        TRY(get_raw(c, "part_recv" + std::to_string(2 * mu + side), bytes, &recv));
        if (n->device == c->device) CK(cudaMemcpyAsync(recv, send, bytes, cudaMemcpyDeviceToDevice, c->stream));
        else CK(cudaMemcpyPeerAsync(recv, c->device, send, n->device, bytes, c->stream));
        CK(part_unpack_any(prec, c, recv, f, c->h + c->pg.foff[mu][side], c->pg.fsz[mu], c->stream));
      }
    }
  }
  for (dwf_ctx *c : ps.at) CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

// one hop stage on every part: out (parity outp) from in (the other parity, halos filled);
// m5: 0 none, 1 M5, 2 M5^T; optional operand fields y, r (updated in place) and b, and the
// reduction's result slot fin (each part's own sum; the caller adds the parts' sums)
struct PartHop {
  int epi;
  std::string in, out, y, r, b;
  int outp, m5;
  double coef;
  int fin = FIN_NONE;
};
dwf_status part_hop(const PartSet &ps, int prec, const PartHop &h) {
  TRY(part_exchange(ps, h.in, prec, 1 - h.outp));
  for (dwf_ctx *c : ps.at) {
    HopArgs a = hop_args(c, prec, h.outp);
    TRY(part_field(c, h.in, prec, &a.in));
    if (!h.out.empty()) TRY(part_field(c, h.out, prec, &a.out));
    if (!h.y.empty()) TRY(part_field(c, h.y, prec, &a.y));
    if (!h.r.empty()) TRY(part_field(c, h.r, prec, &a.r));
    if (!h.b.empty()) TRY(part_field(c, h.b, prec, &a.b));
    if (h.m5) set_m5(a, c, prec, h.m5 == 2);
    a.coef = h.coef;
    a.fin = h.fin;
    CK(hop_any(prec, h.epi, a, c->stream));
  }
  return DWF_OK;
}
dwf_status part_hop(const PartSet &ps, int prec, int epi, const std::string &in, const std::string &out,
                    const std::string &y, int outp, int m5, double coef) {
  PartHop h;
  h.epi = epi;
  h.in = in;
  h.out = out;
  h.y = y;
  h.outp = outp;
  h.m5 = m5;
  h.coef = coef;
  return part_hop(ps, prec, h);
}

// the parts of one decomposed lattice, checked: the same lattice, grid and operator, every
// block exactly once; the gauge forms of precisions prec (and FP64) built
dwf_status part_set(int nparts, dwf_ctx *const *parts, int prec, PartSet *ps) {
  dwf_ctx *c0 = parts[0];
  long total = 1;
  for (int mu = 0; mu < 4; ++mu) {
    ps->grid[mu] = c0->pg.grid[mu];
    total *= ps->grid[mu];
  }
  if (!c0->part || total != nparts) return fail(c0, DWF_EINVAL, "the parts must cover the grid once each");
  ps->at.assign(nparts, nullptr);
  for (int k = 0; k < nparts; ++k) {
    dwf_ctx *c = parts[k];
    if (!c || !c->part || c->Ns != c0->Ns || c->m0 != c0->m0 || c->mq != c0->mq || c->omega != c0->omega ||
        c->sigma != c0->sigma || memcmp(c->pg.G, c0->pg.G, sizeof(c->pg.G)) ||
        memcmp(c->pg.grid, c0->pg.grid, sizeof(c->pg.grid)))
      return fail(c0, DWF_EINVAL, "parts of different lattices or operators");
    const int *q = c->pg.coord;
    dwf_ctx *&slot = ps->at[q[0] + ps->grid[0] * (q[1] + ps->grid[1] * (q[2] + ps->grid[2] * q[3]))];
    if (slot) return fail(c0, DWF_EINVAL, "two parts at one grid position");
    slot = c;
    TRY(check_ctx(c));
    TRY(ensure_part_gauge(c, prec));
    TRY(ensure_part_gauge(c, P_F64));
  }
  return DWF_OK;
}

// this process's part under the caller's transport: the same checks as part_set for one part
dwf_status part_set_comm(dwf_ctx *c, const dwf_part_comm *comm, int prec, PartSet *ps) {
  if (!c->part) return fail(c, DWF_EINVAL, "not a partitioned context");
  if (!comm || !comm->exchange || !comm->allreduce) return fail(c, DWF_EINVAL, "null transport or callback");
  for (int mu = 0; mu < 4; ++mu) ps->grid[mu] = c->pg.grid[mu];
  ps->at.assign(1, c);
  ps->comm = comm;
  TRY(ensure_part_gauge(c, prec));
  TRY(ensure_part_gauge(c, P_F64));
  return DWF_OK;
}

// one part's field `name` (parity p) from its block in the local host layout, or into it
dwf_status part_scatter_local(dwf_ctx *c, const double *in, const std::string &name, int prec, int p) {
  const size_t n = (size_t)2 * c->pg.h * c->Ns * 24;
  void *d;
  TRY(get_raw(c, "part_host", n * sizeof(double), &d));
  CK(cudaMemcpyAsync(d, in, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  Field f;
  TRY(part_field(c, name, prec, &f));
  CK(pack_any(prec, static_cast<const double *>(d), f, local_geom(c->pg, c->Ns), p, c->sm_count, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}
dwf_status part_gather_local(dwf_ctx *c, const std::string &name, int prec, int p, double *out) {
  const size_t n = (size_t)2 * c->pg.h * c->Ns * 24;
  void *d;
  TRY(get_raw(c, "part_host", n * sizeof(double), &d));
  CK(cudaMemcpyAsync(d, out, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  Field f;
  TRY(part_field(c, name, prec, &f));
  CK(unpack_any(prec, f, static_cast<double *>(d), local_geom(c->pg, c->Ns), p, c->sm_count, c->stream));
  CK(cudaMemcpyAsync(out, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DWF_OK;
}

// where the caller's source comes from and the result goes: the global host arrays of
// dwf_part_apply / dwf_part_solve, or one part's local block under a transport
struct PartIO {
  std::function<dwf_status(const std::string &, int, int)> scatter;  // (field, prec, parity)
  std::function<dwf_status(const std::string &, int, int)> gather;   // into the output's sites of the parity
  std::function<void()> zero;                                       // the output set to 0
};

// every part's share of a global full-lattice host array into its field `name` (parity p)
dwf_status part_scatter(const PartSet &ps, const double *g_in, const std::string &name, int prec, int p) {
  std::vector<double> buf;
  for (dwf_ctx *c : ps.at) {
    TRY(check_ctx(c));
    const PartGeom &g = c->pg;
    const size_t gsite = (size_t)c->Ns * 24;
    buf.assign((size_t)2 * g.h * gsite, 0.0);
    for (long site = 0; site < 2 * g.h; ++site) {
      int x[4];
      long r = site;
      for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(r % g.L[mu]) + g.coord[mu] * g.L[mu];
        r /= g.L[mu];
      }
      const size_t gs = x[0] + (size_t)g.G[0] * (x[1] + (size_t)g.G[1] * (x[2] + (size_t)g.G[2] * x[3]));
      memcpy(&buf[site * gsite], g_in + gs * gsite, gsite * sizeof(double));
    }
    void *d;
    TRY(get_raw(c, "part_host", buf.size() * sizeof(double), &d));
    CK(cudaMemcpyAsync(d, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    Field f;
    TRY(part_field(c, name, prec, &f));
    CK(pack_any(prec, static_cast<const double *>(d), f, local_geom(g, c->Ns), p, c->sm_count, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DWF_OK;
}

// every part's field `name` (parity p) into the global host array (its sites of parity p)
dwf_status part_gather(const PartSet &ps, const std::string &name, int prec, int p, double *g_out) {
  std::vector<double> buf;
  for (dwf_ctx *c : ps.at) {
    TRY(check_ctx(c));
    const PartGeom &g = c->pg;
    const size_t gsite = (size_t)c->Ns * 24;
    void *d;
    TRY(get_raw(c, "part_host", (size_t)2 * g.h * gsite * sizeof(double), &d));
    CK(cudaMemsetAsync(d, 0, (size_t)2 * g.h * gsite * sizeof(double), c->stream));
    Field f;
    TRY(part_field(c, name, prec, &f));
    CK(unpack_any(prec, f, static_cast<double *>(d), local_geom(g, c->Ns), p, c->sm_count, c->stream));
    buf.assign((size_t)2 * g.h * gsite, 0.0);
    CK(cudaMemcpyAsync(buf.data(), d, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (long site = 0; site < 2 * g.h; ++site) {
      int x[4];
      long r = site;
      for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(r % g.L[mu]) + g.coord[mu] * g.L[mu];
        r /= g.L[mu];
      }
      if (((x[0] + x[1] + x[2] + x[3]) & 1) != p) continue;
      const size_t gs = x[0] + (size_t)g.G[0] * (x[1] + (size_t)g.G[1] * (x[2] + (size_t)g.G[2] * x[3]));
      memcpy(g_out + gs * gsite, &buf[site * gsite], gsite * sizeof(double));
    }
  }
  return DWF_OK;
}

}  // namespace

extern "C" dwf_status dwf_create_part(const dwf_partition *pt, int Ns, double m0, double mq, const double *omega,
                                      const double *sigma, dwf_ctx **out) {
  if (!pt || !out) return DWF_EINVAL;
  *out = nullptr;
  int L[4];
  for (int mu = 0; mu < 4; ++mu) {
    if (pt->grid[mu] < 1 || pt->global_dims[mu] < 2 || pt->global_dims[mu] % pt->grid[mu]) return DWF_EINVAL;
    L[mu] = pt->global_dims[mu] / pt->grid[mu];
    if (L[mu] < 2 || (L[mu] & 1) || pt->coord[mu] < 0 || pt->coord[mu] >= pt->grid[mu]) return DWF_EINVAL;
  }
  dwf_ctx *c = nullptr;
  TRY(dwf_create(L, Ns, m0, mq, omega, sigma, &c));
  c->part = true;
  c->pg = make_part_geom(pt->global_dims, pt->grid, pt->coord);
  for (int p = 0; p < 2; ++p) k_part_neighbours<0><<<vec_grid(c->h, c->sm_count), 256, 0, c->stream>>>(c->d_nbr[p], c->pg, p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    dwf_destroy(c);
    return DWF_ECUDA;
  }
  *out = c;
  return DWF_OK;
}

extern "C" dwf_status dwf_load_gauge_part(dwf_ctx *c, const double *U) {
  TRY(check_ctx(c));
  if (!c->part) return fail(c, DWF_EINVAL, "not a partitioned context");
  if (!U) return fail(c, DWF_EINVAL, "null gauge pointer");
  const size_t bytes = (size_t)c->pg.G[0] * c->pg.G[1] * c->pg.G[2] * c->pg.G[3] * 72 * sizeof(double);
  if (!c->d_Ug) CK(dmalloc((void **)&c->d_Ug, bytes, c->device, c->stream));
  CK(cudaMemcpyAsync(c->d_Ug, U, bytes, cudaMemcpyHostToDevice, c->stream));
  for (bool &r : c->gauge_ready) r = false;
  TRY(ensure_part_gauge(c, P_F64));
  TRY(ensure_part_gauge(c, P_F32));
  return DWF_OK;
}

namespace {

dwf_status check_part_op(dwf_ctx *c0, int op, int prec, int parity) {
  if (!valid_prec(prec)) return fail(c0, DWF_EINVAL, "unknown precision");
  if (op < DWF_OP_DEO || op > DWF_OP_CCDAG || op == DWF_OP_M5 || op == DWF_OP_M5T)
    return fail(c0, DWF_EINVAL, "dwf_part_apply applies DEO, DOE, C, CDAG or CCDAG");
  if (op >= DWF_OP_C && parity != 0 && parity != 1) return fail(c0, DWF_EINVAL, "parity must be 0 or 1");
  return DWF_OK;
}

dwf_status part_apply_core(const PartSet &ps, const PartIO &io, int op, int prec, int parity) {
  const int inpar = op == DWF_OP_DEO ? 1 : op == DWF_OP_DOE ? 0 : parity;
  const int outpar = op == DWF_OP_DEO ? 0 : op == DWF_OP_DOE ? 1 : parity;
  TRY(io.scatter("in", prec, inpar));
  const int sp = parity, opp = 1 - parity;
  switch (op) {
    case DWF_OP_DEO:
    case DWF_OP_DOE:
      TRY(part_hop(ps, prec, E_PLAIN, "in", "out", "", outpar, 0, -0.5));
      break;
    case DWF_OP_C:  // Eq. 11: u = -1/2 M5 H v; out = v + 1/2 M5 H u
      TRY(part_hop(ps, prec, E_M, "in", "u", "", opp, 1, -0.5));
      TRY(part_hop(ps, prec, E_M_XPAY, "u", "out", "in", sp, 1, 0.5));
      break;
    case DWF_OP_CDAG:
    case DWF_OP_CCDAG: {
      // C^dag v = g5 (1 - D M5^T D M5^T) g5 v: w = M5^T g5 v; t = -1/2 M5^T H w; q = v + 1/2 g5 H t
      for (dwf_ctx *c : ps.at) {
        Field fi, fw;
        TRY(part_field(c, "in", prec, &fi));
        TRY(part_field(c, "w", prec, &fw));
        TRY(smix(c, c->stream, prec, S_G5, fi, fw, MK_M5T, 1.0, DWF_KC_OTHER));
      }
      const std::string q = op == DWF_OP_CDAG ? "out" : "q";
      TRY(part_hop(ps, prec, E_M, "w", "t", "", opp, 2, -0.5));
      TRY(part_hop(ps, prec, E_XPAY_G5, "t", q, "in", sp, 0, 0.5));
      if (op == DWF_OP_CCDAG) {
        TRY(part_hop(ps, prec, E_M, "q", "u", "", opp, 1, -0.5));
        TRY(part_hop(ps, prec, E_M_XPAY, "u", "out", "q", sp, 1, 0.5));
      }
      break;
    }
  }
  io.zero();
  return io.gather("out", prec, outpar);
}

// the global host arrays of dwf_part_apply / dwf_part_solve
PartIO global_io(const PartSet &ps, const double *in, double *out) {
  dwf_ctx *c0 = ps.at[0];
  PartIO io;
  io.scatter = [&ps, in](const std::string &name, int prec, int p) { return part_scatter(ps, in, name, prec, p); };
  io.gather = [&ps, out](const std::string &name, int prec, int p) { return part_gather(ps, name, prec, p, out); };
  io.zero = [c0, out]() {
    const int *G = c0->pg.G;
    memset(out, 0, (size_t)G[0] * G[1] * G[2] * G[3] * c0->Ns * 24 * sizeof(double));
  };
  return io;
}

// one part's local blocks under a transport
PartIO local_io(dwf_ctx *c, const double *in, double *out) {
  PartIO io;
  io.scatter = [c, in](const std::string &name, int prec, int p) { return part_scatter_local(c, in, name, prec, p); };
  io.gather = [c, out](const std::string &name, int prec, int p) { return part_gather_local(c, name, prec, p, out); };
  io.zero = [c, out]() { memset(out, 0, (size_t)2 * c->pg.h * c->Ns * 24 * sizeof(double)); };
  return io;
}

}  // namespace

extern "C" dwf_status dwf_part_apply(int nparts, dwf_ctx *const *parts, int op, int prec, int parity,
                                     const double *in, double *out) {
  if (nparts < 1 || !parts || !parts[0] || !in || !out) return DWF_EINVAL;
  dwf_ctx *c0 = parts[0];
  TRY(check_ctx(c0));
  TRY(check_part_op(c0, op, prec, parity));
  PartSet ps;
  TRY(part_set(nparts, parts, prec, &ps));
  return part_apply_core(ps, global_io(ps, in, out), op, prec, parity);
}

extern "C" dwf_status dwf_part_apply_comm(dwf_ctx *part, const dwf_part_comm *comm, int op, int prec, int parity,
                                          const double *in, double *out) {
  TRY(check_ctx(part));
  if (!in || !out) return fail(part, DWF_EINVAL, "null field pointer");
  TRY(check_part_op(part, op, prec, parity));
  PartSet ps;
  TRY(part_set_comm(part, comm, prec, &ps));
  return part_apply_core(ps, local_io(part, in, out), op, prec, parity);
}

namespace {

// the parts' reduction results added over the parts (the allreduce of a multi-GPU run):
// slot 0 = red, 1 = red2 of every part's scalar block
dwf_status part_sum(const PartSet &ps, int slot, double *out) {
  double s = 0;
  for (dwf_ctx *c : ps.at) {
    TRY(pull_scalars(c, c->stream));
    s += slot ? c->h_sc->red2 : c->h_sc->red;
  }
  if (ps.comm && ps.comm->allreduce(ps.comm->user, &s, 1) != 0)
    return fail(ps.at[0], DWF_ECOMM, "the allreduce callback failed");
  *out = s;
  return DWF_OK;
}

// alpha and beta of the inner CG to every part's scalar block
dwf_status part_set_ab(const PartSet &ps, double alpha, double beta) {
  for (dwf_ctx *c : ps.at) {
    CGScalars &h = *c->h_sc;
    h.alpha = alpha;
    h.alpha_f = (float)alpha;
    h.beta = beta;
    h.beta_f = (float)beta;
    h.restart_flag = 0;
    TRY(push_scalars(c, c->stream));
  }
  return DWF_OK;
}

dwf_status part_norm2(const PartSet &ps, const std::string &name, int prec, double *out) {
  for (dwf_ctx *c : ps.at) {
    Field f;
    TRY(part_field(c, name, prec, &f));
    TRY(norm2(c, c->stream, prec, f, FIN_RED));
  }
  return part_sum(ps, 0, out);
}

// rh = b - C C^dag xh in FP64 on Schur parity sp, |rh|^2 over all parts (Eq. 11)
dwf_status part_resid64(const PartSet &ps, int sp, double *rr) {
  for (dwf_ctx *c : ps.at) {
    Field x, w;
    TRY(part_field(c, "xh", P_F64, &x));
    TRY(part_field(c, "w64", P_F64, &w));
    TRY(smix(c, c->stream, P_F64, S_G5, x, w, MK_M5T, 1.0, DWF_KC_F64));
  }
  TRY(part_hop(ps, P_F64, E_M, "w64", "t64", "", 1 - sp, 2, -0.5));
  TRY(part_hop(ps, P_F64, E_XPAY_G5, "t64", "q64", "xh", sp, 0, 0.5));
  TRY(part_hop(ps, P_F64, E_M, "q64", "u64", "", 1 - sp, 1, -0.5));
  PartHop h;
  h.epi = E_RESID;
  h.in = "u64";
  h.out = "rh";
  h.y = "q64";
  h.b = "b";
  h.outp = sp;
  h.m5 = 1;
  h.coef = 0.5;
  h.fin = FIN_RED;
  TRY(part_hop(ps, P_F64, h));
  return part_sum(ps, 0, rr);
}

}  // namespace

namespace {

dwf_status part_solve_params(dwf_ctx *c0, const dwf_solve_params *pp, dwf_solve_params *prm) {
  if (pp) *prm = *pp;
  else dwf_solve_params_default(prm);
  if (!(prm->tol > 0.0) || !valid_prec(prm->inner_prec) ||
      (prm->system != DWF_SYS_FULL && prm->system != DWF_SYS_NORMAL) ||
      (prm->schur_parity != 0 && prm->schur_parity != 1) || prm->max_iter < 1)
    return fail(c0, DWF_EINVAL, "invalid solve parameters");
  return DWF_OK;
}

// the solve across the parts of ps (all of them, or this process's one under a transport)
dwf_status part_solve_core(const PartSet &ps, const PartIO &io, const dwf_solve_params &prm,
                           dwf_solve_stats *stats) {
  dwf_ctx *c0 = ps.at[0];
  const int P = prm.inner_prec, sp = prm.schur_parity, opp = 1 - sp;
  const bool full = prm.system == DWF_SYS_FULL;
  const double delta = prm.delta > 0.0 ? prm.delta : default_delta(prm.inner_prec);
  const auto t0 = std::chrono::steady_clock::now();
  // ---- the Schur-parity source (Eq. 10 for the full system): b = eta'_sp - M5 D eta'_op
  if (full) {
    for (int p = 0; p < 2; ++p) TRY(io.scatter("eta" + std::to_string(p), P_F64, p));
    for (dwf_ctx *c : ps.at)
      for (int p = 0; p < 2; ++p) {
        Field e, ep;
        TRY(part_field(c, "eta" + std::to_string(p), P_F64, &e));
        TRY(part_field(c, "etap" + std::to_string(p), P_F64, &ep));
        TRY(smix(c, c->stream, P_F64, S_PLAIN, e, ep, MK_S1, 1.0, DWF_KC_F64));
      }
    TRY(part_hop(ps, P_F64, E_M_XPAY, "etap" + std::to_string(opp), "b", "etap" + std::to_string(sp), sp, 1, 0.5));
  } else {
    TRY(io.scatter("b", P_F64, sp));
  }
  double bnorm2 = 0;
  TRY(part_norm2(ps, "b", P_F64, &bnorm2));
  const double tol_schur = full ? 0.01 * (prm.schur_target_pct > 0 ? prm.schur_target_pct : 50) * prm.tol : prm.tol;
  // x_hat = 0, r_hat = b, r = b in the inner precision, x = p = 0
  for (dwf_ctx *c : ps.at) {
    Field xh, rh, b, x, p, r;
    TRY(part_field(c, "xh", P_F64, &xh));
    TRY(part_field(c, "rh", P_F64, &rh));
    TRY(part_field(c, "b", P_F64, &b));
    TRY(part_field(c, "cg_x", xprec(P), &x));
    TRY(part_field(c, "cg_p", P, &p));
    TRY(part_field(c, "cg_r", P, &r));
    const size_t n = (size_t)c->h * c->Ns;
    CK(cudaMemsetAsync(xh.v, 0, n * site_bytes(P_F64), c->stream));
    CK(cudaMemcpyAsync(rh.v, b.v, n * site_bytes(P_F64), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(x.v, 0, n * site_bytes(xprec(P)), c->stream));
    CK(cudaMemsetAsync(p.v, 0, n * site_bytes(P), c->stream));
    if (p.nrm) CK(cudaMemsetAsync(p.nrm, 0, n * sizeof(float), c->stream));
    TRY(convert(c, c->stream, P_F64, b, P, r, DWF_KC_OTHER));
  }
  double rr = 0;
  TRY(part_norm2(ps, "cg_r", P, &rr));
  double rhat2 = bnorm2, rmax = rr, alpha = 0, beta = 0;
  int iters = 0, restarts = 0;
  bool converged = bnorm2 == 0.0;
  // ---- mixed-precision CG on C C^dag (Algorithm 1) with FP64 reliable updates (Sec. 2.3),
  // the global sums of every reduction taken over the parts
  while (!converged && iters < prm.max_iter) {
    TRY(part_set_ab(ps, alpha, beta));
    for (dwf_ctx *c : ps.at) {  // x += alpha p (the previous step), p = r + beta p, w = M5^T g5 p
      SmixArgs m;
      memset(&m, 0, sizeof(m));
      TRY(part_field(c, "cg_w", P, &m.out));
      TRY(part_field(c, "cg_r", P, &m.r));
      TRY(part_field(c, "cg_p", P, &m.p));
      TRY(part_field(c, "cg_x", xprec(P), &m.x));
      m.K = dmat(c, P, MK_M5T);
      m.K2 = dmat(c, P, MK_ID);
      m.coef = 1.0;
      m.h = c->h;
      m.Ns = c->Ns;
      m.sc = c->d_sc;
      CK(smix_any(P, S_CGP, m, c->stream));
    }
    TRY(part_hop(ps, P, E_M, "cg_w", "cg_t", "", opp, 2, -0.5));
    PartHop xq;
    xq.epi = E_XPAY_G5;
    xq.in = "cg_t";
    xq.out = "cg_q";
    xq.y = "cg_p";
    xq.outp = sp;
    xq.m5 = 0;
    xq.coef = 0.5;
    xq.fin = FIN_RED;
    TRY(part_hop(ps, P, xq));
    double qq = 0;
    TRY(part_sum(ps, 0, &qq));
    alpha = rr / qq;  // (r, r) / (p, A p), (p, A p) = |C^dag p|^2
    TRY(part_set_ab(ps, alpha, beta));
    TRY(part_hop(ps, P, E_M, "cg_q", "cg_u", "", opp, 1, -0.5));
    PartHop up;
    up.epi = E_CG_UPDATE;
    up.in = "cg_u";
    up.y = "cg_q";
    up.r = "cg_r";
    up.outp = sp;
    up.m5 = 1;
    up.coef = 0.5;
    up.fin = FIN_RED2;
    TRY(part_hop(ps, P, up));  // r -= alpha (q + 1/2 M5 H u), |r|^2
    double rr_new = 0;
    TRY(part_sum(ps, 1, &rr_new));
    ++iters;
    beta = rr_new / rr;
    const double rr_prev = rr;
    rr = rr_new;
    rmax = std::max(rmax, rr);
    if (!(rr > tol_schur * tol_schur * bnorm2) || !(rr > delta * delta * rmax) || iters >= prm.max_iter) {
      // FP64 restart: x_hat += x + alpha p, x = 0; r_hat = b - C C^dag x_hat; r = r_hat
      for (dwf_ctx *c : ps.at) {
        VecArgs v;
        memset(&v, 0, sizeof(v));
        TRY(part_field(c, "xh", P_F64, &v.a));
        TRY(part_field(c, "cg_x", xprec(P), &v.b));
        TRY(part_field(c, "cg_p", P, &v.c));
        v.sc = c->d_sc;
        v.n = c->h * c->Ns;
        v.Ns = c->Ns;
        CK(accum_any(P, v, c->sm_count, c->stream));
      }
      TRY(part_resid64(ps, sp, &rhat2));
      ++restarts;
      for (dwf_ctx *c : ps.at) {
        Field rh, r;
        TRY(part_field(c, "rh", P_F64, &rh));
        TRY(part_field(c, "cg_r", P, &r));
        TRY(convert(c, c->stream, P_F64, rh, P, r, DWF_KC_F64));
      }
      TRY(part_norm2(ps, "cg_r", P, &rr));
      converged = rhat2 <= tol_schur * tol_schur * bnorm2;
      // reliable update: keep p, beta from the recomputed residual; the pending step is in x_hat
      beta = rr / rr_prev;
      alpha = 0;
      rmax = rr;
    }
  }
  double res_full = 0;
  if (full) {
    // phi_sp = C^dag x_hat; phi_op = eta'_op - M5 D phi_sp; psi = S2 phi (Eq. 9-10)
    for (dwf_ctx *c : ps.at) {
      Field x, w;
      TRY(part_field(c, "xh", P_F64, &x));
      TRY(part_field(c, "w64", P_F64, &w));
      TRY(smix(c, c->stream, P_F64, S_G5, x, w, MK_M5T, 1.0, DWF_KC_F64));
    }
    TRY(part_hop(ps, P_F64, E_M, "w64", "t64", "", opp, 2, -0.5));
    TRY(part_hop(ps, P_F64, E_XPAY_G5, "t64", "phi" + std::to_string(sp), "xh", sp, 0, 0.5));
    TRY(part_hop(ps, P_F64, E_M_XPAY, "phi" + std::to_string(sp), "phi" + std::to_string(opp),
                 "etap" + std::to_string(opp), opp, 1, 0.5));
    for (dwf_ctx *c : ps.at)
      for (int p = 0; p < 2; ++p) {
        Field ph, psi, t, z;
        TRY(part_field(c, "phi" + std::to_string(p), P_F64, &ph));
        TRY(part_field(c, "psi" + std::to_string(p), P_F64, &psi));
        TRY(smix(c, c->stream, P_F64, S_PLAIN, ph, psi, MK_S2, 1.0, DWF_KC_F64));
        // D psi of Eq. 5 on both parities: z = ((d - m0)(omega + sigma L) + 1 - L) psi, t = (omega + sigma L) psi
        TRY(part_field(c, "tt" + std::to_string(p), P_F64, &t));
        TRY(part_field(c, "z" + std::to_string(p), P_F64, &z));
        TRY(smix(c, c->stream, P_F64, S_DUAL, psi, t, MK_W, 1.0, DWF_KC_F64, z, MK_Z));
      }
    io.zero();
    for (int p = 0; p < 2; ++p) {
      TRY(io.gather("psi" + std::to_string(p), P_F64, p));
      TRY(part_hop(ps, P_F64, E_XPAY, "tt" + std::to_string(1 - p), "dpsi" + std::to_string(p),
                   "z" + std::to_string(p), p, 0, -0.5));
    }
    double num = 0, den = 0;
    for (int p = 0; p < 2; ++p) {
      for (dwf_ctx *c : ps.at) {
        VecArgs v;
        memset(&v, 0, sizeof(v));
        TRY(part_field(c, "eta" + std::to_string(p), P_F64, &v.a));
        TRY(part_field(c, "dpsi" + std::to_string(p), P_F64, &v.b));
        v.n = c->h * c->Ns;
        v.Ns = c->Ns;
        v.fin = FIN_RED;
        v.sc = c->d_sc;
        v.partials = c->d_part;
        v.ticket = c->d_ticket;
        CK(diff_norm2_launch(v, c->sm_count, c->stream));
      }
      double a = 0, b = 0;
      TRY(part_sum(ps, 0, &a));
      TRY(part_norm2(ps, "eta" + std::to_string(p), P_F64, &b));
      num += a;
      den += b;
    }
    res_full = den > 0 ? sqrt(num / den) : 0.0;
  } else {
    io.zero();
    TRY(io.gather("xh", P_F64, sp));
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iters = iters;
    stats->restarts = restarts;
    stats->mode_used = DWF_MODE_RELIABLE;
    stats->converged = converged ? 1 : 0;
    stats->true_res = bnorm2 > 0 ? sqrt(rhat2 / bnorm2) : 0.0;
    stats->true_res_full = res_full;
    stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const double n = (double)c0->pg.G[0] * c0->pg.G[1] * c0->pg.G[2] * c0->pg.G[3] / 2 * c0->Ns;
    stats->flops = n * (iters * flops_cg_iter(c0->Ns) + restarts * flops_restart(c0->Ns) +
                        (full ? flops_prep_recon(c0->Ns) : 0.0));
    stats->inner_prec_used = P;
  }
  if (!converged) return fail(c0, DWF_ENOCONV, "max_iter reached");
  if (full && res_full > prm.tol) return fail(c0, DWF_ENOCONV, "full-system residual above tol");
  return DWF_OK;
}

}  // namespace

extern "C" dwf_status dwf_part_solve(int nparts, dwf_ctx *const *parts, const double *rhs, double *sol,
                                     const dwf_solve_params *pp, dwf_solve_stats *stats) {
  if (nparts < 1 || !parts || !parts[0] || !rhs || !sol) return DWF_EINVAL;
  dwf_ctx *c0 = parts[0];
  TRY(check_ctx(c0));
  dwf_solve_params prm;
  TRY(part_solve_params(c0, pp, &prm));
  PartSet ps;
  TRY(part_set(nparts, parts, prm.inner_prec, &ps));
  return part_solve_core(ps, global_io(ps, rhs, sol), prm, stats);
}

extern "C" dwf_status dwf_part_solve_comm(dwf_ctx *part, const dwf_part_comm *comm, const double *rhs, double *sol,
                                          const dwf_solve_params *pp, dwf_solve_stats *stats) {
  TRY(check_ctx(part));
  if (!rhs || !sol) return fail(part, DWF_EINVAL, "null field pointer");
  dwf_solve_params prm;
  TRY(part_solve_params(part, pp, &prm));
  PartSet ps;
  TRY(part_set_comm(part, comm, prm.inner_prec, &ps));
  return part_solve_core(ps, local_io(part, rhs, sol), prm, stats);
}
