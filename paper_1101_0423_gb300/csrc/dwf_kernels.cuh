// dwf_kernels.cuh -- kernel templates of the domain-wall solver (sm_103a).
//
// Kernels (the paper's five catalogs of Sec. 3, re-designed):
//   k_hop    Eq. 12 hopping block on every s-slice, links staged once per CTA in shared
//            memory by a TMA bulk copy and reused by the Ns threads of a site (Sec. 3.2),
//            with fused epilogues: M5 (Sec. 3.3), vector add/sub (Sec. 3.5), CG update and
//            the block partial sums of the reductions (Sec. 3.4).
//   k_smix   per-site matrices along s (M5, M5^T, S1, S2, omega + sigma L, ...), with the
//            CG direction update p = r + beta p fused in front.
//   k_pack / k_unpack  host layout <-> device layout (Sec. 3.1), precision conversion.
//   k_norm2, k_accum, k_convert  reductions and vector updates.
// Reductions: per-thread partials promoted to FP64, warp shuffles, block sums written to
// a partials array; the last block to finish (atomic ticket) sums the partials in a fixed
// order, so every result is deterministic and stays on the device.
#pragma once

#include "dwf_device.cuh"

namespace dwf {

// ------------------------------------------------------------------ TMA bulk copy + mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// bounded wait on phase `ph`; false if the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t ph, uint32_t max_tries) {
  for (uint32_t i = 0; i < max_tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(ph)
        : "memory");
    if (done) return true;
  }
  return false;
}
// each try_wait suspends for a bounded time (measured on GB300: about 3.8 us when the phase
// does not complete), so the default bound gives up after about one second
constexpr uint32_t kWaitTries = 1u << 18;

enum { ERR_TMA_TIMEOUT = 1 };

// ------------------------------------------------------------------ reductions

// sum over the first `nact` lanes of a warp (lanes >= nact may not exist: the block size
// need not be a multiple of 32); result valid in lane 0
__device__ __forceinline__ int lin_tid() {
  return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

template <typename V>
__device__ __forceinline__ V warp_sum(V v, int nact) {
  const int lane = lin_tid() & 31;
  const unsigned mask = nact >= 32 ? 0xffffffffu : ((1u << nact) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const V t = __shfl_down_sync(mask, v, o);
    if (lane + o < nact) v += t;
  }
  return v;
}

// sum over the block (result valid in thread 0); `ws` holds >= 32 doubles.  The 32 lanes
// of a warp are summed in the kernel's own precision V (FP32 kernels keep their FP32
// pipes; GB300's FP64 units are few), the warp sums in FP64 and in a fixed order.
template <typename V>
__device__ __forceinline__ double block_sum(V v, double *ws) {
  const int tid = lin_tid();
  const int nthr = nthreads();
  const int nw = (nthr + 31) >> 5;
  v = warp_sum<V>(v, min(32, nthr - (tid & ~31)));
  __syncthreads();
  if ((tid & 31) == 0) ws[tid >> 5] = (double)v;
  __syncthreads();
  double r = 0;
  if (tid < 32) {
    r = tid < nw ? ws[tid] : 0.0;
    r = warp_sum<double>(r, 32);
  }
  return r;
}

// which scalar the last block writes
enum { FIN_NONE = 0, FIN_RED = 1, FIN_RED2 = 2, FIN_QQ = 3, FIN_CG = 4 };

__device__ __forceinline__ void finish(int fin, double tot, CGScalars *sc) {
  if (fin == FIN_RED) sc->red = tot;
  else if (fin == FIN_RED2) sc->red2 = tot;
  else if (fin == FIN_QQ) {
    // Algorithm 1: alpha = (r, r) / (p, A p), with (p, A p) = |C^dag p|^2
    sc->qq = tot;
    sc->alpha = sc->rr / tot;
    sc->alpha_f = (float)sc->alpha;
  }
  else if (fin == FIN_CG) {
    // end of one CG iteration (Algorithm 1): beta = (r_new, r_new) / (r, r)
    const double rr_new = tot;
    sc->beta = rr_new / sc->rr;
    sc->beta_f = (float)sc->beta;
    sc->rr_old = sc->rr;
    sc->rr = rr_new;
    sc->iter += 1;
    if (rr_new > sc->rmax2) sc->rmax2 = rr_new;
    if (rr_new < sc->rr_min) {
      sc->rr_min = rr_new;
      sc->iter_min = sc->iter;
    }
    // FP64 restart due (Sec. 2.3): the residual fell by delta (reliable update) or reached
    // the target; or the iteration cap; or the recursion diverged, stalled or stopped
    // being a number (then the host resets the search direction)
    if (!(rr_new > sc->target2)) sc->restart_flag = RS_TARGET;
    else if (!(rr_new > sc->delta2 * sc->rmax2)) sc->restart_flag = RS_DELTA;
    else if (sc->iter >= sc->iter_cap) sc->restart_flag = RS_CAP;
    else if (!(rr_new < 1e6 * sc->rr_start)) sc->restart_flag = RS_DIVERGED;
    else if (sc->iter - sc->iter_min > sc->stall_iters) sc->restart_flag = RS_STALLED;
  }
}

// grid-wide deterministic sum; every thread of every block must call it
template <typename V>
__device__ __forceinline__ void grid_sum(V v, double *partials, unsigned *ticket, int fin, CGScalars *sc) {
  __shared__ double ws[32];
  __shared__ int am_last;
  const int tid = lin_tid();
  const int nthr = nthreads();
  double bs = block_sum<V>(v, ws);
  if (tid == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    // all of this thread's partials are requested before any is added (one L2 round trip
    // instead of one per partial: the rest of the GPU idles during this tail); the order of
    // the additions is fixed by the grid, so the sum is reproducible
    constexpr int U = 8;
    double s = 0;
    unsigned i = tid;
    for (; i + (U - 1) * nthr < gridDim.x; i += U * nthr) {
      double q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) q[u] = __ldcg(partials + i + u * nthr);
#pragma unroll
      for (int u = 0; u < U; ++u) s += q[u];
    }
    for (; i < gridDim.x; i += nthr) s += __ldcg(partials + i);
    double tot = block_sum<double>(s, ws);
    if (tid == 0) {
      finish(fin, tot, sc);
      *ticket = 0u;
    }
  }
}

// ------------------------------------------------------------------ hop kernel

// epilogues of k_hop (H = raw hopping sum, D = -H/2; K = matrix along s, coefficient folded in)
enum {
  E_PLAIN = 0,     // out = coef H
  E_M = 1,         // out = K H
  E_XPAY_G5 = 2,   // out = y + coef g5 H, |out|^2 -> fin
  E_XPAY = 3,      // out = y + coef H
  E_M_XPAY = 4,    // out = y + K H
  E_CG_UPDATE = 5, // Ap = y + K H; r -= alpha Ap; |r|^2 -> FIN_CG
  E_RESID = 6      // out = b - (y + K H), |out|^2 -> fin
};

template <int EPI> struct EpiT {
  static constexpr bool has_m = EPI == E_M || EPI == E_M_XPAY || EPI == E_CG_UPDATE || EPI == E_RESID;
  static constexpr bool has_red = EPI == E_XPAY_G5 || EPI == E_CG_UPDATE || EPI == E_RESID;
};

struct HopArgs {
  Field in, out, y, b, r;
  const void *gauge;   // doubled gauge of the output parity: [cb][SITE_LREALS], links [8][LREALS]
  const int *nbr;      // [cb][8] for the output parity
  const void *K;       // FP32 arithmetic: M5 or M5^T, dense, kernel order K[chi][t][s]
  const void *rec;     // FP64: the same as a recurrence table along s, per chirality Ns
                       // steps of {PS, PN, BB, AI, QS, QN, W, 0}
  int mtrans;          // 0: M5, 1: M5^T (direction of each chirality's recurrence)
  double kappa;        // corner of L, -mq / (2 m0) (Eq. 4)
  double coef;         // scale of H (plain/xpay) or of the matrix (M5 epilogues)
  long h;              // sites per parity
  int Ns;
  int fin;             // FIN_* of the reduction
  int use_flag;        // honour CGScalars::restart_flag (skip work once set)
  uint32_t wait_tries; // bound of each wait for a tile's copies, in mbarrier polls
  int skip_copies;     // failure-detection hook: issue no copies, so every wait runs out
  CGScalars *sc;
  double *partials;
  unsigned *ticket;
  // batches of right-hand sides: blockIdx.y selects one; its fields start fstride bytes
  // (norms nstride floats) after the previous one's, and it has its own scalars, partial
  // sums (part_stride doubles apart) and ticket
  int nrhs;
  size_t fstride, nstride;
  size_t part_stride;
  // launch shape chosen by the host (autotuner); 0 threads: the default shape
  int shape_threads;
  int shape_persistent;
};

__device__ __forceinline__ Field field_rhs(Field f, int rb, size_t fstride, size_t nstride) {
  if (f.v) f.v = static_cast<char *>(f.v) + rb * fstride;
  if (f.nrm) f.nrm += rb * nstride;
  return f;
}

// L2 prefetch of a contiguous range (an epilogue operand of this CTA's sites)
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// dynamic shared memory of k_hop, in bytes:
//   [mbarriers, 64][links as copied] x nb [neighbour indices] x nb [16-bit links expanded][M]
// with nb = 2 when a persistent CTA receives the next tile while computing this one, else 1
// (links and indices arrive by TMA bulk copies).  FP32 and FP64 kernels use the links as
// copied (FP32 links are padded to 80 bytes, so the nine complex entries are five aligned
// float4); the 16-bit forms rebuild each link's third row and expand the tile's links into
// that same FP32 form.  The M5 staging rows overlay everything from offset 64 on (kernels
// with an M5 epilogue take one tile per CTA, so the link buffers are dead by then).  Shared
// memory is kept small on purpose: what the CTAs leave of the SM's 256 KB is the L1 that
// holds the neighbour gathers in flight.
template <int P> struct HopSmem {
  static constexpr bool F2 = !(P == P_F64);
  using RL = typename PT<P>::real;
  __host__ __device__ static size_t raw(int nsite) {
    return (size_t)nsite * PT<P>::SITE_LREALS * sizeof(typename PT<P>::lreal);
  }
  __host__ __device__ static size_t off_raw(int spb, int b) { return 64 + (size_t)b * align16(raw(spb)); }
  __host__ __device__ static size_t off_nbr(int spb, int nb, int b) {
    return 64 + (size_t)nb * align16(raw(spb)) + (size_t)b * align16((size_t)spb * 8 * 4);
  }
  __host__ __device__ static size_t off_exp(int spb, int nb) {
    return 64 + (size_t)nb * (align16(raw(spb)) + align16((size_t)spb * 8 * 4));
  }
  // one row of 24 reals per s, padded by 16 bytes so that the eight s-rows a quarter-warp
  // stores fall in distinct bank groups; sites padded by another 16 bytes
  static constexpr int ROW = 24 + 16 / (int)sizeof(RL);
  __host__ __device__ static size_t stage(int spb, int Ns) { return (size_t)spb * (Ns * ROW * sizeof(RL) + 16); }
  // FP32 links are used as copied; the 16-bit forms are expanded
  static constexpr bool EXPAND = F2 && P != P_F32;
  __host__ __device__ static size_t off_k(int spb, int Ns, int nb, bool has_m) {
    const size_t e = off_exp(spb, nb) + (EXPAND ? (size_t)spb * LINK_SITE_F4 * 16 : 0);
    const size_t st = has_m ? 64 + stage(spb, Ns) : 0;
    return align16(e > st ? e : st);
  }
  // M5 / M5^T: dense (FP32 arithmetic) or a recurrence table of 2 chiralities x Ns steps x
  // 8 reals (FP64).  Dense, even Ns: per chirality and t a row of Ns/2 pairs
  // (K[b][t], K[b + Ns/2][t]), the second chirality kq_stride pairs after the first; odd Ns:
  // (k, k) pairs K[chi][t][s].
  __host__ __device__ static int kq_stride(int Ns) {
    // pad so that the two chiralities' rows start 16 banks apart: a half-warp reads one t-row
    // of each chirality at once (Ns/2 pairs = Ns words each, Ns <= 16), or one of a single
    // chirality (Ns = 32)
    return Ns * (Ns / 2) + ((16 - (Ns * Ns) % 32 + 32) % 32) / 2;
  }
  __host__ __device__ static size_t kbytes(int Ns) {
    if (!F2) return (size_t)2 * Ns * 8 * sizeof(RL);
    const size_t dense = (size_t)2 * Ns * Ns * 8, paired = (size_t)2 * kq_stride(Ns) * 8;
    return dense > paired ? dense : paired;
  }
  __host__ __device__ static size_t bytes(int spb, int Ns, int nb, bool has_m) {
    return off_k(spb, Ns, nb, has_m) + (has_m ? align16(kbytes(Ns)) : 0);
  }
};

// the dense FP32 M5 epilogue's layout with four K entries per 16-byte read (Ns divides 32)
__host__ __device__ constexpr bool m5_quad(int Ns) { return Ns == 8 || Ns == 16 || Ns == 32; }

// thread -> (site of the tile, s-slice) in the hop phase.  FP32-arithmetic kernels with Ns a
// multiple of 8 give each quarter-warp eight consecutive slices of one site, so a warp holds
// four sites.  An LDS.128 costs one wavefront per half-warp even when every lane reads the
// same address (measured on GB300), so the broadcast link reads are shared by four sites per
// two wavefronts instead of two; each site's gathers stay whole 128-byte lines (eight
// slices x 16 bytes).  Otherwise thread = s + Ns * site, the Ns slices of a site adjacent.
template <bool F2>
__device__ __forceinline__ void hop_thread(int tid, int Ns, int spb, int &sl, int &s) {
  if (F2 && (Ns & 7) == 0) {
    const int g = tid >> 3;
    sl = g % spb;
    s = ((g / spb) << 3) | (tid & 7);
  } else {
    sl = tid / Ns;
    s = tid - sl * Ns;
  }
}
// kernels without an M5 epilogue run persistent CTAs (measured: hop_xpay 96 -> 79 us); the
// M5 kernels keep one tile per CTA and the smaller footprint (a double-buffered persistent
// form took hop_m5 93 -> 104 us and hop_update 158 -> 188 us by shrinking the L1)
template <int EPI> constexpr bool hop_persistent() { return !EpiT<EPI>::has_m; }
template <int P, int EPI>
__host__ __device__ inline size_t hop_smem_bytes(int spb, int Ns) {
  return HopSmem<P>::bytes(spb, Ns, hop_persistent<EPI>() ? 2 : 1, EpiT<EPI>::has_m);
}

// k_hop: one thread per (site, s), CTA = (Ns, spb) = one tile of spb sites (kernels without
// an M5 epilogue: a grid of as many CTAs as fit on the GPU at once, walking all tiles).  Per
// tile: eight gathers of the neighbours' spinors (Eq. 12), the hop sum in packed FP32 pairs
// (or FP64), the epilogue.
template <int P, int EPI, int NSC>
__global__ void __launch_bounds__(256) k_hop(const HopArgs a) {
  // one right-hand side of a batch per grid row; fields are offset where they are used, so
  // the pointers stay in parameter space instead of registers
  const int rb = blockIdx.y;
  auto F = [&](const Field &f) { return rb ? field_rhs(f, rb, a.fstride, a.nstride) : f; };
  CGScalars *const sc_ = a.sc + rb;
  using T = PT<P>;
  using R = typename T::real;
  using E = EpiT<EPI>;
  using SM = HopSmem<P>;
  constexpr bool F2 = SM::F2;
  extern __shared__ __align__(128) unsigned char sm[];
  const int Ns = NSC ? NSC : a.Ns;
  const int spb = blockDim.y;
  const int tid = lin_tid();
  const int nthr = nthreads();
  int sl, s;  // this thread's site of the tile and s-slice in the hop phase
  hop_thread<F2>(tid, Ns, spb, sl, s);
  const long ntile = (a.h + spb - 1) / spb;

  if (a.use_flag && sc_->restart_flag) return;  // uniform over the grid

  constexpr bool PST = hop_persistent<EPI>();
  constexpr int NB = PST ? 2 : 1;  // link / neighbour buffers
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);  // bar[b]: buffer b's copies landed
  float4 *sP = reinterpret_cast<float4 *>(sm + SM::off_exp(spb, NB));
  unsigned char *sS = sm + 64;
  unsigned char *sKb = sm + SM::off_k(spb, Ns, NB, E::has_m);
  auto sLb = [&](int b) { return reinterpret_cast<typename T::lreal *>(sm + SM::off_raw(spb, b)); };
  auto sNb = [&](int b) { return reinterpret_cast<int *>(sm + SM::off_nbr(spb, NB, b)); };

  // tile t's links and neighbour indices arrive in buffer b with two TMA bulk copies (both
  // contiguous and 16-byte sized); its epilogue operands are prefetched into L2 when the
  // tile starts
  auto issue = [&](long t, int b) {
    const long c0 = t * spb;
    const int ns_t = (int)min((long)spb, a.h - c0);
    const uint32_t lbytes = (uint32_t)SM::raw(ns_t), nbytes = (uint32_t)ns_t * 8 * 4;
    mbar_expect_tx(bar + b, lbytes + nbytes);
    bulk_g2s(sLb(b), static_cast<const typename T::lreal *>(a.gauge) + (size_t)c0 * T::SITE_LREALS, lbytes, bar + b);
    bulk_g2s(sNb(b), a.nbr + c0 * 8, nbytes, bar + b);
  };
  auto prefetch_ops = [&](long t) {
    const long c0 = t * spb;
    const int ns_t = (int)min((long)spb, a.h - c0);
    const uint32_t ob = (uint32_t)((size_t)ns_t * T::NCH * Ns * 16);
    const size_t off = (size_t)c0 * T::NCH * Ns * 16;
    if constexpr (EPI == E_XPAY_G5 || EPI == E_XPAY || EPI == E_M_XPAY || EPI == E_CG_UPDATE || EPI == E_RESID)
      prefetch_l2(static_cast<const unsigned char *>(F(a.y).v) + off, ob);
    if constexpr (EPI == E_CG_UPDATE) prefetch_l2(static_cast<const unsigned char *>(F(a.r).v) + off, ob);
    if constexpr (EPI == E_RESID) prefetch_l2(static_cast<const unsigned char *>(F(a.b).v) + off, ob);
  };

  if (tid == 0) {
    mbar_init(bar, 1);
    if constexpr (PST) mbar_init(bar + 1, 1);
  }
  if constexpr (E::has_m) {
    if constexpr (F2) {
      const float *Kg = static_cast<const float *>(a.K);  // K[chi][t][s]
      float2 *sK2 = reinterpret_cast<float2 *>(sKb);
      if (m5_quad(Ns)) {
        // per chirality, t-pair and b: (K[b][t], K[b + Ns/2][t], K[b][t + 1], K[b + Ns/2][t + 1])
        const int half = Ns >> 1;
        float4 *sK4 = reinterpret_cast<float4 *>(sKb);
        for (int i = tid; i < Ns * Ns / 2; i += nthr) {
          const int chi = i / (half * half), rem = i - chi * half * half;
          const int tp = rem / half, b = rem - tp * half;
          const float *c0 = Kg + ((size_t)chi * Ns + 2 * tp) * Ns, *c1 = c0 + Ns;
          const float cf = (float)a.coef;
          sK4[i] = make_float4(cf * c0[b], cf * c0[b + half], cf * c1[b], cf * c1[b + half]);
        }
      } else if ((Ns & 1) == 0) {
        const int half = Ns >> 1, kst = SM::kq_stride(Ns);
        for (int i = tid; i < Ns * Ns; i += nthr) {
          const int chi = i / (Ns * half), rem = i - chi * Ns * half;
          const int t = rem / half, b = rem - t * half;
          const float *col = Kg + ((size_t)chi * Ns + t) * Ns;
          sK2[chi * kst + t * half + b] = make_float2((float)a.coef * col[b], (float)a.coef * col[b + half]);
        }
      } else {
        for (int i = tid; i < 2 * Ns * Ns; i += nthr) {
          const float k = (float)a.coef * Kg[i];
          sK2[i] = make_float2(k, k);
        }
      }
    } else {
      // the matrix acts on coef H: coef scales g and the closure (entries PS, PN, W)
      const R *Tg = static_cast<const R *>(a.rec);
      R *sT = reinterpret_cast<R *>(sKb);
      for (int i = tid; i < 2 * Ns * 8; i += nthr) {
        const int e = i & 7;
        sT[i] = (e == 0 || e == 1 || e == 6) ? (R)(a.coef * (double)Tg[i]) : Tg[i];
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (!a.skip_copies) issue(blockIdx.x, 0);
    prefetch_ops(blockIdx.x);
  }

  // tiles blockIdx.x, blockIdx.x + gridDim.x, ... in this order, so that the CTA's share of
  // a reduction is summed in a fixed order (one tile per CTA unless persistent)
  R part = 0;
  int it = 0;
  for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x, ++it) {
    const int bsel = PST ? (it & 1) : 0;
    const uint32_t par = PST ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
    const long cb0 = tile * spb;
    const int nsite = (int)min((long)spb, a.h - cb0);
    const bool active = sl < nsite;
    const long cb = cb0 + sl;
    const typename T::lreal *sL = sLb(bsel);
    const int *sN = sNb(bsel);
    if constexpr (!PST) {
      if (it > 0) {  // one buffer: the previous tile must be finished before it is refilled
        __syncthreads();
        if (tid == 0) {
          if (!a.skip_copies) issue(tile, 0);
          prefetch_ops(tile);
        }
      }
    }
    // bounded wait, outcome agreed by the whole CTA before anyone acts on it; the barrier
    // also ends every thread's use of the previous tile's buffers and staging rows
    {
      const bool ok = mbar_wait(bar + bsel, par, a.wait_tries);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(&sc_->error, ERR_TMA_TIMEOUT);
        mbar_wait(bar + bsel, par, a.wait_tries);  // the copy in flight
        return;
      }
    }
    if constexpr (PST) {
      // the other buffer held the previous tile, consumed before the barrier above
      if (tid == 0) {
        if (tile + gridDim.x < ntile && !a.skip_copies) issue(tile + gridDim.x, bsel ^ 1);
        if (it > 0) prefetch_ops(tile);
      }
    }
    if constexpr (SM::EXPAND) {
      // 16-bit links: rebuild row 3 and expand each link into the padded FP32 form
      for (int l = tid; l < nsite * 8; l += nthr) {
        float W[18];
        load_link<P>(sL + (size_t)l * T::LREALS, W);
        float4 *o = sP + (size_t)(l >> 3) * LINK_SITE_F4 + (l & 7) * 5;
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = make_float4(W[4 * e], W[4 * e + 1], W[4 * e + 2], W[4 * e + 3]);
        o[4] = make_float4(W[16], W[17], 0.f, 0.f);
      }
      __syncthreads();
    }

    R acc[24];
    bool chunk_done = false;  // the M5 epilogue already stored this tile's results
    if (active) {
      const int *nb = sN + sl * 8;
      if constexpr (F2) {
        f2 ac2[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) ac2[q] = pk2(0.f, 0.f);
        const SignPairs fw = sign_pairs(-1.f), bw = sign_pairs(1.f);
        const float4 *myW =
            (SM::EXPAND ? sP : reinterpret_cast<const float4 *>(sL)) + (size_t)sl * LINK_SITE_F4;
        // the forward and backward hops of one direction in turn: both gather from the same
        // rows of the input for mu = x, so the second finds most of its lines in L1
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
          const int d = (dd >> 1) + 4 * (dd & 1);
          float ps1[24];
          load_sp_ro<P>(F(a.in), nb[d], s, Ns, ps1);
          f2 ps[12];
#pragma unroll
          for (int q = 0; q < 12; ++q) ps[q] = pk2(ps1[2 * q], ps1[2 * q + 1]);
          switch (d) {  // forward hops (1 - g_mu), then backward hops (1 + g_mu)
            case 0: hop_dir_raw<0>(ac2, ps, myW, fw); break;
            case 1: hop_dir_raw<1>(ac2, ps, myW + 5, fw); break;
            case 2: hop_dir_raw<2>(ac2, ps, myW + 10, fw); break;
            case 3: hop_dir_raw<3>(ac2, ps, myW + 15, fw); break;
            case 4: hop_dir_raw<0>(ac2, ps, myW + 20, bw); break;
            case 5: hop_dir_raw<1>(ac2, ps, myW + 25, bw); break;
            case 6: hop_dir_raw<2>(ac2, ps, myW + 30, bw); break;
            default: hop_dir_raw<3>(ac2, ps, myW + 35, bw); break;
          }
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) upk2(ac2[q], acc[2 * q], acc[2 * q + 1]);
      } else {
#pragma unroll
        for (int c = 0; c < 24; ++c) acc[c] = 0;
        const typename T::lreal *myL = sL + (size_t)sl * T::SITE_LREALS;
        R ps[24], W[18];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          load_sp_ro<P>(F(a.in), nb[d], s, Ns, ps);
          load_link<P>(myL + d * T::LREALS, W);
          const R S = d < 4 ? (R)-1 : (R)1;
          switch (d & 3) {
            case 0: hop_dir_s<0>(acc, ps, W, S); break;
            case 1: hop_dir_s<1>(acc, ps, W, S); break;
            case 2: hop_dir_s<2>(acc, ps, W, S); break;
            default: hop_dir_s<3>(acc, ps, W, S); break;
          }
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 24; ++c) acc[c] = 0;
    }

    if constexpr (E::has_m) {
      // M5-type epilogue (Sec. 3.3): out_s = sum_t (M5)_{st} H_t per chirality; the Ns
      // slices of a site are in this CTA, staged through shared memory (rows and sites padded
      // by 16 bytes against bank conflicts; the stage overlays the link buffers)
      R *sB = reinterpret_cast<R *>(sS);
      constexpr int ROW = SM::ROW;
      const int sstride = Ns * ROW + 16 / (int)sizeof(R);
      R *mine = sB + (size_t)sl * sstride + (size_t)s * ROW;
      __syncthreads();  // every warp is done with the links the stage overwrites
#pragma unroll
      for (int c = 0; c < 24; ++c) mine[c] = acc[c];
      __syncthreads();
      if constexpr (F2) {
        if ((Ns & 1) == 0) {
          // FP32 arithmetic, even Ns: thread = (site, chirality, slice pair (b, b + Ns/2)),
          // forming 12 outputs (one chirality) of two slices from the site's staged rows:
          // each row piece read serves two slices, and a half-warp reads the pieces of at
          // most two (site, chirality) pairs (one shared-memory wavefront per half-warp)
          const int half = Ns >> 1;
          const bool quad = m5_quad(Ns);
          int sl2, chi, bq;
          if (quad) {
            // Ns divides 32: each half-warp one chirality of 32/Ns sites (lanes chi, site, b),
            // so the K entries a half-warp reads are one 16-byte row per b, for two t at once
            const int lane = tid & 31, rest = lane & 15;
            chi = lane >> 4;
            bq = rest % half;
            sl2 = (tid >> 5) * (32 / Ns) + rest / half;
          } else {
            sl2 = tid / Ns;
            const int r2 = tid - sl2 * Ns;
            chi = r2 >= half ? 1 : 0;
            bq = r2 - chi * half;
          }
          const bool act2 = sl2 < nsite;
          f2 o1[6], o2[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) o1[q] = o2[q] = pk2(0.f, 0.f);
          // o1 += K[b][t] H_t, o2 += K[b + Ns/2][t] H_t on this chirality's 12 reals
          auto step = [&](const R *row, float k1s, float k2s) {
            const f2 k1 = pk2(k1s, k1s), k2 = pk2(k2s, k2s);
            const float4 *v4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float4 v = v4[k];
              const f2 lo = pk2(v.x, v.y), hi = pk2(v.z, v.w);
              o1[2 * k] = fma2(k1, lo, o1[2 * k]);
              o1[2 * k + 1] = fma2(k1, hi, o1[2 * k + 1]);
              o2[2 * k] = fma2(k2, lo, o2[2 * k]);
              o2[2 * k + 1] = fma2(k2, hi, o2[2 * k + 1]);
            }
          };
          if (act2) {
            const R *site = sB + (size_t)sl2 * sstride + 12 * chi;
            if (quad) {
              const float4 *kq = reinterpret_cast<const float4 *>(sKb) + chi * (half * half) + bq;
#pragma unroll 2
              for (int tp = 0; tp < half; ++tp) {
                const float4 kk = kq[tp * half];
                step(site + (2 * tp) * ROW, kk.x, kk.y);
                step(site + (2 * tp + 1) * ROW, kk.z, kk.w);
              }
            } else {
              const float2 *kq = reinterpret_cast<const float2 *>(sKb) + chi * SM::kq_stride(Ns) + bq;
#pragma unroll 4
              for (int t = 0; t < Ns; ++t) {
                const float2 kk = kq[t * half];  // (K[b][t], K[b + Ns/2][t])
                step(site + t * ROW, kk.x, kk.y);
              }
            }
          }
          if constexpr (!T::HALF) {
            // FP32 storage: the epilogue works on this thread's six 16-byte chunks
            // (chunks 3 chi .. 3 chi + 2 of slices b and b + Ns/2); for each chunk the
            // threads of a (site, chirality) cover Ns/2 consecutive slices
            chunk_done = true;
            if (act2) {
              const long cb2 = cb0 + sl2;
              R alpha = 0;
              if constexpr (EPI == E_CG_UPDATE) alpha = sc_->alpha_f;
              auto emit = [&](int sv, const f2 (&o)[6]) {
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                  const int k = 3 * chi + kk;
                  R v[4];
                  upk2(o[2 * kk], v[0], v[1]);
                  upk2(o[2 * kk + 1], v[2], v[3]);
                  if constexpr (EPI == E_M) {
                    store_chunk<P>(F(a.out), cb2, sv, Ns, k, v);
                  } else if constexpr (EPI == E_M_XPAY) {
                    R y[4];
                    load_chunk<P>(F(a.y), cb2, sv, Ns, k, y);
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[j] += y[j];
                    store_chunk<P>(F(a.out), cb2, sv, Ns, k, v);
                  } else if constexpr (EPI == E_CG_UPDATE) {
                    // Ap = y + K H; r -= alpha Ap (alpha formed with (p, A p))
                    R y[4], r[4];
                    load_chunk<P>(F(a.y), cb2, sv, Ns, k, y);
                    load_chunk<P>(F(a.r), cb2, sv, Ns, k, r);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                      r[j] -= alpha * (y[j] + v[j]);
                      part += r[j] * r[j];
                    }
                    store_chunk<P>(F(a.r), cb2, sv, Ns, k, r);
                  } else if constexpr (EPI == E_RESID) {
                    R y[4], bb[4];
                    load_chunk<P>(F(a.y), cb2, sv, Ns, k, y);
                    load_chunk<P>(F(a.b), cb2, sv, Ns, k, bb);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                      bb[j] -= y[j] + v[j];
                      part += bb[j] * bb[j];
                    }
                    store_chunk<P>(F(a.out), cb2, sv, Ns, k, bb);
                  }
                }
              };
              emit(bq, o1);
              emit(bq + half, o2);
            }
          } else {
            // 16-bit storage normalises each (site, s) row as a whole: the results go back
            // into the stage and the per-(site, s) epilogue below stores them
            __syncthreads();  // every thread is done reading the staged rows
            if (act2) {
              float4 *w1 = reinterpret_cast<float4 *>(sB + (size_t)sl2 * sstride + (size_t)bq * ROW + 12 * chi);
              float4 *w2 = reinterpret_cast<float4 *>(sB + (size_t)sl2 * sstride + (size_t)(bq + half) * ROW + 12 * chi);
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                float x0, x1, x2, x3;
                upk2(o1[2 * k], x0, x1);
                upk2(o1[2 * k + 1], x2, x3);
                w1[k] = make_float4(x0, x1, x2, x3);
                upk2(o2[2 * k], x0, x1);
                upk2(o2[2 * k + 1], x2, x3);
                w2[k] = make_float4(x0, x1, x2, x3);
              }
            }
            __syncthreads();
            if (active) {
#pragma unroll
              for (int c = 0; c < 24; ++c) acc[c] = mine[c];
            }
          }
        } else if (active) {
          // odd Ns: dense, every (site, s) thread forms its own output row from the site's
          // Ns staged rows
          const R *site = sB + (size_t)sl * sstride;
          const f2 *sK2 = reinterpret_cast<const f2 *>(sKb);
          f2 o[12];
#pragma unroll
          for (int q = 0; q < 12; ++q) o[q] = pk2(0.f, 0.f);
#pragma unroll 4
          for (int t = 0; t < Ns; ++t) {
            const f2 kp = sK2[t * Ns + s];            // (K+[s][t], K+[s][t])
            const f2 km = sK2[Ns * Ns + t * Ns + s];  // (K-[s][t], K-[s][t])
            const float4 *v4 = reinterpret_cast<const float4 *>(site + t * ROW);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              const float4 v = v4[k];
              const f2 kk = k < 3 ? kp : km;
              o[2 * k] = fma2(kk, pk2(v.x, v.y), o[2 * k]);
              o[2 * k + 1] = fma2(kk, pk2(v.z, v.w), o[2 * k + 1]);
            }
          }
#pragma unroll
          for (int q = 0; q < 12; ++q) upk2(o[q], acc[2 * q], acc[2 * q + 1]);
        }
      } else {
        // FP64: M5 (or M5^T) along s, Eq. 8, as a recurrence, which halves the FP64
        // operations that limit these kernels: one 16-byte column (two reals of one
        // chirality) of one site per item; a closure sweep, then the sweep that overwrites
        // the column with the result (the item owns its column)
        {
          constexpr int CW = 2, NCK = 12;
          using V = double2;
          const R kap = (R)a.kappa;
          const R *sT = reinterpret_cast<const R *>(sKb);
          for (int item = tid; item < nsite * NCK; item += nthr) {
            const int l = item / NCK, k = item - l * NCK;
            const int chi = k >= NCK / 2 ? 1 : 0;
            const bool bwd = (chi ^ a.mtrans) != 0;
            const R *Tc = sT + chi * Ns * 8;
            R *col = sB + (size_t)l * sstride + k * CW;
            R zc[CW], vl[CW];
#pragma unroll
            for (int q = 0; q < CW; ++q) zc[q] = 0;
#pragma unroll 4
            for (int j = 0; j < Ns; ++j) {
              const int sj = bwd ? Ns - 1 - j : j;
              const V w4 = *reinterpret_cast<const V *>(col + sj * ROW);
              const R *v = reinterpret_cast<const R *>(&w4);
              const R w = Tc[j * 8 + 6];
#pragma unroll
              for (int q = 0; q < CW; ++q) {
                zc[q] += w * v[q];
                vl[q] = v[q];
              }
            }
            R zp[CW], vp[CW];
#pragma unroll
            for (int q = 0; q < CW; ++q) {
              zp[q] = kap * zc[q];
              vp[q] = kap * vl[q];
            }
#pragma unroll 4
            for (int j = 0; j < Ns; ++j) {
              const int sj = bwd ? Ns - 1 - j : j;
              R t[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) t[e] = Tc[j * 8 + e];
              V *cp = reinterpret_cast<V *>(col + sj * ROW);
              const V w4 = *cp;
              const R *v = reinterpret_cast<const R *>(&w4);
              V o4;
              R *o = reinterpret_cast<R *>(&o4);
#pragma unroll
              for (int q = 0; q < CW; ++q) {
                const R g = t[0] * v[q] + t[1] * vp[q];
                const R z = (g - t[2] * zp[q]) * t[3];
                o[q] = t[4] * z + t[5] * zp[q];
                zp[q] = z;
                vp[q] = v[q];
              }
              *cp = o4;
            }
          }
        }
        __syncthreads();
        if (active) {
          const R *row = sB + (size_t)sl * sstride + (size_t)s * ROW;
#pragma unroll
          for (int c = 0; c < 24; ++c) acc[c] = row[c];
        }
      }
    }
    if (active && !chunk_done) {
      if constexpr (EPI == E_PLAIN) {
#pragma unroll
        for (int c = 0; c < 24; ++c) acc[c] *= (R)a.coef;
        store_sp<P>(F(a.out), cb, s, Ns, acc);
      } else if constexpr (EPI == E_M) {
        store_sp<P>(F(a.out), cb, s, Ns, acc);
      } else if constexpr (EPI == E_XPAY_G5 || EPI == E_XPAY) {
        R y[24];
        load_sp<P>(F(a.y), cb, s, Ns, y);
        const R cf = (R)a.coef;
#pragma unroll
        for (int c = 0; c < 24; ++c) {
          const R g = (EPI == E_XPAY_G5 && c >= 12) ? -cf : cf;
          y[c] += g * acc[c];
          part += y[c] * y[c];
        }
        store_sp<P>(F(a.out), cb, s, Ns, y);
      } else if constexpr (EPI == E_M_XPAY) {
        R y[24];
        load_sp<P>(F(a.y), cb, s, Ns, y);
#pragma unroll
        for (int c = 0; c < 24; ++c) y[c] += acc[c];
        store_sp<P>(F(a.out), cb, s, Ns, y);
      } else if constexpr (EPI == E_CG_UPDATE) {
        // alpha = (r, r) / (p, A p) was formed once by the reduction that produced (p, A p)
        R alpha;
        if constexpr (P == P_F64) alpha = sc_->alpha;
        else alpha = sc_->alpha_f;
        // (x += alpha p is deferred to the next iteration's p-update, which reads p anyway)
        if constexpr (!T::HALF) {
          // chunk by chunk: two operands of 16 bytes live at a time, not 2 x 24 reals
          constexpr int RPC = T::RPC;
#pragma unroll
          for (int k = 0; k < T::NCH; ++k) {
            R y[RPC], r[RPC];
            load_chunk<P>(F(a.y), cb, s, Ns, k, y);
            load_chunk<P>(F(a.r), cb, s, Ns, k, r);
#pragma unroll
            for (int j = 0; j < RPC; ++j) {
              r[j] -= alpha * (y[j] + acc[k * RPC + j]);
              part += r[j] * r[j];
            }
            store_chunk<P>(F(a.r), cb, s, Ns, k, r);
          }
        } else {
          R y[24], r[24];
          load_sp<P>(F(a.y), cb, s, Ns, y);
          load_sp<P>(F(a.r), cb, s, Ns, r);
#pragma unroll
          for (int c = 0; c < 24; ++c) {
            r[c] -= alpha * (y[c] + acc[c]);
            part += r[c] * r[c];
          }
          store_sp<P>(F(a.r), cb, s, Ns, r);
        }
      } else if constexpr (EPI == E_RESID) {
        R y[24], bb[24];
        load_sp<P>(F(a.y), cb, s, Ns, y);
        load_sp<P>(F(a.b), cb, s, Ns, bb);
#pragma unroll
        for (int c = 0; c < 24; ++c) {
          bb[c] -= y[c] + acc[c];
          part += bb[c] * bb[c];
        }
        store_sp<P>(F(a.out), cb, s, Ns, bb);
      }
    }
  }
  if constexpr (E::has_red) grid_sum<R>(part, a.partials + rb * a.part_stride, a.ticket + rb, a.fin, sc_);
}

// ------------------------------------------------------------------ s-mixing kernel

enum {
  S_PLAIN = 0,  // out = K in
  S_G5 = 1,     // out = K g5 in
  S_CGP = 2,    // x += alpha p, then p = r + beta p (both stored); out = K g5 p
  S_DUAL = 3    // out = K in; out2 = K2 in
};

struct SmixArgs {
  Field in, out, out2, r, p, x;
  const void *K, *K2;  // K[chi][t][s]
  double coef;
  long h;
  int Ns;
  int use_flag;
  CGScalars *sc;
  int nrhs;               // batches of right-hand sides as in HopArgs
  size_t fstride, nstride;
  size_t xfstride;        // bytes between the rows' x (FP32 when the inner fields are 16-bit)
};

// the inner CG's solution increment x is accumulated in FP32 when the other inner fields
// are 16-bit: x is never gathered by a hop, and 16-bit rounding of x over a cycle of inner
// iterations would leave the true residual far above the iterated one
template <int P> constexpr int x_prec() { return PT<P>::HALF ? P_F32 : P; }

template <int P>
__host__ __device__ inline size_t smix_smem_bytes(int spb, int Ns, bool dual) {
  size_t b = (size_t)(dual ? 4 : 2) * Ns * Ns * sizeof(typename PT<P>::real);
  b = (b + 15) & ~size_t(15);
  return b + (size_t)spb * Ns * 24 * sizeof(typename PT<P>::real);
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) k_smix(const SmixArgs a) {
  const int rb = blockIdx.y;  // one right-hand side of a batch per grid row
  auto F = [&](const Field &f) { return rb ? field_rhs(f, rb, a.fstride, a.nstride) : f; };
  CGScalars *const sc_ = a.sc + rb;
  using R = typename PT<P>::real;
  extern __shared__ __align__(128) unsigned char sm[];
  const int Ns = a.Ns;
  const int s = threadIdx.x, sl = threadIdx.y, spb = blockDim.y;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const long cb = (long)blockIdx.x * spb + sl;
  const bool active = cb < a.h;
  if (a.use_flag && sc_->restart_flag) return;
  constexpr bool dual = MODE == S_DUAL;
  R *sK = reinterpret_cast<R *>(sm);
  R *sB = reinterpret_cast<R *>(sm + ((((size_t)(dual ? 4 : 2) * Ns * Ns * sizeof(R)) + 15) & ~size_t(15)));
  {
    const R *Kg = static_cast<const R *>(a.K);
    for (int i = tid; i < 2 * Ns * Ns; i += nthr) sK[i] = (R)a.coef * Kg[i];
    if constexpr (dual) {
      const R *K2 = static_cast<const R *>(a.K2);
      for (int i = tid; i < 2 * Ns * Ns; i += nthr) sK[2 * Ns * Ns + i] = (R)a.coef * K2[i];
    }
  }
  R v[24];
  if (active) {
    if constexpr (MODE == S_CGP) {
      // Algorithm 1: the previous iteration's x += alpha p (alpha is still that iteration's;
      // 0 after a restart, which adds the pending step itself), then p = r + beta p
      R beta, alpha;
      if constexpr (P == P_F64) {
        beta = sc_->beta;
        alpha = sc_->alpha;
      } else {
        beta = sc_->beta_f;
        alpha = sc_->alpha_f;
      }
      load_sp<P>(F(a.p), cb, s, Ns, v);
      {
        constexpr int PX = x_prec<P>();
        const Field fx = rb ? field_rhs(a.x, rb, a.xfstride, 0) : a.x;
        R xx[24];
        load_sp<PX>(fx, cb, s, Ns, xx);
#pragma unroll
        for (int c = 0; c < 24; ++c) xx[c] += alpha * v[c];
        store_sp<PX>(fx, cb, s, Ns, xx);
      }
      R r[24];
      load_sp<P>(F(a.r), cb, s, Ns, r);
#pragma unroll
      for (int c = 0; c < 24; ++c) v[c] = r[c] + beta * v[c];
      store_sp<P>(F(a.p), cb, s, Ns, v);
    } else {
      load_sp_ro<P>(F(a.in), cb, s, Ns, v);
    }
    if constexpr (MODE == S_CGP || MODE == S_G5) {
#pragma unroll
      for (int c = 12; c < 24; ++c) v[c] = -v[c];
    }
    R *mine = sB + ((size_t)sl * Ns + s) * 24;
#pragma unroll
    for (int c = 0; c < 24; ++c) mine[c] = v[c];
  }
  __syncthreads();
  if (!active) return;
  const R *site = sB + (size_t)sl * Ns * 24;
  for (int which = 0; which < (dual ? 2 : 1); ++which) {
    const R *K = sK + which * 2 * Ns * Ns;
    R o[24];
#pragma unroll
    for (int c = 0; c < 24; ++c) o[c] = 0;
    for (int t = 0; t < Ns; ++t) {
      const R kp = K[t * Ns + s], km = K[Ns * Ns + t * Ns + s];
      const R *vv = site + t * 24;
#pragma unroll
      for (int c = 0; c < 12; ++c) o[c] += kp * vv[c];
#pragma unroll
      for (int c = 12; c < 24; ++c) o[c] += km * vv[c];
    }
    store_sp<P>(which == 0 ? F(a.out) : F(a.out2), cb, s, Ns, o);
  }
}

// ------------------------------------------------------------------ per-(site, s) vector kernels

struct VecArgs {
  Field a, b, c;     // operands (meaning per kernel)
  long n;            // h * Ns
  int Ns;
  double coef;
  int fin;
  CGScalars *sc;
  double *partials;
  unsigned *ticket;
};

// |a|^2 -> fin (precision P)
template <int P>
__global__ void __launch_bounds__(256) k_norm2(const VecArgs v) {
  using R = typename PT<P>::real;
  double part = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += (long)gridDim.x * blockDim.x) {
    R x[24];
    load_sp_ro<P>(v.a, i / v.Ns, (int)(i % v.Ns), v.Ns, x);
    R pr = 0;
#pragma unroll
    for (int c = 0; c < 24; ++c) pr += x[c] * x[c];
    part += (double)pr;
  }
  grid_sum(part, v.partials, v.ticket, v.fin, v.sc);
}

// b (precision PB) = a (precision PA), element-wise with the layout conversion
template <int PA, int PB>
__global__ void __launch_bounds__(256) k_convert(const VecArgs v) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += (long)gridDim.x * blockDim.x) {
    const long cb = i / v.Ns;
    const int s = (int)(i % v.Ns);
    typename PT<PA>::real x[24];
    load_sp_ro<PA>(v.a, cb, s, v.Ns, x);
    typename PT<PB>::real y[24];
#pragma unroll
    for (int c = 0; c < 24; ++c) y[c] = (typename PT<PB>::real)x[c];
    store_sp<PB>(v.b, cb, s, v.Ns, y);
  }
}

// FP64 a += (precision P) (b + alpha c); b = 0  (x_hat += x at a restart, Algorithm 2, with
// the CG step x += alpha p of the last inner iteration, deferred to a p-update that did not
// run, added first; c may be absent)
template <int P>
__global__ void __launch_bounds__(256) k_accum(const VecArgs v) {
  using R = typename PT<P>::real;
  R alpha = 0;
  if (v.c.v) {
    if constexpr (P == P_F64) alpha = v.sc->alpha;
    else alpha = v.sc->alpha_f;
  }
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += (long)gridDim.x * blockDim.x) {
    const long cb = i / v.Ns;
    const int s = (int)(i % v.Ns);
    constexpr int PX = x_prec<P>();  // x in FP32 when the inner fields are 16-bit
    double xa[24];
    R xb[24];
    load_sp<P_F64>(v.a, cb, s, v.Ns, xa);
    load_sp<PX>(v.b, cb, s, v.Ns, xb);
    if (v.c.v) {
      R pc[24];
      load_sp<P>(v.c, cb, s, v.Ns, pc);
#pragma unroll
      for (int c = 0; c < 24; ++c) xb[c] += alpha * pc[c];
    }
#pragma unroll
    for (int c = 0; c < 24; ++c) { xa[c] += (double)xb[c]; xb[c] = 0; }
    store_sp<P_F64>(v.a, cb, s, v.Ns, xa);
    store_sp<PX>(v.b, cb, s, v.Ns, xb);
  }
}

// ------------------------------------------------------------------ layout conversion (Sec. 3.1)

struct Geom {
  int d[4];     // Nx, Ny, Nz, Nt
  long h;       // V4 / 2
  int Ns;
};

// y = a + sb b on full-lattice host-layout arrays (24 reals per (site, s)), on the sites of
// parity `keep` (every site if keep < 0; the others are set to 0); b may be null (0).
// |y|^2 -> fin.
struct HostAxpyArgs {
  double *y;
  const double *a, *b;
  double sb;
  Geom g;
  int keep;
  int fin;
  CGScalars *sc;
  double *partials;
  unsigned *ticket;
};

// lexicographic site of checkerboard index cb in parity p
__device__ __forceinline__ long cb_to_site(const Geom &g, long cb, int p, int (&c)[4]) {
  const int hx = g.d[0] >> 1;
  long r = cb;
  const int xh = (int)(r % hx); r /= hx;
  c[1] = (int)(r % g.d[1]); r /= g.d[1];
  c[2] = (int)(r % g.d[2]); r /= g.d[2];
  c[3] = (int)r;
  c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
  return c[0] + (long)g.d[0] * (c[1] + (long)g.d[1] * (c[2] + (long)g.d[2] * c[3]));
}

// device copy of the host layout (FP64, full lattice) -> parity p in precision P
template <int P>
__global__ void __launch_bounds__(256) k_pack(const double *host, Field out, Geom g, int p) {
  const long n = g.h * g.Ns;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long cb = i / g.Ns;
    const int s = (int)(i % g.Ns);
    int c[4];
    const long site = cb_to_site(g, cb, p, c);
    const double2 *src = reinterpret_cast<const double2 *>(host + ((size_t)site * g.Ns + s) * 24);
    typename PT<P>::real v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 t = __ldg(src + k);
      v[2 * k] = (typename PT<P>::real)t.x;
      v[2 * k + 1] = (typename PT<P>::real)t.y;
    }
    store_sp<P>(out, cb, s, g.Ns, v);
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_unpack(Field in, double *host, Geom g, int p) {
  const long n = g.h * g.Ns;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long cb = i / g.Ns;
    const int s = (int)(i % g.Ns);
    int c[4];
    const long site = cb_to_site(g, cb, p, c);
    typename PT<P>::real v[24];
    load_sp_ro<P>(in, cb, s, g.Ns, v);
    double2 *dst = reinterpret_cast<double2 *>(host + ((size_t)site * g.Ns + s) * 24);
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
  }
}

// doubled gauge field of output parity p from the FP64 host layout
template <int P>
__global__ void k_gauge(const double *U, typename PT<P>::lreal *G, Geom g, int p) {
  using L = typename PT<P>::lreal;
  constexpr int LR = PT<P>::LREALS;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < g.h * 8; i += (long)gridDim.x * blockDim.x) {
    const long cb = i >> 3;
    const int dir = (int)(i & 7);
    const int mu = dir & 3;
    int c[4];
    long site = cb_to_site(g, cb, p, c);
    bool dag = false;
    if (dir >= 4) {
      c[mu] = (c[mu] + g.d[mu] - 1) % g.d[mu];
      site = c[0] + (long)g.d[0] * (c[1] + (long)g.d[1] * (c[2] + (long)g.d[2] * c[3]));
      dag = true;
    }
    const double *u = U + ((size_t)site * 4 + mu) * 18;
    L *o = G + (size_t)cb * PT<P>::SITE_LREALS + dir * LR;
    for (int e = 18; e < LR; ++e) o[e] = L(0.f);  // padding of the FP32 form
    if (dir == 7)                                 // and of the site's block of links
      for (int e = 8 * LR; e < PT<P>::SITE_LREALS; ++e) G[(size_t)cb * PT<P>::SITE_LREALS + e] = L(0.f);
    for (int a = 0; a < 3 && a * 6 < LR; ++a)
      for (int b = 0; b < 3; ++b) {
        double re = dag ? u[2 * (3 * b + a)] : u[2 * (3 * a + b)];
        double im = dag ? -u[2 * (3 * b + a) + 1] : u[2 * (3 * a + b) + 1];
        if constexpr (P == P_F64) { o[2 * (3 * a + b)] = re; o[2 * (3 * a + b) + 1] = im; }
        else if constexpr (P == P_F32) { o[2 * (3 * a + b)] = (float)re; o[2 * (3 * a + b) + 1] = (float)im; }
        else if constexpr (P == P_F16) { o[2 * (3 * a + b)] = __double2half(re); o[2 * (3 * a + b) + 1] = __double2half(im); }
        else { o[2 * (3 * a + b)] = __double2bfloat16(re); o[2 * (3 * a + b) + 1] = __double2bfloat16(im); }
      }
  }
}

#ifdef DWF_DEFINE_PLAIN_KERNELS  // non-template kernels: defined in one translation unit only

// |a - b|^2 (both FP64) -> fin
__global__ void __launch_bounds__(256) k_diff_norm2(const VecArgs v) {
  double part = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += (long)gridDim.x * blockDim.x) {
    double x[24], y[24];
    load_sp_ro<P_F64>(v.a, i / v.Ns, (int)(i % v.Ns), v.Ns, x);
    load_sp_ro<P_F64>(v.b, i / v.Ns, (int)(i % v.Ns), v.Ns, y);
    for (int c = 0; c < 24; ++c) part += (x[c] - y[c]) * (x[c] - y[c]);
  }
  grid_sum(part, v.partials, v.ticket, v.fin, v.sc);
}

__global__ void __launch_bounds__(256) k_host_axpy(const HostAxpyArgs v) {
  const long per_site = (long)v.g.Ns * 24;
  const long n = 2 * v.g.h * per_site;
  double part = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    long site = i / per_site;
    int par = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      par += (int)(site % v.g.d[mu]);
      site /= v.g.d[mu];
    }
    par = (par + (int)site) & 1;
    double y = 0.0;
    if (v.keep < 0 || par == v.keep) y = v.a[i] + (v.b ? v.sb * v.b[i] : 0.0);
    v.y[i] = y;
    part += y * y;
  }
  grid_sum(part, v.partials, v.ticket, v.fin, v.sc);
}

// neighbour table of output parity p: nbr[cb][dir]
__global__ void k_neighbours(int *nbr, Geom g, int p) {
  for (long cb = (long)blockIdx.x * blockDim.x + threadIdx.x; cb < g.h; cb += (long)gridDim.x * blockDim.x) {
    int c[4];
    cb_to_site(g, cb, p, c);
    for (int dir = 0; dir < 8; ++dir) {
      const int mu = dir & 3;
      int e[4] = {c[0], c[1], c[2], c[3]};
      e[mu] = (e[mu] + (dir < 4 ? 1 : g.d[mu] - 1)) % g.d[mu];
      const long site = e[0] + (long)g.d[0] * (e[1] + (long)g.d[1] * (e[2] + (long)g.d[2] * e[3]));
      nbr[cb * 8 + dir] = (int)(site >> 1);
    }
  }
}

// ------------------------------------------------------------------ propagators
//
// 12 point sources at site x0 (full-lattice host layout, one after another): source
// (beta, b) has a 1 in spin beta, colour b on the s-slice of its chirality's wall
// (P+ spins 0,1 on s = 0, P- spins 2,3 on s = Ns - 1).
__global__ void k_point_sources(double *rhs, long x0site, long V4, int Ns) {
  const int k = threadIdx.x;
  if (k >= 12) return;
  const int beta = k / 3, b = k % 3;
  const int s = beta < 2 ? 0 : Ns - 1;
  rhs[(size_t)k * V4 * Ns * 24 + (((size_t)x0site * Ns + s) * 12 + 3 * beta + b) * 2] = 1.0;
}

// 4D quark field q(x) = P- psi(x, s = 0) + P+ psi(x, s = Ns - 1) of the 12 solutions, as
// prop[site][alpha][a][beta][b] complex
__global__ void k_prop_extract(const double *sol, double *prop, long V4, int Ns) {
  const long n = V4 * 144;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long site = i / 144;
    const int r = (int)(i % 144), sink = r / 12, src = r % 12;
    const int alpha = sink / 3, a = sink % 3;
    const int s = alpha < 2 ? Ns - 1 : 0;
    const double2 v = *reinterpret_cast<const double2 *>(
        sol + (size_t)src * V4 * Ns * 24 + (((size_t)site * Ns + s) * 12 + 3 * alpha + a) * 2);
    reinterpret_cast<double2 *>(prop)[i] = v;
  }
}

#endif

}  // namespace dwf
