// dwf_device.cuh -- device code of the domain-wall solver for sm_103a.
//
// Data layout in HBM (one parity of the 4D lattice at a time; cb = checkerboard index of
// a site within its parity, cb = site / 2 with site = x + Nx (y + Ny (z + Nz t))):
//   spinor (Sec. 3.1 "Vector Index Conversion", re-derived for 16-byte loads):
//     chunk k of (cb, s) at element ((cb * NCH + k) * Ns + s) of 16-byte chunks, so the
//     Ns threads of one site read consecutive 16 bytes for every chunk;
//     F64: 12 chunks of double2, F32: 6 chunks of float4, F16/BF16: 3 chunks of 8
//     halves plus a per-(cb, s) FP32 norm at nrm[cb * Ns + s].
//     Inside a (cb, s) the 24 reals keep the host order c = reim + 2 (colour + 3 spin).
//   gauge, doubled per output parity: G[p][cb][dir][*] with dir 0..3 = U_mu(x) and
//     dir 4..7 = U_mu(x - mu)^dagger (stored daggered), 18 reals (F64/F32) or the first
//     two rows, 12 reals (F16/BF16; the third row is rebuilt as conj(row0 x row1)).
//   neighbours: nbr[p][cb][dir] = cb of x + mu (dir < 4) / x - mu (dir >= 4) in parity 1-p.
//
// The hopping term of Eq. 12 is evaluated as H = sum_mu [(1 - g_mu) U psi(x+mu) +
// (1 + g_mu) U^dag psi(x-mu)] with D = -H/2.  In the chiral basis g_mu = [[0, A],[A^dag, 0]]
// so (1 + S g_mu) psi = (h, S A^dag h) with h = psi_up + S A psi_dn: the link multiplies
// only the projected 2-spinor h (the spin-projection trick of Sec. 3.2) and the lower two
// spins are rebuilt from U h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwf {

enum { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

template <int P> struct PT;
// LREALS: reals per link; SITE_LREALS: reals per site's eight links, padding included
template <> struct PT<P_F64> {
  using real = double; using chunk = double2; using lreal = double;
  static constexpr int NCH = 12, RPC = 2, LREALS = 18, SITE_LREALS = 8 * 18; static constexpr bool HALF = false;
};
template <> struct PT<P_F32> {
  using real = float; using chunk = float4; using lreal = float;
  // links padded to 20 reals (80 bytes) so that the nine complex entries load as five float4;
  // a site's eight links padded by 16 bytes to 656 (41 float4), so that sites adjacent in a
  // half-warp read their broadcast link entries from different bank groups
  static constexpr int NCH = 6, RPC = 4, LREALS = 20, SITE_LREALS = 8 * 20 + 4; static constexpr bool HALF = false;
};
template <> struct PT<P_F16> {
  using real = float; using chunk = uint4; using lreal = __half;
  static constexpr int NCH = 3, RPC = 8, LREALS = 12, SITE_LREALS = 8 * 12; static constexpr bool HALF = true;
};
template <> struct PT<P_BF16> {
  using real = float; using chunk = uint4; using lreal = __nv_bfloat16;
  static constexpr int NCH = 3, RPC = 8, LREALS = 12, SITE_LREALS = 8 * 12; static constexpr bool HALF = true;
};
// float4 per site of the FP32 link form the hop reads (as stored, or expanded from 16 bits)
constexpr int LINK_SITE_F4 = 41;

struct Field {
  void *v;
  float *nrm;  // 16-bit precisions only
};

// scalars of one CG solve, resident in device memory (FP64 throughout)
struct CGScalars {
  double rr;       // |r|^2 of the current inner residual
  double rr_old;   // previous |r|^2 (denominator of beta)
  double qq;       // |C^dag p|^2 = (p, C C^dag p)
  double beta;     // p = r + beta p
  double rmax2;    // max |r|^2 since the last restart
  double delta2;   // reliable-update threshold squared
  double target2;  // (tol |b|)^2
  double red;      // result slot of plain norm reductions
  double red2;
  double alpha;     // (r, r) / (p, A p), set by the reduction that finishes |C^dag p|^2
  float alpha_f;    // the same in FP32 for the FP32-arithmetic kernels
  float beta_f;     // beta in FP32
  double rr_start;  // |r|^2 at the last restart (divergence guard)
  double rr_min;    // smallest |r|^2 since the last restart (stall guard)
  int restart_flag;  // set on device when an FP64 restart is due (a RS_* reason); kernels then skip work
  int iter;          // inner iterations done
  int iter_cap;      // restart when iter reaches this
  int error;         // kernel error word (bounded wait gave up)
  int iter_min;      // iteration at which rr_min was reached
  int stall_iters;   // restart when rr_min has not improved for this many iterations
};

// reasons for an FP64 restart
enum { RS_NONE = 0, RS_DELTA = 1, RS_TARGET = 2, RS_CAP = 3, RS_DIVERGED = 4, RS_STALLED = 5 };

// ------------------------------------------------------------------ spinor access

template <int P>
__device__ __forceinline__ void load_sp(const Field f, long cb, int s, int Ns,
                                        typename PT<P>::real (&o)[24]) {
  using T = PT<P>;
  const typename T::chunk *b = (const typename T::chunk *)f.v + (size_t)cb * T::NCH * Ns + s;
  if constexpr (P == P_F64) {
#pragma unroll
    for (int k = 0; k < 12; ++k) { double2 c = b[(size_t)k * Ns]; o[2 * k] = c.x; o[2 * k + 1] = c.y; }
  } else if constexpr (P == P_F32) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 c = b[(size_t)k * Ns];
      o[4 * k] = c.x; o[4 * k + 1] = c.y; o[4 * k + 2] = c.z; o[4 * k + 3] = c.w;
    }
  } else {
    const float nm = f.nrm[(size_t)cb * Ns + s];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c = b[(size_t)k * Ns];
      uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 v;
        if constexpr (P == P_F16) v = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
        else v = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w[j]));
        o[8 * k + 2 * j] = v.x * nm;
        o[8 * k + 2 * j + 1] = v.y * nm;
      }
    }
  }
}

// read-only variant for kernel inputs that no thread writes during the launch
template <int P>
__device__ __forceinline__ void load_sp_ro(const Field f, long cb, int s, int Ns,
                                           typename PT<P>::real (&o)[24]) {
  using T = PT<P>;
  const typename T::chunk *b = (const typename T::chunk *)f.v + (size_t)cb * T::NCH * Ns + s;
  if constexpr (P == P_F64) {
#pragma unroll
    for (int k = 0; k < 12; ++k) { double2 c = __ldg(b + (size_t)k * Ns); o[2 * k] = c.x; o[2 * k + 1] = c.y; }
  } else if constexpr (P == P_F32) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 c = __ldg(b + (size_t)k * Ns);
      o[4 * k] = c.x; o[4 * k + 1] = c.y; o[4 * k + 2] = c.z; o[4 * k + 3] = c.w;
    }
  } else {
    const float nm = __ldg(f.nrm + (size_t)cb * Ns + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c = __ldg(b + (size_t)k * Ns);
      uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 v;
        if constexpr (P == P_F16) v = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
        else v = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w[j]));
        o[8 * k + 2 * j] = v.x * nm;
        o[8 * k + 2 * j + 1] = v.y * nm;
      }
    }
  }
}

template <int P>
__device__ __forceinline__ void store_sp(Field f, long cb, int s, int Ns,
                                         const typename PT<P>::real (&v)[24]) {
  using T = PT<P>;
  typename T::chunk *b = (typename T::chunk *)f.v + (size_t)cb * T::NCH * Ns + s;
  if constexpr (P == P_F64) {
#pragma unroll
    for (int k = 0; k < 12; ++k) b[(size_t)k * Ns] = make_double2(v[2 * k], v[2 * k + 1]);
  } else if constexpr (P == P_F32) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
      b[(size_t)k * Ns] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < 24; ++c) mx = fmaxf(mx, fabsf(v[c]));
    const float sc = mx > 0.f ? 1.0f / mx : 0.f;
    f.nrm[(size_t)cb * Ns + s] = mx;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float a = v[8 * k + 2 * j] * sc, bb = v[8 * k + 2 * j + 1] * sc;
        if constexpr (P == P_F16) { __half2 h = __floats2half2_rn(a, bb); w[j] = *reinterpret_cast<uint32_t *>(&h); }
        else { __nv_bfloat162 h = __floats2bfloat162_rn(a, bb); w[j] = *reinterpret_cast<uint32_t *>(&h); }
      }
      b[(size_t)k * Ns] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// one 16-byte chunk k of (cb, s) (FP64: 2 reals, FP32: 4 reals); unnormalised precisions only
template <int P>
__device__ __forceinline__ void load_chunk(const Field f, long cb, int s, int Ns, int k,
                                           typename PT<P>::real (&o)[PT<P>::RPC]) {
  static_assert(!PT<P>::HALF, "chunk access needs an unnormalised precision");
  const typename PT<P>::chunk c = ((const typename PT<P>::chunk *)f.v)[((size_t)cb * PT<P>::NCH + k) * Ns + s];
  if constexpr (P == P_F64) { o[0] = c.x; o[1] = c.y; }
  else { o[0] = c.x; o[1] = c.y; o[2] = c.z; o[3] = c.w; }
}
template <int P>
__device__ __forceinline__ void store_chunk(Field f, long cb, int s, int Ns, int k,
                                            const typename PT<P>::real (&v)[PT<P>::RPC]) {
  static_assert(!PT<P>::HALF, "chunk access needs an unnormalised precision");
  typename PT<P>::chunk *b = (typename PT<P>::chunk *)f.v + ((size_t)cb * PT<P>::NCH + k) * Ns + s;
  if constexpr (P == P_F64) *b = make_double2(v[0], v[1]);
  else *b = make_float4(v[0], v[1], v[2], v[3]);
}

// ------------------------------------------------------------------ links

template <int P>
__device__ __forceinline__ void load_link(const typename PT<P>::lreal *L, typename PT<P>::real (&W)[18]) {
  if constexpr (!PT<P>::HALF) {
#pragma unroll
    for (int i = 0; i < 18; ++i) W[i] = L[i];
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      if constexpr (P == P_F16) W[i] = __half2float(L[i]);
      else W[i] = __bfloat162float(L[i]);
    }
    // third row = conj(row0 x row1) for an SU(3) matrix
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
      // (r0 x r1)_b = r0_{b1} r1_{b2} - r0_{b2} r1_{b1}
      float re = (W[2 * b1] * W[6 + 2 * b2] - W[2 * b1 + 1] * W[6 + 2 * b2 + 1]) -
                 (W[2 * b2] * W[6 + 2 * b1] - W[2 * b2 + 1] * W[6 + 2 * b1 + 1]);
      float im = (W[2 * b1] * W[6 + 2 * b2 + 1] + W[2 * b1 + 1] * W[6 + 2 * b2]) -
                 (W[2 * b2] * W[6 + 2 * b1 + 1] + W[2 * b2 + 1] * W[6 + 2 * b1]);
      W[12 + 2 * b] = re;
      W[12 + 2 * b + 1] = -im;
    }
  }
}

// ------------------------------------------------------------------ spin projection

// A_mu = upper-right block of gamma_mu; each row of A and A^dag has one non-zero
// entry, phase code 0: 1, 1: i, 2: -1, 3: -i.
__host__ __device__ constexpr int a_col(int mu, int j) { return (mu == 0 || mu == 1) ? 1 - j : j; }
__host__ __device__ constexpr int a_ph(int mu, int j) {
  return mu == 0 ? 3 : mu == 1 ? (j == 0 ? 2 : 0) : mu == 2 ? (j == 0 ? 3 : 1) : 0;
}
__host__ __device__ constexpr int ad_col(int mu, int k) { return (mu == 0 || mu == 1) ? 1 - k : k; }
__host__ __device__ constexpr int ad_ph(int mu, int k) {
  return mu == 0 ? 1 : mu == 1 ? (k == 0 ? 0 : 2) : mu == 2 ? (k == 0 ? 1 : 3) : 0;
}

template <int PH, typename R>
__device__ __forceinline__ void phase(R &re, R &im) {
  if constexpr (PH == 1) { R t = re; re = -im; im = t; }
  else if constexpr (PH == 2) { re = -re; im = -im; }
  else if constexpr (PH == 3) { R t = re; re = im; im = -t; }
}

// ------------------------------------------------------------------ packed FP32 pairs
//
// Blackwell executes two FP32 operations per instruction on a 64-bit register pair
// (add/sub/mul/fma .rn.f32x2).  A complex number (re, im) is such a pair; a sum of
// complex products sum_b w_b h_b is two packed FMA chains, P = sum_b w_b (hr_b, hr_b) and
// Q = sum_b w_b (hi_b, hi_b), joined as P + (-1, 1) (Q.y, Q.x).

struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 pk2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(f2 x, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// a * b + c
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 swp2(f2 x) {
  float a, b;
  upk2(x, a, b);
  return pk2(b, a);
}

// up + S * phase(PH) * z with the sign S a run-time value, given as the packed pairs
// s2 = (S, S), ns2 = (-S, -S), sa = (-S, S), nsa = (S, -S)
struct SignPairs {
  f2 s2, ns2, sa, nsa;
};
__device__ __forceinline__ SignPairs sign_pairs(float S) {
  return SignPairs{pk2(S, S), pk2(-S, -S), pk2(-S, S), pk2(S, -S)};
}
template <int PH>
__device__ __forceinline__ f2 add_phase_rt(f2 up, f2 z, const SignPairs &sg) {
  if constexpr (PH == 0) return fma2(z, sg.s2, up);
  else if constexpr (PH == 2) return fma2(z, sg.ns2, up);
  else if constexpr (PH == 1) return fma2(swp2(z), sg.sa, up);   // i z = (-zi, zr)
  else return fma2(swp2(z), sg.nsa, up);                          // -i z = (zi, -zr)
}

// acc += (1 + S g_mu) W psi in FP32 pairs, with S = +-1 at run time (forward hops S = -1,
// backward S = +1, so the eight directions run the same instructions) and the link as
// stored (nine complex entries, pairs of them 16-byte aligned):
// W h = P + (-1, 1) (Q.y, Q.x) with P = sum_b W_b (hr_b, hr_b), Q = sum_b W_b (hi_b, hi_b)
template <int MU>
__device__ __forceinline__ void hop_dir_raw(f2 (&acc)[12], const f2 (&ps)[12], const float4 *Wl,
                                            const SignPairs &sg) {
  f2 hr[2][3], hi[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const f2 h0 = add_phase_rt<a_ph(MU, 0)>(ps[a], ps[a + 3 * (2 + a_col(MU, 0))], sg);
    const f2 h1 = add_phase_rt<a_ph(MU, 1)>(ps[a + 3], ps[a + 3 * (2 + a_col(MU, 1))], sg);
    float x, y;
    upk2(h0, x, y);
    hr[0][a] = pk2(x, x);
    hi[0][a] = pk2(y, y);
    upk2(h1, x, y);
    hr[1][a] = pk2(x, x);
    hi[1][a] = pk2(y, y);
  }
  const f2 sgn = pk2(-1.f, 1.f);
  float4 w1;  // row 0 ends and row 1 starts in the second float4
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f2 W0, W1, W2;  // row a: entries 3a, 3a + 1, 3a + 2
    if (a == 0) {
      const float4 w0 = Wl[0];
      w1 = Wl[1];
      W0 = pk2(w0.x, w0.y), W1 = pk2(w0.z, w0.w), W2 = pk2(w1.x, w1.y);
    } else if (a == 1) {
      const float4 w2 = Wl[2];
      W0 = pk2(w1.z, w1.w), W1 = pk2(w2.x, w2.y), W2 = pk2(w2.z, w2.w);
    } else {
      const float4 w3 = Wl[3], w4 = Wl[4];
      W0 = pk2(w3.x, w3.y), W1 = pk2(w3.z, w3.w), W2 = pk2(w4.x, w4.y);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      f2 P = mul2(W0, hr[j][0]);
      P = fma2(W1, hr[j][1], P);
      P = fma2(W2, hr[j][2], P);
      f2 Q = mul2(W0, hi[j][0]);
      Q = fma2(W1, hi[j][1], Q);
      Q = fma2(W2, hi[j][2], Q);
      const f2 wh = fma2(sgn, swp2(Q), P);
      acc[a + 3 * j] = add2(acc[a + 3 * j], wh);
      if (ad_col(MU, 0) == j) acc[a + 6] = add_phase_rt<ad_ph(MU, 0)>(acc[a + 6], wh, sg);
      if (ad_col(MU, 1) == j) acc[a + 9] = add_phase_rt<ad_ph(MU, 1)>(acc[a + 9], wh, sg);
    }
  }
}

// FP64 version of hop_dir with the sign S at run time
template <int MU, typename R>
__device__ __forceinline__ void hop_dir_s(R (&acc)[24], const R (&ps)[24], const R (&W)[18], R S) {
  R h[2][3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int src = 2 + a_col(MU, j);
      R vr = ps[2 * (a + 3 * src)], vi = ps[2 * (a + 3 * src) + 1];
      switch (a_ph(MU, j)) {
        case 1: { R t = vr; vr = -vi; vi = t; } break;
        case 2: vr = -vr; vi = -vi; break;
        case 3: { R t = vr; vr = vi; vi = -t; } break;
        default: break;
      }
      h[j][a][0] = ps[2 * (a + 3 * j)] + S * vr;
      h[j][a][1] = ps[2 * (a + 3 * j) + 1] + S * vi;
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R re = 0, im = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R ur = W[2 * (3 * a + b)], ui = W[2 * (3 * a + b) + 1];
        re += ur * h[j][b][0] - ui * h[j][b][1];
        im += ur * h[j][b][1] + ui * h[j][b][0];
      }
      acc[2 * (a + 3 * j)] += re;
      acc[2 * (a + 3 * j) + 1] += im;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (ad_col(MU, k) != j) continue;
        R vr = re, vi = im;
        switch (ad_ph(MU, k)) {
          case 1: { R t = vr; vr = -vi; vi = t; } break;
          case 2: vr = -vr; vi = -vi; break;
          case 3: { R t = vr; vr = vi; vi = -t; } break;
          default: break;
        }
        acc[2 * (a + 3 * (2 + k))] += S * vr;
        acc[2 * (a + 3 * (2 + k)) + 1] += S * vi;
      }
    }
}

}  // namespace dwf
