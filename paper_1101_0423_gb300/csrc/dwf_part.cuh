// dwf_part.cuh -- 4D domain decomposition: a part's halo layout and the kernels that build
// its neighbour table and gauge field and move spin-projected faces between parts.
//
// The lattice is cut into grid[0] x grid[1] x grid[2] x grid[3] blocks of extents L[mu]
// (even, so a site's parity is the same in local and global coordinates).  A part's field
// of one parity holds its h local sites and, after them, one halo slot per site of that
// parity just outside each cut face: for each cut direction mu a lower slab (x_mu = -1)
// and an upper slab (x_mu = L_mu), fsz[mu] slots each, at h + foff[mu][side].  A halo slot
// holds (h, 0): the spin projection the receiving hop needs (Eq. 12: (1 - g_mu) psi(x + mu)
// for a forward neighbour, (1 + g_mu) psi(x - mu) for a backward one) in the upper two
// spins and zeros below, so that the unchanged hop kernel, projecting it again, gets h back
// (Sec. 3.2's spin projection: only the 12 reals of h per (site, s) travel between parts).
// A face slot's index is its three other local coordinates in lexicographic order (first
// fastest), halved -- the same in the sending and the receiving part.
#pragma once

#include "dwf_kernels.cuh"

namespace dwf {

struct PartGeom {
  int L[4];          // local extents
  int grid[4];       // parts per direction
  int coord[4];      // this part's position in the grid
  int G[4];          // global extents
  long h;            // local sites per parity
  long foff[4][2];   // halo slot offset after h of (mu, lower / upper); -1 when mu is not cut
  long fsz[4];       // sites of one parity on one face of direction mu
  long halo;         // halo slots per parity field
};

inline PartGeom make_part_geom(const int G[4], const int grid[4], const int coord[4]) {
  PartGeom g;
  long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.G[mu] = G[mu];
    g.grid[mu] = grid[mu];
    g.coord[mu] = coord[mu];
    g.L[mu] = G[mu] / grid[mu];
    V *= g.L[mu];
  }
  g.h = V / 2;
  long off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    g.fsz[mu] = V / g.L[mu] / 2;
    if (grid[mu] > 1) {
      g.foff[mu][0] = off;
      g.foff[mu][1] = off + g.fsz[mu];
      off += 2 * g.fsz[mu];
    } else {
      g.foff[mu][0] = g.foff[mu][1] = -1;
    }
  }
  g.halo = off;
  return g;
}

// halved lexicographic index of the three coordinates other than mu
__host__ __device__ inline long face_half(const PartGeom &g, int mu, const int (&c)[4]) {
  long f = 0, m = 1;
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) {
      f += c[nu] * m;
      m *= g.L[nu];
    }
  return f >> 1;
}

// local coordinates of face slot fh of direction mu at x_mu = xmu, parity q
__host__ __device__ inline void face_site(const PartGeom &g, int mu, int xmu, int q, long fh, int (&c)[4]) {
  int nus[3], k = 0;
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) nus[k++] = nu;
  const int e0h = g.L[nus[0]] / 2;
  const long rest = fh / e0h;
  const int ah = (int)(fh - rest * e0h);
  const int b = (int)(rest % g.L[nus[1]]), cc = (int)(rest / g.L[nus[1]]);
  const int bit = (q - (b + cc + xmu)) & 1;  // the site's parity (sum of coordinates) is q
  c[nus[0]] = 2 * ah + bit;
  c[nus[1]] = b;
  c[nus[2]] = cc;
  c[mu] = xmu;
}

__host__ __device__ inline long local_site(const PartGeom &g, const int (&c)[4]) {
  return c[0] + (long)g.L[0] * (c[1] + (long)g.L[1] * (c[2] + (long)g.L[2] * c[3]));
}

__host__ __device__ inline Geom local_geom(const PartGeom &g, int Ns) {
  Geom lg;
  for (int mu = 0; mu < 4; ++mu) lg.d[mu] = g.L[mu];
  lg.h = g.h;
  lg.Ns = Ns;
  return lg;
}

// doubled gauge of output parity p for the local sites (same layout as k_gauge), read from
// the global host-layout field: the backward links of the sites on a lower cut face are the
// neighbouring part's, so no link halo has to be exchanged
template <int P>
__global__ void k_part_gauge(const double *Ug, typename PT<P>::lreal *Gd, PartGeom g, int p) {
  using L = typename PT<P>::lreal;
  constexpr int LR = PT<P>::LREALS;
  const Geom lg = local_geom(g, 0);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < g.h * 8; i += (long)gridDim.x * blockDim.x) {
    const long cb = i >> 3;
    const int dir = (int)(i & 7), mu = dir & 3;
    int c[4];
    cb_to_site(lg, cb, p, c);
    int x[4];
    for (int nu = 0; nu < 4; ++nu) x[nu] = c[nu] + g.coord[nu] * g.L[nu];
    const bool dag = dir >= 4;
    if (dag) x[mu] = (x[mu] + g.G[mu] - 1) % g.G[mu];
    const long site = x[0] + (long)g.G[0] * (x[1] + (long)g.G[1] * (x[2] + (long)g.G[2] * x[3]));
    const double *u = Ug + ((size_t)site * 4 + mu) * 18;
    L *o = Gd + (size_t)cb * PT<P>::SITE_LREALS + dir * LR;
    for (int e = 18; e < LR; ++e) o[e] = L(0.f);
    if (dir == 7)
      for (int e = 8 * LR; e < PT<P>::SITE_LREALS; ++e) Gd[(size_t)cb * PT<P>::SITE_LREALS + e] = L(0.f);
    for (int a = 0; a < 3 && a * 6 < LR; ++a)
      for (int b = 0; b < 3; ++b) {
        const double re = dag ? u[2 * (3 * b + a)] : u[2 * (3 * a + b)];
        const double im = dag ? -u[2 * (3 * b + a) + 1] : u[2 * (3 * a + b) + 1];
        if constexpr (P == P_F64) { o[2 * (3 * a + b)] = re; o[2 * (3 * a + b) + 1] = im; }
        else if constexpr (P == P_F32) { o[2 * (3 * a + b)] = (float)re; o[2 * (3 * a + b) + 1] = (float)im; }
        else if constexpr (P == P_F16) { o[2 * (3 * a + b)] = __double2half(re); o[2 * (3 * a + b) + 1] = __double2half(im); }
        else { o[2 * (3 * a + b)] = __double2bfloat16(re); o[2 * (3 * a + b) + 1] = __double2bfloat16(im); }
      }
  }
}

// neighbour table of output parity p: local sites (periodic along uncut directions), or the
// halo slots of the opposite-parity field across cut faces
template <int X = 0>
__global__ void k_part_neighbours(int *nbr, PartGeom g, int p) {
  const Geom lg = local_geom(g, 0);
  for (long cb = (long)blockIdx.x * blockDim.x + threadIdx.x; cb < g.h; cb += (long)gridDim.x * blockDim.x) {
    int c[4];
    cb_to_site(lg, cb, p, c);
    for (int dir = 0; dir < 8; ++dir) {
      const int mu = dir & 3;
      int e[4] = {c[0], c[1], c[2], c[3]};
      e[mu] += dir < 4 ? 1 : -1;
      long idx;
      if (e[mu] >= 0 && e[mu] < g.L[mu]) {
        idx = local_site(g, e) >> 1;
      } else if (g.grid[mu] == 1) {
        e[mu] = (e[mu] + g.L[mu]) % g.L[mu];
        idx = local_site(g, e) >> 1;
      } else {
        idx = g.h + g.foff[mu][e[mu] < 0 ? 0 : 1] + face_half(g, mu, e);
      }
      nbr[cb * 8 + dir] = (int)idx;
    }
  }
}

// packs face `side` (0: x_mu = 0, 1: x_mu = L_mu - 1) of a parity-q field as the projection
// with sign S (S = -1 for the lower face: forward neighbours of the part below; S = +1 for
// the upper face: backward neighbours of the part above), 12 reals per (slot, s)
template <int P>
__global__ void k_part_pack(const Field in, PartGeom g, int Ns, int mu, int side, int q, double S,
                            typename PT<P>::real *buf) {
  using R = typename PT<P>::real;
  const long n = g.fsz[mu] * Ns;
  const int xmu = side ? g.L[mu] - 1 : 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long fh = i / Ns;
    const int s = (int)(i % Ns);
    int c[4];
    face_site(g, mu, xmu, q, fh, c);
    R v[24];
    load_sp<P>(in, local_site(g, c) >> 1, s, Ns, v);
    R *o = buf + (size_t)i * 12;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int src = 2 + a_col(mu, j);
      const int ph = a_ph(mu, j);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R vr = v[2 * (a + 3 * src)], vi = v[2 * (a + 3 * src) + 1];
        if (ph == 1) { const R t = vr; vr = -vi; vi = t; }
        else if (ph == 2) { vr = -vr; vi = -vi; }
        else if (ph == 3) { const R t = vr; vr = vi; vi = -t; }
        o[2 * (a + 3 * j)] = v[2 * (a + 3 * j)] + (R)S * vr;
        o[2 * (a + 3 * j) + 1] = v[2 * (a + 3 * j) + 1] + (R)S * vi;
      }
    }
  }
}

// writes nslot x Ns packed (slot, s) projections as (h, 0) into halo slots first, first + 1, ...
template <int P>
__global__ void k_part_unpack(const typename PT<P>::real *buf, Field out, long first, long nslot, int Ns) {
  using R = typename PT<P>::real;
  const long n = nslot * Ns;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    R v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = buf[(size_t)i * 12 + k];
#pragma unroll
    for (int k = 12; k < 24; ++k) v[k] = 0;
    store_sp<P>(out, first + i / Ns, (int)(i % Ns), Ns, v);
  }
}

}  // namespace dwf
