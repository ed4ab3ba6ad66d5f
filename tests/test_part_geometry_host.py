"""The domain decomposition's index arithmetic (csrc/dwf_part.cuh) without a GPU: a part's
halo layout, the enumeration of its face sites by slot (face_site) and the slot of a site
(face_half, what a receiving part's neighbour table uses), compiled with nvcc into a host
program that checks them over several lattices and cuts and prints what it found."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1101_0423_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include <set>
#include <vector>
#include "dwf_part.cuh"
using namespace dwf;
static int fails = 0;
#define CHECK(c) do { if (!(c)) { ++fails; if (fails < 10) printf("fail %s line %d\n", #c, __LINE__); } } while (0)
int main() {
  const int cases[][8] = {{4, 4, 4, 8, 2, 1, 1, 1}, {8, 4, 4, 8, 1, 1, 1, 2}, {4, 4, 4, 4, 2, 2, 1, 1},
                          {8, 8, 4, 4, 2, 2, 2, 2}, {6, 4, 2, 8, 3, 2, 1, 2}};
  int checked = 0;
  for (const auto &cs : cases) {
    const int G[4] = {cs[0], cs[1], cs[2], cs[3]}, grid[4] = {cs[4], cs[5], cs[6], cs[7]};
    const int coord[4] = {grid[0] - 1, 0, grid[2] / 2, grid[3] - 1};
    const PartGeom g = make_part_geom(G, grid, coord);
    long V = 1, halo = 0, off = 0;
    for (int mu = 0; mu < 4; ++mu) V *= g.L[mu];
    CHECK(g.h == V / 2);
    for (int mu = 0; mu < 4; ++mu) {
      CHECK(g.L[mu] * grid[mu] == G[mu] && g.L[mu] % 2 == 0);
      CHECK(g.fsz[mu] == V / g.L[mu] / 2);
      if (grid[mu] == 1) {
        CHECK(g.foff[mu][0] == -1 && g.foff[mu][1] == -1);
        continue;
      }
      // the halo slabs follow one another: lower then upper, direction by direction
      CHECK(g.foff[mu][0] == off && g.foff[mu][1] == off + g.fsz[mu]);
      off += 2 * g.fsz[mu];
      halo += 2 * g.fsz[mu];
      for (int q = 0; q < 2; ++q)
        for (int xmu : {0, g.L[mu] - 1, -1, g.L[mu]}) {
          std::set<long> seen;
          for (long fh = 0; fh < g.fsz[mu]; ++fh) {
            int c[4];
            face_site(g, mu, xmu, q, fh, c);
            CHECK(c[mu] == xmu);
            CHECK((((c[0] + c[1] + c[2] + c[3]) % 2) + 2) % 2 == q);  // the parity asked for
            for (int nu = 0; nu < 4; ++nu)
              if (nu != mu) CHECK(c[nu] >= 0 && c[nu] < g.L[nu]);
            CHECK(face_half(g, mu, c) == fh);  // the slot of the site is the slot enumerated
            if (xmu >= 0 && xmu < g.L[mu]) {
              const long cb = local_site(g, c) >> 1;
              CHECK(cb >= 0 && cb < g.h);
              seen.insert(cb);
            } else {
              seen.insert(fh);
            }
            ++checked;
          }
          CHECK((long)seen.size() == g.fsz[mu]);  // every face site once
        }
      // sender and receiver agree: the face x_mu = L - 1 of the part below, as enumerated by
      // the sender, is the receiver's lower halo x_mu = -1 slot for slot (and the face x_mu = 0
      // of the part above its upper halo x_mu = L), the other coordinates and parity equal
      for (int q = 0; q < 2; ++q)
        for (long fh = 0; fh < g.fsz[mu]; ++fh) {
          int s[4], r[4];
          face_site(g, mu, g.L[mu] - 1, q, fh, s);
          face_site(g, mu, -1, q, fh, r);
          for (int nu = 0; nu < 4; ++nu)
            if (nu != mu) CHECK(s[nu] == r[nu]);
          face_site(g, mu, 0, q, fh, s);
          face_site(g, mu, g.L[mu], q, fh, r);
          for (int nu = 0; nu < 4; ++nu)
            if (nu != mu) CHECK(s[nu] == r[nu]);
        }
    }
    CHECK(g.halo == halo);
  }
  printf("checked %d fails %d\n", checked, fails);
  return fails ? 1 : 0;
}
'''


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("partgeom")
    src = d / "partgeom.cu"
    src.write_text(PROG)
    exe = d / "partgeom"
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    return r.returncode, r.stdout


def test_halo_layout_and_face_slots(output):
    rc, out = output
    assert rc == 0, out
    last = out.strip().splitlines()[-1].split()
    assert last[0] == "checked" and int(last[1]) > 1000 and last[3] == "0", out
