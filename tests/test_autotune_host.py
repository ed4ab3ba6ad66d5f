"""The autotuner's host logic (csrc/dwf_tune.h) without a GPU: the candidate launch shapes
for each Ns, the choice of the fastest timed candidate, and the thread-safe cache, compiled
with g++ into a small program that prints what it computes."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1101_0423_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include <thread>
#include "dwf_tune.h"
using namespace dwf;
int main() {
  for (int ns : {1, 5, 8, 12, 16, 24, 32, 64}) {
    printf("cand %d", ns);
    for (const HopShape &s : hop_candidates(ns)) printf(" %d:%d:%d", s.threads, (int)s.persistent, shape_spb(s, ns));
    printf("\n");
  }
  HopShape a{128, false}, b{64, true}, c{256, false};
  HopShape p = pick_fastest({{a, 3.0}, {b, 2.0}, {c, 2.5}}, a);
  printf("pick %d %d\n", p.threads, (int)p.persistent);
  p = pick_fastest({{a, 2.0}, {b, 2.0}}, c);
  printf("tie %d %d\n", p.threads, (int)p.persistent);
  p = pick_fastest({{a, -1.0}, {b, 0.0}}, c);
  printf("none %d %d\n", p.threads, (int)p.persistent);
  printf("vclass %d %d %d\n", volume_class(1), volume_class(65536), volume_class(65537));
  TuneCache cache;
  HopShape got;
  printf("miss %d\n", (int)cache.get(TuneCache::Key(0, 1, 1, 16, 16), &got));
  std::thread t1([&] { for (int i = 0; i < 1000; ++i) cache.put(TuneCache::Key(0, 1, 1, i % 7, 16), b); });
  std::thread t2([&] { for (int i = 0; i < 1000; ++i) cache.put(TuneCache::Key(1, 1, 1, i % 5, 16), c); });
  t1.join();
  t2.join();
  printf("size %zu\n", cache.size());
  const bool hit = cache.get(TuneCache::Key(0, 1, 1, 3, 16), &got);
  printf("hit %d %d %d\n", (int)hit, got.threads, (int)got.persistent);
  printf("other %d\n", (int)cache.get(TuneCache::Key(0, 2, 1, 3, 16), &got));
  cache.clear();
  printf("cleared %zu\n", cache.size());
  return 0;
}
'''


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    d = tmp_path_factory.mktemp("tune")
    src, exe = d / "t.cpp", d / "t"
    src.write_text(PROG)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)])
    lines = subprocess.check_output([str(exe)], text=True).splitlines()
    return {ln.split()[0] + ("" if not ln.startswith("cand") else ln.split()[1]): ln.split()[1:] for ln in lines}


def _cands(output, ns):
    return [tuple(map(int, c.split(":"))) for c in output[f"cand{ns}"][1:]]


def test_candidates_cover_three_cta_sizes_both_grids(output):
    c16 = _cands(output, 16)
    assert c16[0] == (128, 0, 8)                     # the default shape is timed first
    assert {(t, p) for t, p, _ in c16} == {(t, p) for t in (64, 128, 256) for p in (0, 1)}
    for ns in (1, 5, 8, 12, 16, 24, 32, 64):
        for t, p, spb in _cands(output, ns):
            assert 1 <= spb <= 64 and spb * ns <= 256  # a CTA holds at most 256 threads, 64 sites


def test_candidates_drop_shapes_with_equal_site_counts(output):
    # Ns = 64: 64 and 128 threads give one and two sites; 256 threads four
    assert [spb for _, p, spb in _cands(output, 64) if p == 0] == [2, 1, 4]
    # Ns = 1: 64 sites is the cap, so 128 and 256 threads collapse onto it
    assert len({spb for _, _, spb in _cands(output, 1)}) == len(_cands(output, 1)) // 2


def test_pick_fastest(output):
    assert output["pick"] == ["64", "1"]
    assert output["tie"] == ["128", "0"]     # first of equal times
    assert output["none"] == ["256", "0"]    # every candidate failed: the fallback


def test_volume_class_and_cache(output):
    assert output["vclass"] == ["0", "16", "16"]
    assert output["miss"] == ["0"]
    assert output["size"] == ["12"]          # 7 + 5 distinct keys written from two threads
    assert output["hit"] == ["1", "64", "1"]
    assert output["other"] == ["0"]
    assert output["cleared"] == ["0"]
