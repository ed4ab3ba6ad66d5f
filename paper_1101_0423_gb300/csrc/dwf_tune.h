// dwf_tune.h -- launch-shape autotuner of the hop kernels (host code, no CUDA types).
//
// A hop kernel's launch shape is its CTA size (Ns slices x spb sites) and its grid: one
// tile per CTA, or a persistent grid of as many CTAs as are resident at once, each walking
// tiles.  Which is fastest depends on Ns, the precision, the epilogue and the lattice
// volume, so the first solve of a (device, precision, epilogue, Ns, volume class) times
// every candidate shape on the solve's own buffers and keeps the fastest for the rest of
// the process.  The candidates, the choice and the cache are plain host logic, kept here
// so that they can be tested without a GPU.
#pragma once

#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

namespace dwf {

struct HopShape {
  int threads = 128;       // CTA size; spb = max(1, min(64, threads / Ns)) sites per CTA
  bool persistent = false; // grid limited to the CTAs resident at once
  bool operator==(const HopShape &o) const { return threads == o.threads && persistent == o.persistent; }
};

// sites per CTA of a shape
inline int shape_spb(const HopShape &s, int Ns) {
  int spb = s.threads / Ns;
  if (spb > 64) spb = 64;
  return spb < 1 ? 1 : spb;
}

// the shapes worth timing for Ns: CTAs of 64, 128 and 256 threads (distinct site counts
// only; a CTA holds at most 256 threads and at most 64 sites), each as one tile per CTA
// and as a persistent grid
inline std::vector<HopShape> hop_candidates(int Ns) {
  std::vector<HopShape> out;
  std::vector<int> seen;
  for (int t : {128, 64, 256}) {
    HopShape s;
    s.threads = t;
    const int spb = shape_spb(s, Ns);
    if (spb * Ns > 256) continue;
    bool dup = false;
    for (int x : seen) dup = dup || x == spb;
    if (dup) continue;
    seen.push_back(spb);
    for (bool p : {false, true}) {
      s.persistent = p;
      out.push_back(s);
    }
  }
  return out;
}

// the fastest of the timed candidates (the first one on a tie, so the default shape, listed
// first, wins unless another is faster); non-positive times mark candidates that failed
inline HopShape pick_fastest(const std::vector<std::pair<HopShape, double>> &timed, const HopShape &fallback) {
  HopShape best = fallback;
  double best_t = -1.0;
  for (const auto &c : timed)
    if (c.second > 0.0 && (best_t < 0.0 || c.second < best_t)) {
      best = c.first;
      best_t = c.second;
    }
  return best;
}

// volume class of a lattice: the log2 of its half-lattice site count
inline int volume_class(long h) {
  int v = 0;
  while (h > 1) {
    h >>= 1;
    ++v;
  }
  return v;
}

// tuned shapes, keyed by (device, precision, epilogue, Ns, volume class); thread-safe
class TuneCache {
 public:
  using Key = std::tuple<int, int, int, int, int>;
  bool get(const Key &k, HopShape *out) const {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = map_.find(k);
    if (it == map_.end()) return false;
    *out = it->second;
    return true;
  }
  void put(const Key &k, const HopShape &s) {
    std::lock_guard<std::mutex> lock(mu_);
    map_[k] = s;
  }
  size_t size() const {
    std::lock_guard<std::mutex> lock(mu_);
    return map_.size();
  }
  void clear() {
    std::lock_guard<std::mutex> lock(mu_);
    map_.clear();
  }

 private:
  mutable std::mutex mu_;
  std::map<Key, HopShape> map_;
};

}  // namespace dwf
