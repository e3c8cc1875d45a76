// Launch-policy autotuner: the first call for a key (kernel, precision,
// shape) times every candidate policy with CUDA events on the caller's
// stream and keeps the fastest, in memory and, when GBMG_TUNE_CACHE names a
// file, on disk ("key value" lines, read on first use).  GBMG_TUNE=0 turns
// tuning off (the first candidate is used).  A stream that is being
// captured into a CUDA graph is never timed: the cached or first candidate
// is used, so tune (make one call) before capturing.
#pragma once

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace gbmg {

class Tuner {
 public:
  static Tuner& get() {
    static Tuner t;
    return t;
  }

  // Returns the chosen candidate.  launch(c) must enqueue one launch with
  // policy c on stream st; it is called repeatedly while timing.
  template <typename F>
  int choose(const std::string& key, const std::vector<int>& cands, cudaStream_t st, F&& launch) {
    std::lock_guard<std::mutex> lk(mu_);
    load();
    auto it = best_.find(key);
    // a cached or pinned choice is used only if it is a candidate of this call
    if (it != best_.end() &&
        std::find(cands.begin(), cands.end(), it->second) != cands.end())
      return it->second;
    if (!enabled_ || cands.size() == 1) return cands.front();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return cands.front();
    cudaEvent_t a, b;
    GB_CHECK(cudaEventCreate(&a));
    GB_CHECK(cudaEventCreate(&b));
    int pick = cands.front();
    float best_ms = 1e30f;
    std::vector<std::pair<int, float>> times;
    for (int c : cands) {
      launch(c);  // warm-up
      GB_CHECK(cudaEventRecord(a, st));
      for (int r = 0; r < 3; ++r) launch(c);
      GB_CHECK(cudaEventRecord(b, st));
      GB_CHECK(cudaEventSynchronize(b));
      float ms = 0.f;
      GB_CHECK(cudaEventElapsedTime(&ms, a, b));
      times.emplace_back(c, ms / 3.f);
      if (ms < best_ms) {
        best_ms = ms;
        pick = c;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    best_[key] = pick;
    timings_[key] = times;
    if (!path_.empty()) {
      std::ofstream f(path_, std::ios::app);
      if (f) f << key << " " << pick << "\n";
    }
    return pick;
  }

  // number of entries (tests)
  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return best_.size();
  }

  // pin a choice for key (choice < 0 removes the entry, so the next call
  // tunes again); the pin is not written to the cache file
  void set(const std::string& key, int choice) {
    std::lock_guard<std::mutex> lk(mu_);
    load();
    if (choice < 0)
      best_.erase(key);
    else
      best_[key] = choice;
  }
  // the candidates timed when `key` was last tuned, with ms per launch
  std::vector<std::pair<int, float>> report(const std::string& key) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = timings_.find(key);
    return it == timings_.end() ? std::vector<std::pair<int, float>>{} : it->second;
  }
  int get(const std::string& key) {
    std::lock_guard<std::mutex> lk(mu_);
    load();
    auto it = best_.find(key);
    return it == best_.end() ? -1 : it->second;
  }

 private:
  Tuner() {
    const char* e = std::getenv("GBMG_TUNE");
    enabled_ = !(e && std::string(e) == "0");
    const char* p = std::getenv("GBMG_TUNE_CACHE");
    if (p) path_ = p;
  }
  void load() {
    if (loaded_) return;
    loaded_ = true;
    if (path_.empty()) return;
    std::ifstream f(path_);
    std::string k;
    int v;
    while (f >> k >> v) best_[k] = v;
  }
  std::mutex mu_;
  std::unordered_map<std::string, int> best_;
  std::unordered_map<std::string, std::vector<std::pair<int, float>>> timings_;
  bool loaded_ = false;
  bool enabled_ = true;
  std::string path_;
};

}  // namespace gbmg
