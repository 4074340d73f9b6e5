// Small host utilities shared by the plan implementations.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace pfft {

// cudaMalloc with the library's status mapping: out of memory vs. any other
// runtime failure (no device, driver mismatch, ...).
inline int device_alloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) return 0;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? 6 /* PFFT_ERR_OOM */ : 7 /* PFFT_ERR_CUDA */;
}

// Bump allocator over large device chunks: the tables of many small plans
// (a batch of patterns) without one cudaMalloc each.  Freed all at once.
class Arena {
 public:
  int alloc(void** p, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (chunks_.empty() || used_ + bytes > cap_) {
      const size_t c = bytes > kChunk ? bytes : kChunk;
      void* q = nullptr;
      if (int e = device_alloc(&q, c)) return e;
      chunks_.push_back(q);
      cap_ = c;
      used_ = 0;
    }
    *p = static_cast<char*>(chunks_.back()) + used_;
    used_ += bytes;
    return 0;
  }
  size_t reserved() const {
    size_t s = 0;
    for (size_t i = 0; i + 1 < chunks_.size(); ++i) s += kChunk;
    return s + cap_;
  }
  ~Arena() {
    for (void* c : chunks_) cudaFree(c);
  }

 private:
  static constexpr size_t kChunk = size_t(64) << 20;
  std::vector<void*> chunks_;
  size_t used_ = 0, cap_ = 0;
};

// Per-kernel timing with CUDA events recorded on the launching stream.
class Profiler {
 public:
  bool enable(bool on, int nkinds, const char* const* names) {
    drain();
    on_ = on;
    nkinds_ = nkinds;
    names_ = names;
    ms_.assign(nkinds, 0.0);
    count_.assign(nkinds, 0);
    return true;
  }
  void begin(int k, cudaStream_t s) {
    if (!on_) return;
    Rec r;
    r.k = k;
    r.a = take();
    r.b = take();
    cudaEventRecord(r.a, s);
    recs_.push_back(r);
  }
  void end(int k, cudaStream_t s) {
    if (!on_ || recs_.empty() || recs_.back().k != k) return;
    cudaEventRecord(recs_.back().b, s);
  }
  bool read(const char** names, int64_t* launches, double* ms, int cap, int* n) {
    bool ok = collect();
    int c = 0;
    for (int k = 0; k < nkinds_ && c < cap; ++k, ++c) {
      if (names) names[c] = names_[k];
      if (launches) launches[c] = count_[k];
      if (ms) ms[c] = ms_[k];
    }
    if (n) *n = c;
    return ok;
  }
  ~Profiler() {
    drain();
    for (auto e : pool_) cudaEventDestroy(e);
  }

 private:
  struct Rec {
    int k;
    cudaEvent_t a, b;
  };
  cudaEvent_t take() {
    if (!pool_.empty()) {
      cudaEvent_t e = pool_.back();
      pool_.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  bool collect() {
    bool ok = true;
    for (auto& r : recs_) {
      float t = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
        ok = false;
      ms_[r.k] += t;
      count_[r.k] += 1;
      pool_.push_back(r.a);
      pool_.push_back(r.b);
    }
    recs_.clear();
    return ok;
  }
  void drain() {
    for (auto& r : recs_) {
      cudaEventSynchronize(r.b);
      pool_.push_back(r.a);
      pool_.push_back(r.b);
    }
    recs_.clear();
  }
  bool on_ = false;
  int nkinds_ = 0;
  const char* const* names_ = nullptr;
  std::vector<double> ms_;
  std::vector<int64_t> count_;
  std::vector<Rec> recs_;
  std::vector<cudaEvent_t> pool_;
};

}  // namespace pfft
