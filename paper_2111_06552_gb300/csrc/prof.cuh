// Per-kernel-class CUDA-event profile (enabled by gcge_options.profile) -- internal.
#pragma once
#include <vector>

#include "common.cuh"

namespace gcge {

struct KProf {
  cudaStream_t st = nullptr;
  struct Slot {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops;
  };
  std::vector<Slot> pool;
  size_t used = 0;
  double ms[12] = {0}, bytes[12] = {0}, flops[12] = {0};
  int64_t calls[12] = {0};

  ~KProf() {
    harvest();
    for (auto &s : pool) {
      cudaEventDestroy(s.a);
      cudaEventDestroy(s.b);
    }
  }
  // Start a timed launch; returns the slot index.
  size_t begin(int cls, double by, double fl) {
    if (used == pool.size()) {
      if (pool.size() >= 8192) harvest();
      if (used == pool.size()) {
        Slot s{};
        cudaEventCreate(&s.a);
        cudaEventCreate(&s.b);
        pool.push_back(s);
      }
    }
    Slot &s = pool[used];
    s.cls = cls;
    s.bytes = by;
    s.flops = fl;
    cudaEventRecord(s.a, st);
    return used++;
  }
  void end(size_t i) { cudaEventRecord(pool[i].b, st); }
  // Accumulate all finished slots (waits for the last recorded event).
  void harvest() {
    if (used == 0) return;
    cudaEventSynchronize(pool[used - 1].b);
    for (size_t i = 0; i < used; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, pool[i].a, pool[i].b);
      const int c = pool[i].cls;
      ms[c] += t;
      calls[c] += 1;
      bytes[c] += pool[i].bytes;
      flops[c] += pool[i].flops;
    }
    used = 0;
  }
};

// RAII guard: times the launches issued inside its scope (no-op when p is null).
struct ProfScope {
  KProf *p;
  size_t i = 0;
  ProfScope(KProf *pp, int cls, double by, double fl) : p(pp) {
    if (p) i = p->begin(cls, by, fl);
  }
  ~ProfScope() {
    if (p) p->end(i);
  }
};

}  // namespace gcge
