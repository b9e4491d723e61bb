// Per-kernel launch timing with CUDA events (the library's tracing subsystem).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace fld {

class Tracer {
 public:
  bool on = false;
  bool major_only = false;  // skip the coarse-level and bookkeeping scopes (cheaper to record)
  void begin(const char* name, cudaStream_t s);
  void end(cudaStream_t s);
  void clear();
  // name -> (launches, total ms); synchronises on the recorded events
  struct Entry {
    std::string name;
    int launches;
    double ms;
  };
  std::vector<Entry> report();

 private:
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs_;
  std::vector<cudaEvent_t> pool_;
  const char* pending_ = nullptr;
  cudaEvent_t pending_ev_ = nullptr;
  cudaEvent_t get();
};

Tracer& tracer();

// Scopes of the coarse multigrid levels and of small bookkeeping kernels ("..._Lc", "coarse_...",
// "reduce", "fmg_restrict")
bool minor_scope(const char* name);

// Records the launches between construction and destruction under `name` when tracing is on.
struct TraceScope {
  cudaStream_t s;
  bool active;
  TraceScope(const char* name, cudaStream_t st)
      : s(st), active(tracer().on && !(tracer().major_only && minor_scope(name))) {
    if (active) tracer().begin(name, s);
  }
  ~TraceScope() {
    if (active) tracer().end(s);
  }
};

}  // namespace fld
