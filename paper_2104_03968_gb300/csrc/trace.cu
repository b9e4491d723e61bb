// Per-kernel launch timing with CUDA events.
#include <map>

#include "fld_common.cuh"
#include "trace.h"

namespace fld {

std::atomic<unsigned long long> g_kernel_launches{0};  // declared in fld_common.cuh

Tracer& tracer() {
  static Tracer t;
  return t;
}

cudaEvent_t Tracer::get() {
  if (!pool_.empty()) {
    cudaEvent_t e = pool_.back();
    pool_.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Tracer::begin(const char* name, cudaStream_t s) {
  pending_ = name;
  pending_ev_ = get();
  cudaEventRecord(pending_ev_, s);
}

void Tracer::end(cudaStream_t s) {
  if (!pending_) return;
  cudaEvent_t b = get();
  cudaEventRecord(b, s);
  recs_.push_back({pending_, pending_ev_, b});
  pending_ = nullptr;
}

void Tracer::clear() {
  for (auto& r : recs_) {
    pool_.push_back(r.a);
    pool_.push_back(r.b);
  }
  recs_.clear();
}

std::vector<Tracer::Entry> Tracer::report() {
  std::map<std::string, std::pair<int, double>> acc;
  for (auto& r : recs_) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& v = acc[r.name];
    v.first += 1;
    v.second += ms;
  }
  std::vector<Entry> out;
  for (auto& kv : acc) out.push_back({kv.first, kv.second.first, kv.second.second});
  return out;
}

bool minor_scope(const char* name) {
  const std::string n(name);
  const size_t L = n.size();
  return (L > 3 && n.compare(L - 3, 3, "_Lc") == 0) || n.compare(0, 7, "coarse_") == 0 || n == "reduce" ||
         n == "fmg_restrict";
}

}  // namespace fld
