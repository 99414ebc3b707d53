// Launch profile: per kernel class, launch counts, CUDA-event durations and the
// algorithmic flops / bytes of each launch (computed on the host from the launch
// arguments, not from hardware counters).
#include <mutex>
#include <vector>

#include "../../include/kr.h"
#include "kr_engine.h"
#include "kr_profile.h"

namespace kr {

namespace {

struct Pending {
  int cls;
  cudaEvent_t a, b;
};

struct ProfState {
  bool on = false;
  bool timed = false;
  std::mutex mu;
  int64_t launches[8] = {0};
  double ms[8] = {0};
  double flops[8] = {0};
  double bytes[8] = {0};
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
};

ProfState& P() {
  static ProfState s;
  return s;
}

cudaEvent_t take_event(ProfState& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  KR_CUDA(cudaEventCreate(&e));
  return e;
}

void drain(ProfState& p) {
  for (Pending& q : p.pending) {
    KR_CUDA(cudaEventSynchronize(q.b));
    float ms = 0.f;
    KR_CUDA(cudaEventElapsedTime(&ms, q.a, q.b));
    p.ms[q.cls] += ms;
    p.pool.push_back(q.a);
    p.pool.push_back(q.b);
  }
  p.pending.clear();
}

}  // namespace

bool prof_active() { return P().on; }

ProfToken prof_begin(int cls, cudaStream_t st) {
  ProfState& p = P();
  ProfToken t;
  t.cls = cls;
  if (!p.on) return t;
  t.active = true;
  if (p.timed) {
    std::lock_guard<std::mutex> lk(p.mu);
    t.a = take_event(p);
    KR_CUDA(cudaEventRecord(t.a, st));
  }
  return t;
}

void prof_end(ProfToken& t, cudaStream_t st, double flops, double bytes) {
  if (!t.active) return;
  ProfState& p = P();
  std::lock_guard<std::mutex> lk(p.mu);
  p.launches[t.cls] += 1;
  p.flops[t.cls] += flops;
  p.bytes[t.cls] += bytes;
  if (t.a) {
    cudaEvent_t b = take_event(p);
    KR_CUDA(cudaEventRecord(b, st));
    p.pending.push_back(Pending{t.cls, t.a, b});
    if (p.pending.size() > 100000) drain(p);
  }
}

// ----- algorithmic work of the row kernels ----------------------------------------------
double red_flops(const RedSet& rs, int64_t n, int s) {
  double f = 0.0;
  for (int i = 0; i < rs.nred; ++i) {
    switch (rs.r[i].kind) {
      case RED_GRAM: f += 8.0 * s * s * n; break;
      case RED_NORM2: f += 4.0 * s * n; break;
      default: f += 8.0 * s * n; break;
    }
  }
  return f;
}

double red_bytes(const RedSet& rs, int64_t n, int s, double elem, const void* const* counted, int ncounted) {
  double b = 0.0;
  for (int i = 0; i < rs.nred; ++i) {
    const RedSpec& r = rs.r[i];
    if (r.ureg >= 0 || r.U == nullptr) continue;
    bool seen = false;
    for (int k = 0; k < ncounted; ++k) seen = seen || counted[k] == r.U;
    if (seen) continue;
    const bool vec = r.kind == RED_SUMV || r.kind == RED_GRAMV;
    b += elem * n * (vec ? 1 : s);
  }
  return b;
}

}  // namespace kr

using namespace kr;

extern "C" {

kr_status kr_profile_enable(int32_t enable, int32_t time_kernels) {
  ProfState& p = P();
  std::lock_guard<std::mutex> lk(p.mu);
  p.on = enable != 0;
  p.timed = p.on && time_kernels != 0;
  return KR_OK;
}

kr_status kr_profile_read(kr_profile* out, int32_t reset) {
  ProfState& p = P();
  try {
    std::lock_guard<std::mutex> lk(p.mu);
    drain(p);
    if (out) {
      for (int i = 0; i < 8; ++i) {
        out->launches[i] = p.launches[i];
        out->ms[i] = p.ms[i];
        out->flops[i] = p.flops[i];
        out->bytes[i] = p.bytes[i];
      }
    }
    if (reset) {
      for (int i = 0; i < 8; ++i) { p.launches[i] = 0; p.ms[i] = p.flops[i] = p.bytes[i] = 0.0; }
    }
  } catch (const CudaError& e) {
    set_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");
    return KR_CUDA_ERROR;
  }
  return KR_OK;
}

}  // extern "C"
