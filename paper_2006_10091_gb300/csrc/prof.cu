// prof.cu -- per-kernel-class timing: when enabled, each instrumented launch
// is bracketed by CUDA events on the context's stream, and the host adds the
// launch's algorithmic work (butterflies, modular products or bytes) to its
// class.  Reading synchronises and sums the event intervals.
#include <string.h>

#include "he_ops.h"

namespace he {

static thread_local bool tl_prof_suppressed = false;

ProfSuppress::ProfSuppress() : prev_(tl_prof_suppressed) { tl_prof_suppressed = true; }
ProfSuppress::~ProfSuppress() { tl_prof_suppressed = prev_; }

ProfScope::ProfScope(he_ctx* c, const char* name, double work, double bytes, double mac, double bfly, double mac3)
    : c_(c) {
  if (!c->prof_on || tl_prof_suppressed) {
    c_ = nullptr;
    return;
  }
  ProfClass& k = c->prof[name];
  k.work += work;
  k.bytes += bytes;
  k.mac += mac;
  k.mac3 += mac3;
  k.bfly += bfly;
  k.launches += 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, c->stream);
  k.events.push_back({a, b});
  stop_ = b;
}

ProfScope::~ProfScope() {
  if (c_) cudaEventRecord(stop_, c_->stream);
}

void prof_clear(he_ctx* c) {
  for (auto& kv : c->prof)
    for (auto& e : kv.second.events) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  c->prof.clear();
}

}  // namespace he

using namespace he;

extern "C" int he_profile_enable(he_ctx* c, int enable) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_CUDA(cudaStreamSynchronize(c->stream));
  prof_clear(c);
  c->prof_on = enable != 0;
  return HE_OK;
}

extern "C" int he_profile_read(he_ctx* c, const char* name, uint64_t* launches, double* total_ms, double* work,
                               double* bytes) {
  if (!c || !name) return fail(HE_EINVAL, "null argument");
  HE_CUDA(cudaStreamSynchronize(c->stream));
  auto it = c->prof.find(name);
  double ms = 0.0;
  uint64_t cnt = 0;
  double w = 0.0, by = 0.0;
  if (it != c->prof.end()) {
    for (auto& e : it->second.events) {
      float t = 0.f;
      HE_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
      ms += t;
    }
    cnt = it->second.launches;
    w = it->second.work;
    by = it->second.bytes;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  if (work) *work = w;
  if (bytes) *bytes = by;
  return HE_OK;
}

extern "C" int he_profile_names(he_ctx* c, char* buf, size_t cap) {
  if (!c || !buf || cap == 0) return fail(HE_EINVAL, "null argument");
  std::string s;
  for (auto& kv : c->prof) {
    if (!s.empty()) s += ",";
    s += kv.first;
  }
  if (s.size() + 1 > cap) return fail(HE_EINVAL, "buffer too small");
  memcpy(buf, s.c_str(), s.size() + 1);
  return HE_OK;
}

extern "C" int he_profile_read_kinds(he_ctx* c, const char* name, double* butterflies, double* macs,
                                     double* split_macs) {
  if (!c || !name) return fail(HE_EINVAL, "null argument");
  auto it = c->prof.find(name);
  if (butterflies) *butterflies = it == c->prof.end() ? 0.0 : it->second.bfly;
  if (macs) *macs = it == c->prof.end() ? 0.0 : it->second.mac;
  if (split_macs) *split_macs = it == c->prof.end() ? 0.0 : it->second.mac3;
  return HE_OK;
}
