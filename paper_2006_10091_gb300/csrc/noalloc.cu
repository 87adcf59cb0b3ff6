// noalloc.cu -- a rescale that allocates no device memory.
//
// he_rescale takes its scratch from the context's workspace, which the
// library grows with cudaMalloc (after synchronising the stream) the first
// time a call needs more.  Some callers cannot let that happen: a host that
// has handed the device's memory to its own pool and admits work against a
// fixed HBM budget (an extra cudaMalloc fails or breaks the accounting), or a
// latency-critical loop that must not hit the device-wide synchronisation an
// allocation implies.  he_rescale_noalloc runs the same kernels with its
// scratch in a static device array instead: every GPU that loads this library
// holds that array (4 MiB) until the process exits, and the entry point calls
// no cudaMalloc, cudaFree or allocating library routine.
//
// The array is shared by every call in the process.  Calls whose kernels
// overlap on the GPU (two streams, two contexts or two host threads on the
// same device at once) race on it; callers must serialise them.  Each call
// writes every scratch word it reads before reading it, so the contents left
// by an earlier call never matter and nothing needs clearing.
#include <mutex>

#include "he_ops.h"

namespace he {

// 2^19 words = 4 MiB: the rescale of one ciphertext needs 2*l*N words plus
// alignment slack (l limbs, ring degree N), e.g. l <= 15 at N = 2^14.
#define HE_NOALLOC_WORDS (1u << 19)
#define HE_NOALLOC_DEVICES 64

static __device__ __align__(256) uint64_t g_noalloc_scratch[HE_NOALLOC_WORDS];

static std::mutex g_noalloc_mu;
static uint64_t* g_noalloc_addr[HE_NOALLOC_DEVICES];

// Device address of the static array on `dev`, looked up once per device
// with that device current (the host-side symbol is not a device address).
// The cache assumes the device's primary context lives as long as the
// process: after cudaDeviceReset the cached address is stale, and this entry
// point must not be called again in that process.
static int noalloc_scratch(int dev, uint64_t** out) {
  if (dev < 0 || dev >= HE_NOALLOC_DEVICES) return fail(HE_EINVAL, "he_rescale_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    int cur = 0;
    HE_CUDA(cudaGetDevice(&cur));
    if (cur != dev) HE_CUDA(cudaSetDevice(dev));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess)
      return fail(HE_ECUDA, std::string("he_rescale_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_noalloc_addr[dev];
  return HE_OK;
}

}  // namespace he

using namespace he;

extern "C" int he_rescale_noalloc(he_ctx* c, const he_ct* a, he_ct* out) {
  if (!c || !a || !out || !a->data || !out->data) return fail(HE_EINVAL, "he_rescale_noalloc: null argument");
  if (((uintptr_t)a->data & 15) || ((uintptr_t)out->data & 15))
    return fail(HE_EINVAL, "he_rescale_noalloc: ciphertext data must be 16-byte aligned");
  const uint32_t level = a->level;
  if (level < 1 || level > (uint32_t)c->L || a->cap < level) return fail(HE_EINVAL, "he_rescale_noalloc: bad level or capacity");
  if (level < 2) return fail(HE_ELEVEL, "he_rescale_noalloc: one limb left");
  if (out->cap < level - 1) return fail(HE_EINVAL, "he_rescale_noalloc: output capacity too small");
  const size_t words = rescale_words(c, level, 1);
  if (words > HE_NOALLOC_WORDS)
    return fail(HE_EINVAL, "he_rescale_noalloc: needs " + std::to_string(words) + " scratch words (2*level*N plus slack), " +
                               "more than the static array's " + std::to_string(HE_NOALLOC_WORDS));
  uint64_t* scratch = nullptr;
  HE_TRY(noalloc_scratch(c->device, &scratch));
  Arena ar;
  ar.base = reinterpret_cast<char*>(scratch);
  ar.size = sizeof(uint64_t) * HE_NOALLOC_WORDS;
  ar.off = 0;
  const double scale = a->scale / (double)c->q[level - 1];
  // kernel timing creates CUDA events: it is suppressed for this call on this
  // thread only (the context's own setting is left alone)
  ProfSuppress quiet;
  HE_TRY(rescale_batch(c, CtBatch{a->data, 0, a->cap, 0}, level, 1, CtBatch{out->data, 0, out->cap, 0}, ar));
  out->level = level - 1;
  out->scale = scale;
  return HE_OK;
}
