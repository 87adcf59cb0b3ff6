// autotune.cu -- picks a context's kernel knobs by timing them on the device.
//
// The knobs never change a residue, only how the work is cut: the NTT tile
// shapes (three per ring size, shared by the plain transforms and the fused
// key-switching kernels) and how many polynomials of one limb an NTT CTA
// transforms with one staging of its twiddles.  The timed operation is the relinearisation key
// switch (iNTT, ModUp + NTT, inner product, ModDown), which carries most of
// the work of every multiplication and rotation, on `count` polynomials of
// uniform residues at `level`; each candidate runs once untimed and then
// `reps` times between CUDA events on the context's stream.
#include <cfloat>
#include <vector>

#include "he_ops.h"

namespace he {

__global__ void k_fill_uniform(uint64_t* out, size_t total, uint32_t level, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)((g / n) % level);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0x5eed, 0xa7), 0x243F6A88u, 0x85A308D3u);
    out[g] = reduce64(((uint64_t)r.x << 32 | r.y) >> 4, primes[t]);
  }
}

struct Knobs {
  int shape;
  uint32_t pb;
};

}  // namespace he

using namespace he;

extern "C" int he_autotune(he_ctx* c, uint32_t level, uint32_t count, double* best_ms) {
  if (!c) return fail(HE_EINVAL, "he_autotune: null context");
  if (level < 1 || level > (uint32_t)c->L || count < 1 || count > 4096)
    return fail(HE_EINVAL, "he_autotune: level in [1, L], count in [1, 4096]");
  const size_t n = c->n;
  const size_t words = (size_t)count * level * n;
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * (words + ks_words(c, level, count) + 2 * (size_t)count * level * n) + 16384));
  Arena ar;
  ar.base = (char*)c->ws.ptr;
  ar.size = c->ws.size;
  ar.off = 0;
  uint64_t* d = ar.take<uint64_t>(words);
  uint64_t* o = ar.take<uint64_t>((size_t)2 * count * level * n);
  Arena scratch = ar;
  k_fill_uniform<<<grid_for(words), 256, 0, c->stream>>>(d, words, level, c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  const CtBatch O{o, (uint64_t)2 * level * n, level, 0};

  std::vector<Knobs> cand;
  const bool shaped = c->log_n >= 12 && c->log_n <= 16 && !c->ntt_generic;
  for (int shape = 0; shape < (shaped ? 3 : 1); ++shape)
    for (uint32_t pb : {1u, 4u, 8u}) cand.push_back(Knobs{shape, pb});
  const Knobs saved{c->ntt_shape, c->ntt_pb_max};
  cudaEvent_t e0, e1;
  HE_CUDA(cudaEventCreate(&e0));
  HE_CUDA(cudaEventCreate(&e1));
  const int reps = 3;
  double best = DBL_MAX;
  Knobs win = saved;
  int rc = HE_OK;
  for (const Knobs& k : cand) {
    c->ntt_shape = k.shape;
    c->ntt_pb_max = k.pb;
    Arena a = scratch;
    rc = keyswitch_batch(c, d, (uint64_t)level * n, level, count, c->d_rlk, O, 0, O, a);  // warm-up
    if (rc != HE_OK) break;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && rc == HE_OK; ++r) {
      a = scratch;
      rc = keyswitch_batch(c, d, (uint64_t)level * n, level, count, c->d_rlk, O, 0, O, a);
    }
    cudaEventRecord(e1, c->stream);
    if (rc != HE_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = fail(HE_ECUDA, "he_autotune: timing failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / reps < best) {
      best = ms / reps;
      win = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->ntt_shape = rc == HE_OK ? win.shape : saved.shape;
  c->ntt_pb_max = rc == HE_OK ? win.pb : saved.pb;
  if (rc == HE_OK && best_ms) *best_ms = best;
  return rc;
}

extern "C" int he_get_tuning(he_ctx* c, const char* key, double* value) {
  if (!c || !key || !value) return fail(HE_EINVAL, "he_get_tuning: null argument");
  const std::string k(key);
  if (k == "chunk_bytes") *value = (double)c->chunk_bytes;
  else if (k == "ntt_generic") *value = c->ntt_generic ? 1.0 : 0.0;
  else if (k == "lr_chunk") *value = c->lr_chunk;
  else if (k == "ntt_shape") *value = c->ntt_shape;
  else if (k == "ntt_pb_max") *value = c->ntt_pb_max;
  else if (k == "ks_ct") *value = c->ks_ct;
  else return fail(HE_EINVAL, "unknown tuning key " + k);
  return HE_OK;
}
