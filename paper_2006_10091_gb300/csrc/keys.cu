// keys.cu -- random streams, key generation and encryption (Sec. 3:
// "Encrypt/Decrypt ... the public key and private key ... R-LWE";
// Algorithm 2: the parameter server generates the keys and encrypts).
//
// Random streams: Philox4x32-10 with key (seed low, seed high) and counter
// (coefficient index, prime index or 0, stream id, domain).  Samplers:
//  ternary  floor(3*w0/2^32) - 1;
//  Gaussian |x| = #{k < K : (w1:w0) >= T[k]} with the cumulative table T of
//           rho_k = exp(-k^2/(2 sigma^2)), sign from bit 0 of w2;
//  uniform  the 128-bit word (w3:w2:w1:w0) mod q, drawn directly in
//           evaluation form.
// Key layout: s [np][N]; pk (b, a) [2][L][N]; switching keys
// [beta][2][np][N] with b_j = -a_j s + e_j + P [t in D_j] s' on limb t < L.
#include <vector>

#include "he_internal.h"
#include "he_kernels.h"
#include "he_ops.h"

namespace he {

__device__ __forceinline__ uint32_t map_prime(uint32_t t, uint32_t level, uint32_t L) {
  return t < level ? t : L + t - level;
}

// kind 0 ternary, 1 Gaussian (both written to every limb), 2 uniform per limb.
__global__ void k_sample(uint64_t* out, uint64_t out_stride, uint32_t kind, uint32_t nl,
                         uint32_t limb0, uint32_t level, uint32_t L, uint64_t seed, uint32_t sid,
                         uint32_t dom, const uint64_t* gauss, int gK, uint32_t count, uint32_t sid_step,
                         int log_n, const PrimeDev* primes, const uint64_t* two64) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)count * n;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g % n), c = (uint32_t)(g / n);
    const uint32_t s = sid + c * sid_step;
    uint64_t* o = out + (size_t)c * out_stride + (size_t)limb0 * n + k;
    if (kind == 2) {
      for (uint32_t tl = 0; tl < nl; ++tl) {
        const uint32_t p = map_prime(limb0 + tl, level, L);
        const uint4 w = philox4x32_10(make_uint4(k, p, s, dom), k0, k1);
        const uint64_t lo = ((uint64_t)w.y << 32) | w.x, hi = ((uint64_t)w.w << 32) | w.z;
        o[(size_t)tl * n] = reduce_u128(hi, lo, primes[p], two64[p]);
      }
      continue;
    }
    const uint4 w = philox4x32_10(make_uint4(k, 0, s, dom), k0, k1);
    int64_t v;
    if (kind == 0) {
      v = (int64_t)(((uint64_t)w.x * 3) >> 32) - 1;
    } else {
      const uint64_t u = ((uint64_t)w.y << 32) | w.x;
      int m = 0;
      while (m < gK && u >= gauss[m]) ++m;
      v = (w.z & 1) ? -m : m;
    }
    for (uint32_t tl = 0; tl < nl; ++tl) {
      const uint32_t p = map_prime(limb0 + tl, level, L);
      o[(size_t)tl * n] = from_signed(v, primes[p]);
    }
  }
}

__global__ void k_signed_to_residues(const int64_t* src, uint64_t* out, uint32_t nl, int log_n,
                                     const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)nl * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(g / n), k = (uint32_t)(g % n);
    out[g] = from_signed(src[k], primes[t]);
  }
}

// Switching-key body for nb digits at once: b = e - a s (+ P s' on the digit's
// own limbs t < L); s' = s^2 when square, else sp.
__global__ void k_evk_combine(uint64_t* key, const uint64_t* e, const uint64_t* s, const uint64_t* sp,
                              int square, uint32_t nb, uint32_t alpha, uint32_t L, uint32_t np,
                              LimbConsts pmod, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)nb * np * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g % n);
    size_t r = g / n;
    const uint32_t t = (uint32_t)(r % np), j = (uint32_t)(r / np);
    const PrimeDev pr = primes[t];
    const uint64_t st = s[(size_t)t * n + k];
    const uint64_t a = key[(((size_t)j * 2 + 1) * np + t) * n + k];
    uint64_t b = sub_mod(e[((size_t)j * np + t) * n + k], mul_mod(a, st, pr), pr.q);
    if (t < L && t >= j * alpha && t < (j + 1) * alpha) {
      const uint64_t spt = square ? mul_mod(st, st, pr) : sp[(size_t)t * n + k];
      b = add_mod(b, mul_shoup(spt, pmod.w[t], pmod.wsh[t], pr.q), pr.q);
    }
    key[(((size_t)j * 2 + 0) * np + t) * n + k] = b;
  }
}

// Encryption body.  pk: out0 = v b + em, out1 = v a + e1; sk: out0 = em - a s
// (a already in out1).  em = NTT(e0 + m), v, e1 in evaluation form.
__global__ void k_enc_combine(CtBatch out, const uint64_t* v, const uint64_t* em, const uint64_t* e1,
                              const uint64_t* pk, const uint64_t* s, int use_sk, uint32_t level,
                              uint32_t L, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)level * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(g / n), k = (uint32_t)(g % n);
    const PrimeDev pr = primes[t];
    uint64_t* o0 = out.base + (size_t)t * n + k;
    uint64_t* o1 = out.base + ((size_t)out.cap + t) * n + k;
    if (use_sk) {
      *o0 = sub_mod(em[g], mul_mod(*o1, s[(size_t)t * n + k], pr), pr.q);
    } else {
      const uint64_t b = pk[(size_t)t * n + k], a = pk[((size_t)L + t) * n + k];
      *o0 = add_mod(mul_mod(v[g], b, pr), em[g], pr.q);
      *o1 = add_mod(mul_mod(v[g], a, pr), e1[g], pr.q);
    }
  }
}

__global__ void k_add_raw(const uint64_t* a, const uint64_t* b, uint64_t* o, uint32_t nl, int log_n,
                          const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)nl * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x)
    o[g] = add_mod(a[g], b[g], primes[g / n].q);
}

static int sample(he_ctx* c, uint64_t* out, uint64_t out_stride, uint32_t kind, uint32_t nl,
                  uint32_t limb0, uint32_t level, uint32_t sid, uint32_t dom, uint32_t count,
                  uint32_t sid_step) {
  const size_t work = (size_t)count * c->n;
  k_sample<<<grid_for(work), 256, 0, c->stream>>>(out, out_stride, kind, nl, limb0, level,
                                                  (uint32_t)c->L, c->prm.seed, sid, dom, c->d_gauss,
                                                  c->gK, count, sid_step, c->log_n, c->d_primes,
                                                  c->d_two64);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

static PolyBatch one_batch(const uint64_t* src, uint64_t* dst, uint64_t stride, uint32_t npolys,
                           uint32_t nl, uint32_t level) {
  PolyBatch b;
  b.src = src;
  b.dst = dst;
  b.src_stride = stride;
  b.dst_stride = stride;
  b.npolys = npolys;
  b.nl = nl;
  b.limb0 = 0;
  b.level = level;
  b.skip_alpha = 0;
  b.skip_beta = 1;
  return b;
}

// Switching key for s' (evaluation form over np primes, or s^2 if sp == NULL).
static int gen_switch_key(he_ctx* c, const uint64_t* sp, uint32_t tag, uint64_t* key) {
  const uint32_t n = c->n, np = c->np, beta = c->beta;
  const size_t words = (size_t)beta * np * n;
  HE_TRY(ws_reserve(c, words * sizeof(uint64_t)));
  uint64_t* e = (uint64_t*)c->ws.ptr;
  // a_j (uniform, evaluation form) into key[j][1]; e_j into scratch
  HE_TRY(sample(c, key + (size_t)np * n, 2ull * np * n, 2, np, 0, np, tag * 256u, DOM_EVK_A, beta, 1));
  HE_TRY(sample(c, e, (size_t)np * n, 1, np, 0, np, tag * 256u, DOM_EVK_E, beta, 1));
  HE_TRY(ntt_forward(c, one_batch(e, e, (size_t)np * n, beta, np, np)));
  LimbConsts pm;
  for (int t = 0; t < c->L; ++t) {
    pm.w[t] = c->P_mod_q[t];
    pm.wsh[t] = h_shoup(c->P_mod_q[t], c->q[t]);
  }
  k_evk_combine<<<grid_for(words), 256, 0, c->stream>>>(key, e, c->d_s, sp, sp == nullptr, beta,
                                                        (uint32_t)c->alpha, (uint32_t)c->L, np, pm,
                                                        c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int keygen(he_ctx* c, const std::vector<int32_t>& rots) {
  const uint32_t n = c->n, np = c->np, L = c->L;
  HE_CUDA(cudaMalloc(&c->d_s, sizeof(uint64_t) * np * n));
  HE_CUDA(cudaMalloc(&c->d_pk, sizeof(uint64_t) * 2 * L * n));
  HE_CUDA(cudaMalloc(&c->d_rlk, sizeof(uint64_t) * c->key_words()));
  // secret: ternary coefficients on every prime, to evaluation form
  HE_TRY(sample(c, c->d_s, 0, 0, np, 0, np, 0, DOM_S, 1, 0));
  HE_TRY(ntt_forward(c, one_batch(c->d_s, c->d_s, 0, 1, np, np)));
  // public key (b, a): a uniform in evaluation form, b = -a s + e
  {
    HE_TRY(ws_reserve(c, sizeof(uint64_t) * L * n));
    uint64_t* e = (uint64_t*)c->ws.ptr;
    HE_TRY(sample(c, c->d_pk + (size_t)L * n, 0, 2, L, 0, L, 0, DOM_PK_A, 1, 0));
    HE_TRY(sample(c, e, 0, 1, L, 0, L, 0, DOM_PK_E, 1, 0));
    HE_TRY(ntt_forward(c, one_batch(e, e, 0, 1, L, L)));
    // b = e - a s with the switching-key combine on a single "digit" that owns no limb
    LimbConsts pm;
    for (uint32_t t = 0; t < L; ++t) { pm.w[t] = 0; pm.wsh[t] = 0; }
    // reuse k_evk_combine with np := L, alpha := 0 (no digit limbs): key = [1][2][L][N]
    k_evk_combine<<<grid_for((size_t)L * n), 256, 0, c->stream>>>(c->d_pk, e, c->d_s, nullptr, 0, 1, 0,
                                                                  L, L, pm, c->log_n, c->d_primes);
    HE_CUDA(cudaGetLastError());
  }
  HE_TRY(gen_switch_key(c, nullptr, 0, c->d_rlk));
  // Galois keys: s' = kappa_g(s)
  uint64_t* sg = nullptr;
  HE_CUDA(cudaMalloc(&sg, sizeof(uint64_t) * np * n));
  for (int32_t r : rots) {
    const uint64_t g = h_galois_elt(c->log_n, r);
    if (g == 1 || c->gal.count(g)) continue;
    CtBatch in{c->d_s, 0, np, 0}, out{sg, 0, np, 0};
    k_automorph<<<grid_for((size_t)np * n), 256, 0, c->stream>>>(in, out, 1, np, g, 1, c->log_n);
    HE_CUDA(cudaGetLastError());
    uint64_t* key = nullptr;
    if (cudaMalloc(&key, sizeof(uint64_t) * c->key_words()) != cudaSuccess) {
      cudaFree(sg);
      return fail(HE_ENOMEM, "Galois key allocation failed");
    }
    c->gal[g] = key;
    HE_TRY(gen_switch_key(c, sg, (uint32_t)g, key));
  }
  HE_CUDA(cudaStreamSynchronize(c->stream));
  cudaFree(sg);
  return HE_OK;
}

// Encrypt integer coefficients already on the device (d_m, N int64).
// scratch: 4 * level * N words.
int encrypt_dev(he_ctx* c, const int64_t* d_m, uint32_t level, int use_sk, uint32_t cid, he_ct* out,
                uint64_t* scratch) {
  const uint32_t n = c->n, L = c->L;
  const size_t lw = (size_t)level * n;
  uint64_t* M = scratch;
  uint64_t* E0 = M + lw;
  uint64_t* V = E0 + lw;
  uint64_t* E1 = V + lw;
  k_signed_to_residues<<<grid_for(lw), 256, 0, c->stream>>>(d_m, M, level, c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  HE_TRY(sample(c, E0, 0, 1, level, 0, L, cid, DOM_ENC_E0, 1, 0));
  k_add_raw<<<grid_for(lw), 256, 0, c->stream>>>(E0, M, E0, level, c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  HE_TRY(ntt_forward(c, one_batch(E0, E0, 0, 1, level, L)));
  CtBatch o{out->data, 0, out->cap, 0};
  if (use_sk) {
    HE_TRY(sample(c, out->data + (size_t)out->cap * n, 0, 2, level, 0, L, cid, DOM_ENC_A, 1, 0));
  } else {
    HE_TRY(sample(c, V, 0, 0, level, 0, L, cid, DOM_ENC_V, 1, 0));
    HE_TRY(sample(c, E1, 0, 1, level, 0, L, cid, DOM_ENC_E1, 1, 0));
    HE_TRY(ntt_forward(c, one_batch(V, V, 0, 1, level, L)));
    HE_TRY(ntt_forward(c, one_batch(E1, E1, 0, 1, level, L)));
  }
  k_enc_combine<<<grid_for(lw), 256, 0, c->stream>>>(o, V, E0, E1, c->d_pk, c->d_s, use_sk, level, L,
                                                     c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  out->level = level;
  return HE_OK;
}

}  // namespace he
