// ntt2_impl.cuh -- the two-pass NTT for N = 2^12 .. 2^16 with compile-time tile
// shapes.  Same transform, same output as ntt.cu (slot j = value at
// psi^(2*brv(j)+1)); what differs is how a pass runs:
//  * each CTA first copies the twiddle pairs (value, Shoup companion) its
//    stages will use into shared memory with coalesced loads -- a column
//    pass (the top index bits) needs tw[1 .. 2^m), a row pass for its K
//    consecutive rows needs K*2^sigma consecutive entries per local stage
//    sigma -- so every butterfly reads its twiddle from shared memory;
//  * tile shapes are template parameters, so index arithmetic is shifts by
//    constants;
//  * forward transforms over primes below 2^58 skip Harvey's per-stage
//    correction: with Shoup products in [0, 2q) a value grows by at most 2q
//    per stage, so after the n <= 16 stages it stays below 33q < 2^64; the
//    last pass reduces once (a Shoup product by 1, then one subtraction).
//    Larger primes keep the corrected butterfly ([0, 4q)).
#pragma once
#include <algorithm>

#include "he_internal.h"
#include "ntt2.cuh"

namespace he {

struct Ntt2Args {
  const uint64_t* src;
  uint64_t* dst;
  uint64_t src_stride, dst_stride;
  uint32_t nl, limb0, level, L;
  uint32_t np, pb;  // polynomials; polynomials per CTA (same limb, so same twiddles)
  uint32_t skip_alpha, skip_beta;
  uint64_t gal;  // first pass: load the source through the automorphism X -> X^gal (0: none)
  const ulonglong2* tw;
  const PrimeDev* primes;
  int last;
};

template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V>
__device__ __forceinline__ void pass_body(const Ntt2Args& a, uint64_t* sm, ulonglong2* stw, uint32_t tile,
                                          const uint64_t* src, uint64_t* dst, const PrimeDev& pr) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  const uint64_t q = pr.q;
  run_rounds<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, LOG_V>(sm, stw, q);
#pragma unroll 4
  for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
    uint32_t k, x;
    if (COL) { x = idx >> LOG_K; k = idx & (S::K - 1); }
    else { k = idx >> LOG_M; x = idx & (S::M - 1); }
    uint64_t v = sm[idx + (idx >> 3)];
    if (a.last) {
      if (INV) {
        v = mul_shoup_lazy(v, pr.n_inv, pr.n_inv_sh, q);
        v = v >= q ? v - q : v;
      } else {
        v = fwd_final<LAZY>(v, pr);
      }
    }
    dst[S::gidx(tile, k, x)] = v;
  }
}

template <bool INV, int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V>
__global__ void __launch_bounds__((1 << (LOG_M + LOG_K)) >> LOG_V) ntt2_kernel(Ntt2Args a) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  const uint32_t tile = blockIdx.x % S::TILES;
  const uint32_t bl = blockIdx.x / S::TILES;
  const uint32_t li = bl % a.nl, pg = bl / a.nl;
  const uint32_t t = a.limb0 + li;
  const uint32_t prime = t < a.level ? t : a.L + t - a.level;
  const PrimeDev pr = a.primes[prime];
  const ulonglong2* tw = a.tw + (size_t)prime * (1u << LOG_N);
  stage_twiddles<LOG_N, LOG_M, LOG_K, COL, LOG_V>(stw, tw, tile);
  const uint32_t p1 = min(pg * a.pb + a.pb, a.np);
  for (uint32_t p = pg * a.pb; p < p1; ++p) {
    if (a.skip_alpha) {
      const uint32_t j = p % a.skip_beta, lo = j * a.skip_alpha;
      const uint32_t hi = min(lo + a.skip_alpha, a.level);
      if (t >= lo && t < hi) continue;
    }
    const uint64_t* src = a.src + p * a.src_stride + (size_t)li * (1u << LOG_N);
    uint64_t* dst = a.dst + p * a.dst_stride + (size_t)li * (1u << LOG_N);
    // stage the data tile (each thread rewrites only the words it wrote out
    // in the previous iteration, so no barrier is needed before this)
#pragma unroll 4
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
      uint32_t k, x;
      if (COL) { x = idx >> LOG_K; k = idx & (S::K - 1); }
      else { k = idx >> LOG_M; x = idx & (S::M - 1); }
      const uint32_t e = S::gidx(tile, k, x);
      sm[idx + (idx >> 3)] = __ldg(src + (a.gal ? automorph_src(e, a.gal, LOG_N) : e));
    }
    __syncthreads();
    if (!INV && pr.q < (1ull << 58))
      pass_body<INV, true, LOG_N, LOG_M, LOG_K, COL, LOG_V>(a, sm, stw, tile, src, dst, pr);
    else
      pass_body<INV, false, LOG_N, LOG_M, LOG_K, COL, LOG_V>(a, sm, stw, tile, src, dst, pr);
  }
}

template <bool INV, int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V>
int launch2(he_ctx* c, const PolyBatch& b, const uint64_t* src, uint64_t* dst, uint64_t src_stride,
                   bool last, uint64_t gal = 0) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  Ntt2Args a;
  a.gal = gal;
  a.src = src;
  a.dst = dst;
  a.src_stride = src_stride;
  a.dst_stride = b.dst_stride;
  a.nl = b.nl;
  a.limb0 = b.limb0;
  a.level = b.level;
  a.L = (uint32_t)c->L;
  a.skip_alpha = b.skip_alpha;
  a.skip_beta = b.skip_beta ? b.skip_beta : 1;
  a.tw = reinterpret_cast<const ulonglong2*>(INV ? c->d_itw : c->d_tw);
  a.primes = c->d_primes;
  a.last = last ? 1 : 0;
  const size_t smem = sizeof(ulonglong2) * S::NTW + sizeof(uint64_t) * (S::TILE + S::TILE / 8);
  static std::atomic<unsigned long long> attr{0};  // per instantiation: one bit per device
  HE_TRY(set_smem_attr_once(attr, c->device, (const void*)ntt2_kernel<INV, LOG_N, LOG_M, LOG_K, COL, LOG_V>, smem));
  // several polynomials of one limb per CTA share its staged twiddles, as
  // long as the grid keeps about four waves of CTAs
  const size_t tiles = (size_t)b.npolys * b.nl * S::TILES;
  const size_t pb = std::max<size_t>(1, std::min<size_t>(c->ntt_pb_max, tiles / (4 * 4 * 152)));
  a.np = b.npolys;
  a.pb = (uint32_t)pb;
  const size_t blocks = (size_t)((b.npolys + pb - 1) / pb) * b.nl * S::TILES;
  if (blocks == 0) return HE_OK;
  if (blocks > 0x7fffffffull) return fail(HE_EINVAL, "NTT batch too large");
  double transforms = (double)b.npolys * b.nl;
  if (b.skip_alpha && c->prof_on) {
    transforms = 0;
    for (uint32_t p = 0; p < b.npolys; ++p) {
      const uint32_t j = p % a.skip_beta, lo = j * b.skip_alpha, hi = min(lo + b.skip_alpha, b.level);
      uint32_t skipped = 0;
      for (uint32_t t = b.limb0; t < b.limb0 + b.nl; ++t) skipped += (t >= lo && t < hi);
      transforms += b.nl - skipped;
    }
  }
  const double nn = (double)(1u << LOG_N);
  // work: the butterflies, and the inverse's scaling by N^-1 in its last pass
  const double scale = INV && last ? transforms * nn : 0.0;
  ProfScope prof(c, INV ? "intt" : "ntt", transforms * nn / 2 * LOG_M + scale, transforms * nn * 16, 0.0,
                 transforms * nn / 2 * LOG_M);
  ntt2_kernel<INV, LOG_N, LOG_M, LOG_K, COL, LOG_V><<<(unsigned)blocks, S::T, smem, c->stream>>>(a);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// Forward: column pass over the top n1 bits, then row pass; inverse: the
// reverse.  Returns 1 if N has no compiled shape (the caller falls back).
template <bool INV, int LOG_N, int M1, int K1, int M2, int K2, int LOG_V>
int run2(he_ctx* c, const PolyBatch& b) {
  if (!INV) {
    const int rc = launch2<false, LOG_N, M1, K1, true, LOG_V>(c, b, b.src, b.dst, b.src_stride, false);
    return rc != HE_OK ? rc : launch2<false, LOG_N, M2, K2, false, LOG_V>(c, b, b.dst, b.dst, b.dst_stride, true);
  }
  const int rc = launch2<true, LOG_N, M2, K2, false, LOG_V>(c, b, b.src, b.dst, b.src_stride, false, b.gal);
  return rc != HE_OK ? rc : launch2<true, LOG_N, M1, K1, true, LOG_V>(c, b, b.dst, b.dst, b.dst_stride, true);
}

template <int LOG_N, int M1, int K1, int M2, int K2, int LOG_V = 3>
int run2_dir(he_ctx* c, const PolyBatch& b, bool inv) {
  return inv ? run2<true, LOG_N, M1, K1, M2, K2, LOG_V>(c, b) : run2<false, LOG_N, M1, K1, M2, K2, LOG_V>(c, b);
}

// Only the first pass (the row pass) of the inverse transform: the fused
// key switch runs the column pass itself on the tiles it converts.
template <int LOG_N, int M1, int K1, int M2, int K2, int LOG_V = 3>
int run2_inv_rows(he_ctx* c, const PolyBatch& b) {
  return launch2<true, LOG_N, M2, K2, false, LOG_V>(c, b, b.src, b.dst, b.src_stride, false, b.gal);
}

// Per ring size (ntt2_n12.cu .. ntt2_n16.cu, compiled in parallel): both
// passes, or the inverse's first pass only, for the tile shape c->ntt_shape.
#define HE_NTT2_DECL(NN)                                          \
  int ntt2_n##NN(he_ctx* c, const PolyBatch& b, bool inv);          \
  int ntt2_inv_rows_n##NN(he_ctx* c, const PolyBatch& b);
HE_NTT2_DECL(12)
HE_NTT2_DECL(13)
HE_NTT2_DECL(14)
HE_NTT2_DECL(15)
HE_NTT2_DECL(16)
#undef HE_NTT2_DECL

}  // namespace he
