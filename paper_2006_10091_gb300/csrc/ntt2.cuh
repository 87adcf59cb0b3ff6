// ntt2.cuh -- building blocks of the compile-time-shaped NTT passes, shared
// by ntt2.cu (plain transforms) and ks_fused.cu (transforms fused into key
// switching).  See ntt2.cu for the pass structure.
#pragma once
#include "he_common.cuh"

namespace he {

// A pass over tiles of 2^LOG_M transform positions x 2^LOG_K rows; each of
// the T threads holds 2^LOG_V elements in registers per round (radix 2^LOG_V).
template <int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
struct Shape {
  static constexpr int M = 1 << LOG_M, K = 1 << LOG_K, TILE = M * K, T = TILE >> LOG_V;
  static constexpr int BIT_LO = COL ? LOG_N - LOG_M : 0;  // lowest index bit this pass transforms
  static constexpr int S0 = LOG_N - BIT_LO - LOG_M;      // global stage of local stage 0
  static constexpr int TILES = 1 << (LOG_N - LOG_M - LOG_K);
  static constexpr int NTW = COL ? M : K * M;             // staged twiddle pairs
  // element (tile, k, x) -> global index
  __device__ static __forceinline__ uint32_t gidx(uint32_t tile, uint32_t k, uint32_t x) {
    const uint32_t f = (tile << LOG_K) | k;
    return COL ? ((x << BIT_LO) | f) : ((f << LOG_M) | x);
  }
  __device__ static __forceinline__ uint32_t sidx(uint32_t k, uint32_t x) {
    const uint32_t i = COL ? ((x << LOG_K) | k) : ((k << LOG_M) | x);
    return i + (i >> 3);
  }
  // staged twiddle of local stage sigma for element (k, x)
  __device__ static __forceinline__ uint32_t tidx(int sigma, uint32_t k, uint32_t x) {
    return COL ? ((1u << sigma) | (x >> (LOG_M - sigma)))
               : (uint32_t)(K * ((1 << sigma) - 1)) + (k << sigma) + (x >> (LOG_M - sigma));
  }
};

// One round: R consecutive local stages (radix 2^R) on groups of G = 2^R
// elements held in registers.  Within a group the elements sit at shared
// memory offsets j*s + (j*s >> 3) from the first (s the group's stride, a
// power of two; the padding of one word per eight never splits a group
// unevenly), so only the first offset is computed.  At stage st the group
// needs 2^st distinct twiddles, one per value of the top st bits of j; each
// is loaded once.
// `tid` is the thread's index among the T threads that share the tile (a CTA
// may hold several tiles, one per group of T threads).
template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int R, int LOG_V = 3>
__device__ __forceinline__ void round2(uint64_t* sm, const ulonglong2* stw, int sig0, uint64_t q, uint32_t tid) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  constexpr int G = 1 << R, GPT = (1 << LOG_V) >> R;
  const uint64_t q2 = q + q;
  const int lo_bits = LOG_M - sig0 - R;
  const uint32_t lo_mask = (1u << lo_bits) - 1;
  const uint32_t s = COL ? (1u << (lo_bits + LOG_K)) : (1u << lo_bits);
#pragma unroll
  for (int u = 0; u < GPT; ++u) {
    const uint32_t g = tid + u * S::T;
    uint32_t k, xhi, xlo;
    if (COL) {
      k = g & (S::K - 1);
      const uint32_t r = g >> LOG_K;
      xlo = r & lo_mask;
      xhi = r >> lo_bits;
    } else {
      xlo = g & lo_mask;
      const uint32_t r = g >> lo_bits;
      xhi = r & ((1u << sig0) - 1);
      k = r >> sig0;
    }
    const uint32_t s0 = S::sidx(k, (xhi << (LOG_M - sig0)) | xlo);
    uint64_t v[G];
#pragma unroll
    for (int j = 0; j < G; ++j) v[j] = sm[s0 + j * s + ((j * s) >> 3)];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int st = INV ? R - 1 - i : i;
      const int sg = sig0 + st, half = G >> (st + 1);
      const uint32_t tb = COL ? ((1u << sg) | (xhi << st))
                              : (uint32_t)(S::K * ((1 << sg) - 1)) + (k << sg) + (xhi << st);
#pragma unroll
      for (int b = 0; b < (1 << st); ++b) {
        const ulonglong2 w = stw[tb + b];
#pragma unroll
        for (int jj = 0; jj < half; ++jj) {
          const int j = (b << (R - st)) + jj;
          if (!INV) {
            uint64_t X = v[j];
            if (!LAZY) X = X >= q2 ? X - q2 : X;
            const uint64_t t = mul_shoup_lazy(v[j + half], w.x, w.y, q);
            v[j] = X + t;
            v[j + half] = X + q2 - t;
          } else {
            const uint64_t X = v[j], Y = v[j + half];
            uint64_t sum = X + Y;
            sum = sum >= q2 ? sum - q2 : sum;
            v[j + half] = mul_shoup_lazy(X + q2 - Y, w.x, w.y, q);
            v[j] = sum;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) sm[s0 + j * s + ((j * s) >> 3)] = v[j];
  }
}

// The same round on NT tiles of the same prime and positions at once (each
// twiddle loaded once for all of them; NT independent groups in registers).
template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int R, int NT, int LOG_V = 3>
__device__ __forceinline__ void round2_n(uint64_t* const* sms, const ulonglong2* stw, int sig0, uint64_t q,
                                         uint32_t tid) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  constexpr int G = 1 << R, GPT = (1 << LOG_V) >> R;
  const uint64_t q2 = q + q;
  const int lo_bits = LOG_M - sig0 - R;
  const uint32_t lo_mask = (1u << lo_bits) - 1;
  const uint32_t s = COL ? (1u << (lo_bits + LOG_K)) : (1u << lo_bits);
#pragma unroll
  for (int u = 0; u < GPT; ++u) {
    const uint32_t g = tid + u * S::T;
    uint32_t k, xhi, xlo;
    if (COL) {
      k = g & (S::K - 1);
      const uint32_t r = g >> LOG_K;
      xlo = r & lo_mask;
      xhi = r >> lo_bits;
    } else {
      xlo = g & lo_mask;
      const uint32_t r = g >> lo_bits;
      xhi = r & ((1u << sig0) - 1);
      k = r >> sig0;
    }
    const uint32_t s0 = S::sidx(k, (xhi << (LOG_M - sig0)) | xlo);
    uint64_t v[NT][G];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int j = 0; j < G; ++j) v[t][j] = sms[t][s0 + j * s + ((j * s) >> 3)];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int st = INV ? R - 1 - i : i;
      const int sg = sig0 + st, half = G >> (st + 1);
      const uint32_t tb = COL ? ((1u << sg) | (xhi << st))
                              : (uint32_t)(S::K * ((1 << sg) - 1)) + (k << sg) + (xhi << st);
#pragma unroll
      for (int b = 0; b < (1 << st); ++b) {
        const ulonglong2 w = stw[tb + b];
#pragma unroll
        for (int jj = 0; jj < half; ++jj) {
          const int j = (b << (R - st)) + jj;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            if (!INV) {
              uint64_t X = v[t][j];
              if (!LAZY) X = X >= q2 ? X - q2 : X;
              const uint64_t tt = mul_shoup_lazy(v[t][j + half], w.x, w.y, q);
              v[t][j] = X + tt;
              v[t][j + half] = X + q2 - tt;
            } else {
              const uint64_t X = v[t][j], Y = v[t][j + half];
              uint64_t sum = X + Y;
              sum = sum >= q2 ? sum - q2 : sum;
              v[t][j + half] = mul_shoup_lazy(X + q2 - Y, w.x, w.y, q);
              v[t][j] = sum;
            }
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int j = 0; j < G; ++j) sms[t][s0 + j * s + ((j * s) >> 3)] = v[t][j];
  }
}

// All rounds of one pass on NT tiles at once (ends with a barrier).
template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int NT, int LOG_V = 3>
__device__ __forceinline__ void run_rounds_n(uint64_t* const* sms, const ulonglong2* stw, uint64_t q, uint32_t tid) {
  constexpr int NR = (LOG_M + LOG_V - 1) / LOG_V;
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) {
    const int r = INV ? NR - 1 - rr : rr;
    const int sig0 = LOG_V * r;
    const int R = LOG_M - sig0 < LOG_V ? LOG_M - sig0 : LOG_V;
    if (R == 4) round2_n<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, (LOG_V >= 4 ? 4 : 1), NT, LOG_V>(sms, stw, sig0, q, tid);
    else if (R == 3) round2_n<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 3, NT, LOG_V>(sms, stw, sig0, q, tid);
    else if (R == 2) round2_n<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 2, NT, LOG_V>(sms, stw, sig0, q, tid);
    else round2_n<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 1, NT, LOG_V>(sms, stw, sig0, q, tid);
    __syncthreads();
  }
}

// Stage the twiddle pairs of one pass into shared memory: a column pass
// needs tw[0 .. M), a row pass for rows f0 .. f0+K-1 needs, per local stage
// sigma, the K*2^sigma entries from 2^(S0+sigma) + f0*2^sigma on.
// (Threads tid = 0 .. nthreads-1 share the copy; by default the tile's T.)
template <int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
__device__ __forceinline__ void stage_twiddles(ulonglong2* stw, const ulonglong2* tw, uint32_t tile,
                                               uint32_t tid, uint32_t nthreads) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  if (COL) {
    for (uint32_t e = tid; e < (uint32_t)S::M; e += nthreads) stw[e] = __ldg(tw + e);
  } else {
    const uint32_t f0 = tile << LOG_K;
#pragma unroll
    for (int sig = 0; sig < LOG_M; ++sig) {
      const uint32_t cnt = (uint32_t)S::K << sig;
      const uint32_t off = (uint32_t)(S::K * ((1 << sig) - 1));
      const ulonglong2* g = tw + (1u << (S::S0 + sig)) + (f0 << sig);
      for (uint32_t e = tid; e < cnt; e += nthreads) stw[off + e] = __ldg(g + e);
    }
  }
}

// The same copies as asynchronous 16-byte copies (cp_async16; the caller
// commits and waits).
template <int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
__device__ __forceinline__ void stage_twiddles_async(ulonglong2* stw, const ulonglong2* tw, uint32_t tile,
                                                     uint32_t tid, uint32_t nthreads) {
  using S = Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>;
  if (COL) {
    for (uint32_t e = tid; e < (uint32_t)S::M; e += nthreads) cp_async16(stw + e, tw + e);
  } else {
    const uint32_t f0 = tile << LOG_K;
#pragma unroll
    for (int sig = 0; sig < LOG_M; ++sig) {
      const uint32_t cnt = (uint32_t)S::K << sig;
      const uint32_t off = (uint32_t)(S::K * ((1 << sig) - 1));
      const ulonglong2* g = tw + (1u << (S::S0 + sig)) + (f0 << sig);
      for (uint32_t e = tid; e < cnt; e += nthreads) cp_async16(stw + off + e, g + e);
    }
  }
}

template <int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
__device__ __forceinline__ void stage_twiddles(ulonglong2* stw, const ulonglong2* tw, uint32_t tile) {
  stage_twiddles<LOG_N, LOG_M, LOG_K, COL, LOG_V>(stw, tw, tile, threadIdx.x,
                                                  (uint32_t)Shape<LOG_N, LOG_M, LOG_K, COL, LOG_V>::T);
}

// All rounds of one pass on the tile in shared memory (ends with a barrier).
template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
__device__ __forceinline__ void run_rounds(uint64_t* sm, const ulonglong2* stw, uint64_t q, uint32_t tid) {
  constexpr int NR = (LOG_M + LOG_V - 1) / LOG_V;
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) {
    const int r = INV ? NR - 1 - rr : rr;
    const int sig0 = LOG_V * r;
    const int R = LOG_M - sig0 < LOG_V ? LOG_M - sig0 : LOG_V;
    if (R == 4) round2<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, (LOG_V >= 4 ? 4 : 1), LOG_V>(sm, stw, sig0, q, tid);
    else if (R == 3) round2<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 3, LOG_V>(sm, stw, sig0, q, tid);
    else if (R == 2) round2<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 2, LOG_V>(sm, stw, sig0, q, tid);
    else round2<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, 1, LOG_V>(sm, stw, sig0, q, tid);
    __syncthreads();
  }
}

template <bool INV, bool LAZY, int LOG_N, int LOG_M, int LOG_K, bool COL, int LOG_V = 3>
__device__ __forceinline__ void run_rounds(uint64_t* sm, const ulonglong2* stw, uint64_t q) {
  run_rounds<INV, LAZY, LOG_N, LOG_M, LOG_K, COL, LOG_V>(sm, stw, q, threadIdx.x);
}

// Canonical residue of a forward-pass output: lazy values (< 33q) by one
// Shoup product by 1, corrected ones ([0, 4q)) by subtractions.
template <bool LAZY>
__device__ __forceinline__ uint64_t fwd_final(uint64_t v, const PrimeDev& pr) {
  const uint64_t q = pr.q, q2 = q + q;
  if (LAZY) v = mul_shoup_lazy(v, 1, pr.one_sh, q);
  else v = v >= q2 ? v - q2 : v;
  return v >= q ? v - q : v;
}

}  // namespace he
