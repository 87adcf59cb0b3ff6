// ks_fused.cuh -- hybrid key switching with ModUp fused into the NTT's first
// pass and the key inner product fused into its second pass (N = 2^12 ..
// 2^16).  Same arithmetic and the same residues as the unfused sequence in
// ops.cu (iNTT, k_modup, NTT, k_inner_product); what it saves is the round
// trips of the converted digits through memory:
//  * ks_modup_col: a CTA of digit j and target limb t builds its column tile
//    straight from the coefficient-form input (the digit's limbs, converted
//    to prime t as in k_modup) and runs the column pass; the ModUp output is
//    never written;
//  * ks_row_rot: a CTA of target limb t and two rows finishes the row pass of
//    every digit's tile (or, on the digit's own limb, reads the input as it
//    is), keeps the tiles in shared memory and adds their products with the
//    key polynomials of each rotation (a plain key switch is one rotation by
//    the identity); the transformed digits are never written.  The products
//    are summed as split sums of 32 x 32 -> 64-bit products on primes that
//    allow it (mac_split3) and as 128-bit multiply-accumulates otherwise.
#pragma once
#include <algorithm>
#include <atomic>
#include "he_ops.h"
#include "ntt2.cuh"

namespace he {

// Dynamic shared memory the all-targets conversion kernels may take.
constexpr size_t kModupAllSmem = 160 * 1024;
// ... and the hoisted rotate-and-sum's row pass (every digit's tile).
constexpr size_t kRotSmemMax = 200 * 1024;

struct KsFusedArgs {
  const uint64_t* d;     // input, evaluation form: count x [level][N] at d_stride
  const uint64_t* d2c;   // input, coefficient form: count x [level][N]
  uint64_t* ext;         // column-pass outputs: count x [beta][nt][N]
  uint64_t* acc;         // accumulators: count x [2][nt][N]
  const uint64_t* evk;   // [beta_top][2][np][N]
  uint64_t d_stride;
  uint64_t gal;            // d is read through the automorphism X -> X^gal (0: none)
  uint32_t level, alpha, beta, L, np, nt;
  const PrimeDev* primes;
  const ulonglong2* tw;
  const ulonglong2* itw;   // inverse twiddles
  int half;                // d2c holds the inverse transform's row pass only (ks_modup_col_all finishes it)
  const uint64_t* consts;  // ModUp constant tables
  uint32_t lo[HE_MAX_PRIMES], cnt[HE_MAX_PRIMES];
  uint64_t off[HE_MAX_PRIMES];
};

__host__ __device__ __forceinline__ uint32_t ks_prime(uint32_t t, uint32_t level, uint32_t L) {
  return t < level ? t : L + t - level;
}

// The basis conversion of one tile into shared memory: for the T threads'
// elements idx of the tile, sum over u < CNT of wv[u][idx] times the constant
// (w[u * stride], its Shoup companion), reduced to [0, q); the CNT constants
// sit in registers for the whole tile.  With vv (ModDown's exact lift), the
// element's multiple of P and h are then subtracted in the same pass:
// - vP[vv[idx]] - h mod q.
template <int TILE, int T, int CNT>
__device__ __forceinline__ void conv_sum_tile(uint64_t* sm, const uint64_t* wv, const uint64_t* w, const uint64_t* wsh,
                                              uint32_t stride, uint64_t q, const uint32_t* vv = nullptr,
                                              const uint64_t* vP = nullptr, uint64_t h = 0) {
  uint64_t cw[CNT], cs[CNT];
#pragma unroll
  for (int u = 0; u < CNT; ++u) {
    cw[u] = w[(size_t)u * stride];
    cs[u] = wsh[(size_t)u * stride];
  }
  const uint64_t q2 = q + q;
#pragma unroll 2
  for (uint32_t idx = threadIdx.x; idx < (uint32_t)TILE; idx += T) {
    uint64_t y = 0;
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
      y += mul_shoup_lazy(wv[(size_t)u * TILE + idx], cw[u], cs[u], q);
      y = y >= q2 ? y - q2 : y;
    }
    y = y >= q ? y - q : y;
    if (vv) y = sub_mod(sub_mod(y, vP[vv[idx]], q), h, q);
    sm[idx + (idx >> 3)] = y;
  }
}

// Column pass with the ModUp conversion in its load.  Grid: count * beta * nt * TILES.
template <int LOG_N, int LOG_M, int LOG_K>
__global__ void __launch_bounds__((1 << (LOG_M + LOG_K)) / 8) ks_modup_col(KsFusedArgs a) {
  using S = Shape<LOG_N, LOG_M, LOG_K, true>;
  constexpr uint32_t N = 1u << LOG_N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  uint32_t b = blockIdx.x;
  const uint32_t tile = b % S::TILES;
  b /= S::TILES;
  const uint32_t t = b % a.nt;
  b /= a.nt;
  const uint32_t j = b % a.beta, i = b / a.beta;
  const uint32_t lo = a.lo[j], cnt = a.cnt[j];
  if (t >= lo && t < lo + cnt) return;  // the digit's own limbs are used as they are
  const uint32_t prime = ks_prime(t, a.level, a.L);
  const PrimeDev pr = a.primes[prime];
  stage_twiddles<LOG_N, LOG_M, LOG_K, true>(stw, a.tw + (size_t)prime * N, tile);
  const uint64_t* tab = a.consts + a.off[j];
  const uint64_t* mat = tab + 2 * cnt;
  const uint64_t* mat_sh = mat + (size_t)cnt * a.np;
  const uint64_t* x = a.d2c + (size_t)i * a.level * N;
  const uint64_t q2 = pr.q + pr.q;
#pragma unroll 2
  for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
    const uint32_t xx = idx >> LOG_K, k = idx & (S::K - 1);
    const uint32_t e = S::gidx(tile, k, xx);
    uint64_t y;
    if (cnt == 1) {
      y = reduce64(__ldg(x + (size_t)lo * N + e), pr);  // Q_j / q_lo = 1
    } else {
      // products by the constant (Q_j/q_i) mod q_t are Shoup products in [0, 2q), kept in [0, 2q)
      y = 0;
      for (uint32_t u = 0; u < cnt; ++u) {
        const uint64_t qa = a.primes[lo + u].q;
        const uint64_t v = mul_shoup(__ldg(x + (size_t)(lo + u) * N + e), tab[2 * u], tab[2 * u + 1], qa);
        y += mul_shoup_lazy(v, mat[(size_t)u * a.np + prime], mat_sh[(size_t)u * a.np + prime], pr.q);
        y = y >= q2 ? y - q2 : y;
      }
      y = y >= pr.q ? y - pr.q : y;
    }
    sm[idx + (idx >> 3)] = y;
  }
  __syncthreads();
  uint64_t* out = a.ext + (((size_t)i * a.beta + j) * a.nt + t) * N;
  if (pr.q < (1ull << 58)) run_rounds<false, true, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
  else run_rounds<false, false, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
#pragma unroll 8
  for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
    const uint32_t xx = idx >> LOG_K, k = idx & (S::K - 1);
    out[S::gidx(tile, k, xx)] = sm[idx + (idx >> 3)];
  }
}

// The same column pass for every target limb of one digit and tile in one
// CTA: the digit's limbs are read once and their products by
// (Q_j/q_i)^-1 mod q_i (or, for a one-limb digit, the limb itself) are kept
// in shared memory for all targets.  Grid: count * beta * TILES; dynamic
// shared memory holds cnt_max * TILE more words.
template <int LOG_N, int LOG_M, int LOG_K>
__global__ void __launch_bounds__((1 << (LOG_M + LOG_K)) / 8) ks_modup_col_all(KsFusedArgs a) {
  using S = Shape<LOG_N, LOG_M, LOG_K, true>;
  constexpr uint32_t N = 1u << LOG_N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  uint64_t* wv = sm + S::TILE + S::TILE / 8;  // [cnt][TILE]
  uint32_t b = blockIdx.x;
  const uint32_t tile = b % S::TILES;
  b /= S::TILES;
  const uint32_t j = b % a.beta, i = b / a.beta;
  const uint32_t lo = a.lo[j], cnt = a.cnt[j];
  const uint64_t* tab = a.consts + a.off[j];
  const uint64_t* mat = tab + 2 * cnt;
  const uint64_t* mat_sh = mat + (size_t)cnt * a.np;
  const uint64_t* x = a.d2c + (size_t)i * a.level * N;
  for (uint32_t u = 0; u < cnt; ++u) {
    const PrimeDev pa = a.primes[lo + u];
    if (a.half) {
      // the inverse transform's column pass on this tile, then the scaling by N^-1
      stage_twiddles<LOG_N, LOG_M, LOG_K, true>(stw, a.itw + (size_t)(lo + u) * N, tile);
#pragma unroll 8
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
        const uint32_t e = S::gidx(tile, idx & (S::K - 1), idx >> LOG_K);
        sm[idx + (idx >> 3)] = __ldg(x + (size_t)(lo + u) * N + e);
      }
      __syncthreads();
      run_rounds<true, false, LOG_N, LOG_M, LOG_K, true>(sm, stw, pa.q);
    }
    if (a.half) {  // the scaling by N^-1 and the product by (Q_j/q_i)^-1 as one constant
      const uint64_t* tabn = mat_sh + (size_t)cnt * a.np;
      const uint64_t w = tabn[2 * u], wsh = tabn[2 * u + 1];
#pragma unroll 8
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T)
        wv[(size_t)u * S::TILE + idx] = mul_shoup(sm[idx + (idx >> 3)], w, wsh, pa.q);
    } else {
#pragma unroll 8
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
        const uint32_t e = S::gidx(tile, idx & (S::K - 1), idx >> LOG_K);
        const uint64_t xv = __ldg(x + (size_t)(lo + u) * N + e);
        wv[(size_t)u * S::TILE + idx] = cnt == 1 ? xv : mul_shoup(xv, tab[2 * u], tab[2 * u + 1], pa.q);
      }
    }
    // the next limb's staging overwrites stw and sm: wait for every thread
    __syncthreads();
  }
  for (uint32_t t = 0; t < a.nt; ++t) {
    if (t >= lo && t < lo + cnt) continue;  // the digit's own limbs are used as they are
    const uint32_t prime = ks_prime(t, a.level, a.L);
    const PrimeDev pr = a.primes[prime];
    const uint64_t q2 = pr.q + pr.q;
    // the previous target's rounds ended with a barrier, and its write-out
    // reads only the words each thread rewrites below
    stage_twiddles<LOG_N, LOG_M, LOG_K, true>(stw, a.tw + (size_t)prime * N, tile);
    // Shoup products by (Q_j/q_i) mod q_t, the digit's limb count a compile-time
    // constant for the usual digit sizes
    if (cnt == 2) conv_sum_tile<S::TILE, S::T, 2>(sm, wv, mat + prime, mat_sh + prime, a.np, pr.q);
    else if (cnt == 3) conv_sum_tile<S::TILE, S::T, 3>(sm, wv, mat + prime, mat_sh + prime, a.np, pr.q);
    else if (cnt == 4) conv_sum_tile<S::TILE, S::T, 4>(sm, wv, mat + prime, mat_sh + prime, a.np, pr.q);
    else
#pragma unroll 2
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
        uint64_t y;
        if (cnt == 1) {
          y = reduce64(wv[idx], pr);  // Q_j / q_lo = 1
        } else {  // kept in [0, 2q)
          y = 0;
          for (uint32_t u = 0; u < cnt; ++u) {
            y += mul_shoup_lazy(wv[(size_t)u * S::TILE + idx], mat[(size_t)u * a.np + prime],
                                mat_sh[(size_t)u * a.np + prime], pr.q);
            y = y >= q2 ? y - q2 : y;
          }
          y = y >= pr.q ? y - pr.q : y;
        }
        sm[idx + (idx >> 3)] = y;
      }
    __syncthreads();
    uint64_t* out = a.ext + (((size_t)i * a.beta + j) * a.nt + t) * N;
    if (pr.q < (1ull << 58)) run_rounds<false, true, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
    else run_rounds<false, false, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
#pragma unroll 8
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
      const uint32_t xx = idx >> LOG_K, k = idx & (S::K - 1);
      out[S::gidx(tile, k, xx)] = sm[idx + (idx >> 3)];
    }
  }
}

// ---- hoisted rotate-and-sum ------------------------------------------------
// The rotations of one rotate-and-sum stage share the decomposition of the
// input: the column pass (ks_modup_col[_all], run once) and the row pass of
// every digit.  Rotation r then needs the products of the permuted digits,
//   acc_r[e] = sum_j D_j[src_r(e)] * evk_r[j][e],  src_r = automorph_src(., gal_r),
// with a permutation of the evaluation points that maps rows to rows: in
// bit-reversed order a row of M points is a residue class of the natural
// index modulo N/M, and X -> X^gal maps residue classes onto residue
// classes.  So the CTA that holds input row c after the row pass can write
// the whole of output row c' = src_{gal^-1}(c M) / M with coalesced stores and
// key loads, reading its sources from shared memory.  When every rotation
// maps each CTA's rows onto themselves, a thread sums all rotations for its
// own positions; otherwise each rotation's row is added atomically to the
// one accumulator (64-bit sums of at most 16 residues below 2^60).
struct KsRotArgs {
  KsFusedArgs k;           // k.acc: the accumulator (summed over the rotations)
  uint32_t nrot, count;
  int closed;              // every rotation maps each tile's rows onto themselves
  uint64_t gal[HE_MAX_ROT], gal_inv[HE_MAX_ROT];
  const uint64_t* evk[HE_MAX_ROT];
  // part 0 of the input (evaluation form, count x [level][N] at c0_stride):
  // when set, part 0 of the accumulator's limbs q_t also receives
  // (P mod q_t) * sum_r kappa_r(c0), which the ModDown turns into
  // sum_r kappa_r(c0) exactly (nullptr: not added; closed stages whose
  // target limbs q_t all take the split sums only)
  const uint64_t* c0;
  uint64_t c0_stride;
};

// Grid: nt * ceil(count / CT) * TILES, target limb slowest and row tile
// fastest, so that the CTAs resident at one time share their keys (one limb
// of each rotation's key) in L2 and finish each ciphertext's limb together.
// A CTA holds CT ciphertexts of one limb and tile: group g of T threads runs
// the row passes of ciphertext i0 + g, and in a closed stage every thread
// then sums the products for its positions of all CT ciphertexts, so each
// key word it loads serves CT ciphertexts (8/CT bytes of key per key
// product).  CT > 1 only for closed stages; a tail CTA repeats its last
// ciphertext in the groups beyond the count and stores nothing for them.
// Shared memory: the tile's twiddles, every digit's transformed tile of each
// ciphertext ([CT][beta][TILE + TILE/8] words) and, with ra.c0, each
// ciphertext's part-0 tile ([CT][TILE + TILE/8]).
template <int LOG_N, int LOG_M, int LOG_K, int CT>
__global__ void __launch_bounds__(CT * ((1 << (LOG_M + LOG_K)) / 8), 4 / CT) ks_row_rot(KsRotArgs ra) {
  using S = Shape<LOG_N, LOG_M, LOG_K, false>;
  constexpr uint32_t N = 1u << LOG_N;
  constexpr int PER = S::TILE / S::T;  // 8
  constexpr uint32_t TW = S::TILE + S::TILE / 8;
  static_assert(CT == 1 || CT == 2 || CT == 4, "ciphertexts per CTA");
  const KsFusedArgs& a = ra.k;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* dig = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  uint32_t b = blockIdx.x;
  const uint32_t tile = b % S::TILES;
  b /= S::TILES;
  const uint32_t ngrp = (ra.count + CT - 1) / CT;
  const uint32_t i0 = (b % ngrp) * CT, t = b / ngrp;
  const uint32_t grp = CT == 1 ? 0u : threadIdx.x / S::T;  // warp-uniform: T is a multiple of 32
  const uint32_t ltid = CT == 1 ? threadIdx.x : threadIdx.x % S::T;
  const uint32_t i = min(i0 + grp, ra.count - 1);
  const uint32_t prime = ks_prime(t, a.level, a.L);
  const PrimeDev pr = a.primes[prime];
  const uint64_t q = pr.q;
  const bool lazy = q < (1ull << 58);
  // the input's part 0, added through each rotation on the limbs q_t
  const bool add_c0 = ra.c0 && t < a.level;
  uint64_t* c0s = dig + (size_t)CT * a.beta * TW;  // its tiles, [CT][TW] after every digit tile
  // 1. every digit's tile in evaluation form, canonical residues: the
  // twiddles and all digit tiles are copied asynchronously up front (one
  // group each, part 0's tile with the last), so that later tiles arrive
  // while earlier ones transform
  stage_twiddles_async<LOG_N, LOG_M, LOG_K, false>(stw, a.tw + (size_t)prime * N, tile, threadIdx.x, CT * S::T);
  cp_async_commit();
  for (uint32_t j = 0; j < a.beta; ++j) {
    uint64_t* sm = dig + ((size_t)grp * a.beta + j) * TW;
    const bool own = t >= a.lo[j] && t < a.lo[j] + a.cnt[j];
    const uint64_t* src = own ? a.d + (size_t)i * a.d_stride + (size_t)t * N
                              : a.ext + (((size_t)i * a.beta + j) * a.nt + t) * N;
    // the own limb is read through the input's automorphism (a single
    // rotation's key switch: the converted tiles already are)
    const uint64_t in_gal = own ? a.gal : 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = ltid + u * S::T;
      const uint32_t e = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
      cp_async8(sm + idx + (idx >> 3), src + (in_gal ? automorph_src(e, in_gal, LOG_N) : e));
    }
    if (add_c0 && j + 1 == a.beta) {
      const uint64_t* s0 = ra.c0 + (size_t)i * ra.c0_stride + (size_t)t * N;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const uint32_t idx = ltid + u * S::T;
        cp_async8(c0s + (size_t)grp * TW + idx + (idx >> 3), s0 + S::gidx(tile, idx >> LOG_M, idx & (S::M - 1)));
      }
    }
    cp_async_commit();
  }
  // the converted digits' row passes, two tiles at a time (one barrier per
  // round for both, each twiddle loaded once for both)
  auto finish_tile = [&](uint64_t* sm) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = ltid + u * S::T;
      const uint64_t v = sm[idx + (idx >> 3)];
      sm[idx + (idx >> 3)] = lazy ? fwd_final<true>(v, pr) : fwd_final<false>(v, pr);
    }
  };
  int pend = -1;  // a converted digit waiting for a partner
  for (uint32_t j = 0; j < a.beta; ++j) {
    const bool own = t >= a.lo[j] && t < a.lo[j] + a.cnt[j];
    if (own) continue;
    if (pend < 0) {
      pend = (int)j;
      continue;
    }
    cp_async_wait_dyn(a.beta - 1 - j);  // the twiddles and tiles 0 .. j have arrived
    __syncthreads();
    uint64_t* sms[2] = {dig + ((size_t)grp * a.beta + (uint32_t)pend) * TW, dig + ((size_t)grp * a.beta + j) * TW};
    if (lazy) run_rounds_n<false, true, LOG_N, LOG_M, LOG_K, false, 2>(sms, stw, q, ltid);
    else run_rounds_n<false, false, LOG_N, LOG_M, LOG_K, false, 2>(sms, stw, q, ltid);
    finish_tile(sms[0]);
    finish_tile(sms[1]);
    pend = -1;
  }
  if (pend >= 0) {
    uint64_t* sm = dig + ((size_t)grp * a.beta + (uint32_t)pend) * TW;
    cp_async_wait_dyn(a.beta - 1 - (uint32_t)pend);
    __syncthreads();
    if (lazy) run_rounds<false, true, LOG_N, LOG_M, LOG_K, false>(sm, stw, q, ltid);
    else run_rounds<false, false, LOG_N, LOG_M, LOG_K, false>(sm, stw, q, ltid);
    finish_tile(sm);
  }
  cp_async_wait<0>();  // the own limb's tile
  __syncthreads();
  // 2. the products of the permuted digits with each rotation's key, summed
  // exactly (split sums or 128-bit sums) and reduced once per residue
  const uint32_t row0 = (uint32_t)tile << LOG_K;
  // key products as split sums (mac_split3) when the prime and the number of
  // summed terms allow it
  const uint32_t sb = (pr.k + 1) >> 1;
  if (ra.closed && 2 * sb + 2 + (32 - __clz(ra.nrot * a.beta)) <= 64) {
    // one pair of neighbouring positions per pass, all CT ciphertexts with
    // each key load
    constexpr int PPT = PER / 2 / CT;
    const uint32_t mask = (1u << sb) - 1;
    uint64_t pm = 1;  // P mod q_t
    if (add_c0)
      for (uint32_t u = 0; u < a.alpha; ++u) pm = mul_mod(pm, reduce64(a.primes[a.L + u].q, pr), pr);
#pragma unroll 1
    for (int v0 = 0; v0 < PPT; ++v0) {
      const uint32_t idx = 2 * (threadIdx.x + v0 * CT * S::T);
      const uint32_t eo = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
      uint64_t ll[CT][2][2], hh[CT][2][2], ss[CT][2][2];  // [ciphertext][part][position]
      uint64_t s0[CT][2];                                  // sum_r kappa_r(c0) (below nrot q)
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        s0[c][0] = s0[c][1] = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int u = 0; u < 2; ++u) ll[c][p][u] = hh[c][p][u] = ss[c][p][u] = 0;
      }
      for (uint32_t r = 0; r < ra.nrot; ++r) {
        uint32_t so[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t p = automorph_src(eo + u, ra.gal[r], LOG_N);
          const uint32_t sl = (((p >> LOG_M) - row0) << LOG_M) | (p & (S::M - 1));
          so[u] = sl + (sl >> 3);
        }
        if (add_c0)
#pragma unroll
          for (int c = 0; c < CT; ++c) {
            s0[c][0] += c0s[(size_t)c * TW + so[0]];
            s0[c][1] += c0s[(size_t)c * TW + so[1]];
          }
        const uint64_t* ev = ra.evk[r];
#pragma unroll 2
        for (uint32_t j = 0; j < a.beta; ++j) {
          const uint64_t* kb = ev + (((size_t)j * 2 + 0) * a.np + prime) * N;
          const uint64_t* ka = ev + (((size_t)j * 2 + 1) * a.np + prime) * N;
          const ulonglong2 wb = __ldg(reinterpret_cast<const ulonglong2*>(kb + eo));
          const ulonglong2 wa = __ldg(reinterpret_cast<const ulonglong2*>(ka + eo));
          const Split3 kb0 = split3(wb.x, sb, mask), kb1 = split3(wb.y, sb, mask);
          const Split3 ka0 = split3(wa.x, sb, mask), ka1 = split3(wa.y, sb, mask);
#pragma unroll
          for (int c = 0; c < CT; ++c) {
            const uint64_t* sm = dig + ((size_t)c * a.beta + j) * TW;
            const Split3 x0 = split3(sm[so[0]], sb, mask), x1 = split3(sm[so[1]], sb, mask);
            mac_split3(ll[c][0][0], hh[c][0][0], ss[c][0][0], x0, kb0);
            mac_split3(ll[c][0][1], hh[c][0][1], ss[c][0][1], x1, kb1);
            mac_split3(ll[c][1][0], hh[c][1][0], ss[c][1][0], x0, ka0);
            mac_split3(ll[c][1][1], hh[c][1][1], ss[c][1][1], x1, ka1);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        if (i0 + c >= ra.count) break;
        uint64_t* o0 = a.acc + ((size_t)(i0 + c) * 2 * a.nt + t) * N;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          uint64_t r2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint64_t lo, hi;
            split3_total(ll[c][p][u], hh[c][p][u], ss[c][p][u], sb, lo, hi);
            if (p == 0 && add_c0) mac128(lo, hi, s0[c][u], pm);
            r2[u] = reduce128_any(hi, lo, pr);
          }
          *reinterpret_cast<ulonglong2*>(o0 + (size_t)p * a.nt * N + eo) = make_ulonglong2(r2[0], r2[1]);
        }
      }
    }
    return;
  }
  if (ra.closed) {
    // each thread sums every rotation's products for its own positions, two
    // neighbouring positions at a time (16-byte key loads and stores), for
    // all CT ciphertexts with each key load
    constexpr int PPT = PER / 2 / CT;          // position pairs per thread
    constexpr int PAIRS = PPT < 2 ? PPT : 2;   // pairs per pass (bounds the registers)
    constexpr int NP = 2 * PAIRS;              // positions per pass
#pragma unroll 1
    for (int v0 = 0; v0 < PPT; v0 += PAIRS) {
      uint32_t eo[PAIRS];  // first of the two positions (even)
      uint64_t a0l[CT][NP], a0h[CT][NP], a1l[CT][NP], a1h[CT][NP];  // 128-bit sums of full products
#pragma unroll
      for (int v = 0; v < PAIRS; ++v) {
        const uint32_t idx = 2 * (threadIdx.x + (v0 + v) * CT * S::T);
        eo[v] = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
      }
#pragma unroll
      for (int c = 0; c < CT; ++c)
#pragma unroll
        for (int u = 0; u < NP; ++u) a0l[c][u] = a0h[c][u] = a1l[c][u] = a1h[c][u] = 0;
      for (uint32_t r = 0; r < ra.nrot; ++r) {
        uint32_t so[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
          const uint32_t p = automorph_src(eo[u >> 1] + (u & 1), ra.gal[r], LOG_N);
          const uint32_t sl = (((p >> LOG_M) - row0) << LOG_M) | (p & (S::M - 1));
          so[u] = sl + (sl >> 3);
        }
        const uint64_t* ev = ra.evk[r];
#pragma unroll 2
        for (uint32_t j = 0; j < a.beta; ++j) {
          const uint64_t* kb = ev + (((size_t)j * 2 + 0) * a.np + prime) * N;
          const uint64_t* ka = ev + (((size_t)j * 2 + 1) * a.np + prime) * N;
#pragma unroll
          for (int v = 0; v < PAIRS; ++v) {
            const ulonglong2 wb = __ldg(reinterpret_cast<const ulonglong2*>(kb + eo[v]));
            const ulonglong2 wa = __ldg(reinterpret_cast<const ulonglong2*>(ka + eo[v]));
#pragma unroll
            for (int c = 0; c < CT; ++c) {
              const uint64_t* sm = dig + ((size_t)c * a.beta + j) * TW;
              const uint64_t x0 = sm[so[2 * v]], x1 = sm[so[2 * v + 1]];
              mac128(a0l[c][2 * v], a0h[c][2 * v], x0, wb.x);
              mac128(a0l[c][2 * v + 1], a0h[c][2 * v + 1], x1, wb.y);
              mac128(a1l[c][2 * v], a1h[c][2 * v], x0, wa.x);
              mac128(a1l[c][2 * v + 1], a1h[c][2 * v + 1], x1, wa.y);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        if (i0 + c >= ra.count) break;
        uint64_t* o0 = a.acc + ((size_t)(i0 + c) * 2 * a.nt + t) * N;
        uint64_t* o1 = o0 + (size_t)a.nt * N;
#pragma unroll
        for (int v = 0; v < PAIRS; ++v) {
          *reinterpret_cast<ulonglong2*>(o0 + eo[v]) =
              make_ulonglong2(reduce128_any(a0h[c][2 * v], a0l[c][2 * v], pr),
                              reduce128_any(a0h[c][2 * v + 1], a0l[c][2 * v + 1], pr));
          *reinterpret_cast<ulonglong2*>(o1 + eo[v]) =
              make_ulonglong2(reduce128_any(a1h[c][2 * v], a1l[c][2 * v], pr),
                              reduce128_any(a1h[c][2 * v + 1], a1l[c][2 * v + 1], pr));
        }
      }
    }
    return;
  }
  if constexpr (CT == 1) {  // rotations that move rows between CTAs (launched with one ciphertext per CTA)
    constexpr int GRP = PER / 2;  // residues per thread and pass (bounds the registers)
    for (uint32_t r = 0; r < ra.nrot; ++r) {
      const uint64_t* ev = ra.evk[r];
      uint64_t* o0 = a.acc + ((size_t)i * 2 * a.nt + t) * N;
      uint64_t* o1 = o0 + (size_t)a.nt * N;
#pragma unroll 1
      for (int u0 = 0; u0 < PER; u0 += GRP) {
        uint32_t so[GRP], eo[GRP];
#pragma unroll
        for (int u = 0; u < GRP; ++u) {
          const uint32_t idx = threadIdx.x + (u0 + u) * S::T;
          const uint32_t k = idx >> LOG_M, x = idx & (S::M - 1);
          const uint32_t row = row0 + k;
          const uint32_t orow = automorph_src(row << LOG_M, ra.gal_inv[r], LOG_N) >> LOG_M;
          const uint32_t e = (orow << LOG_M) | x;
          const uint32_t sl = (k << LOG_M) | (automorph_src(e, ra.gal[r], LOG_N) & (S::M - 1));
          so[u] = sl + (sl >> 3);
          eo[u] = e;
        }
        uint64_t a0l[GRP], a0h[GRP], a1l[GRP], a1h[GRP];  // 128-bit sums of full products
#pragma unroll
        for (int u = 0; u < GRP; ++u) a0l[u] = a0h[u] = a1l[u] = a1h[u] = 0;
        for (uint32_t j = 0; j < a.beta; ++j) {
          const uint64_t* sm = dig + (size_t)j * TW;
          const uint64_t* kb = ev + (((size_t)j * 2 + 0) * a.np + prime) * N;
          const uint64_t* ka = ev + (((size_t)j * 2 + 1) * a.np + prime) * N;
#pragma unroll
          for (int u = 0; u < GRP; ++u) {
            const uint64_t x = sm[so[u]];
            mac128(a0l[u], a0h[u], x, __ldg(kb + eo[u]));
            mac128(a1l[u], a1h[u], x, __ldg(ka + eo[u]));
          }
        }
        // other CTAs add the other rotations' products to these rows: the
        // accumulator (zeroed first) holds sums of nrot residues
#pragma unroll
        for (int u = 0; u < GRP; ++u) {
          atomicAdd(reinterpret_cast<unsigned long long*>(o0 + eo[u]),
                    (unsigned long long)reduce128_any(a0h[u], a0l[u], pr));
          atomicAdd(reinterpret_cast<unsigned long long*>(o1 + eo[u]),
                    (unsigned long long)reduce128_any(a1h[u], a1l[u], pr));
        }
      }
    }
  }
}

// ---- ModDown, fused the same way ------------------------------------------
// The P-part of the accumulators (coefficient form after its inverse NTT,
// whose column pass md_conv_col runs itself when only the row pass was run
// before it) is converted to each target limb inside the load of the forward
// NTT's column pass (as k_moddown_conv: conv = BConv(y + h) - h), and the row pass ends
// with the combine of k_ks_combine: out = add + (acc_Q - NTT(conv)) * P^-1.
// A CTA handles both parts of one ciphertext for one limb and tile, so the
// staged twiddles serve two transforms.
struct MdArgs {
  // The P part (coefficient form): ciphertext i, part p, special prime u at
  // yP + i*yp_stride + p*yp_pstride + u*N.
  const uint64_t* yP;
  uint64_t yp_stride, yp_pstride;
  CtBatch accq;         // the Q part (evaluation form), limbs 0 .. level-1
  uint64_t* conv;       // count x [2][level][N]: column-pass outputs
  CtBatch add, out;
  int has_add;          // 0 none, 1 part 0 only, 2 both parts, 3 permuted on part 0 plus plain on both
  uint32_t n_gal;       // part 0 of the addend is added through each automorphism X -> X^gal[g]
  uint64_t gal[HE_MAX_ROT];
  uint32_t level, alpha, L;
  uint32_t spr[HE_MAX_DIGIT];  // prime indices of the alpha dropped limbs (the special primes; q_l for a
                               // rescale by q_l; q_{l-1} and the special primes for a ModDown merged with it)
  int kind;                    // 0 ModDown, 1 rescale, 2 ModDown merged with the rescale (profile names)
  const uint64_t* addw;        // the addend is multiplied by these Shoup pairs per target limb (nullptr: not)
  const PrimeDev* primes;
  const ulonglong2* tw;
  const ulonglong2* itw;  // inverse twiddles (half)
  int half;               // yP holds only the inverse transform's row pass: md_conv_col finishes it
  const uint64_t* md;   // ModDown tables (params.cu)
};

// Grid: count * 2 * TILES; the conversion's per-special-prime terms and the
// multiple v of P are computed once per element and kept in shared memory
// ([alpha][TILE] words and [TILE] counts) for all level target limbs.
template <int LOG_N, int LOG_M, int LOG_K>
__global__ void __launch_bounds__((1 << (LOG_M + LOG_K)) / 8) md_conv_col(MdArgs a) {
  using S = Shape<LOG_N, LOG_M, LOG_K, true>;
  constexpr uint32_t N = 1u << LOG_N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  uint64_t* wv = sm + S::TILE + S::TILE / 8;                          // [alpha][TILE]
  uint32_t* vv = reinterpret_cast<uint32_t*>(wv + (size_t)a.alpha * S::TILE);  // [TILE]
  uint32_t b = blockIdx.x;
  const uint32_t tile = b % S::TILES;
  b /= S::TILES;
  const uint32_t p = b % 2, i = b / 2;
  const uint64_t* mat = a.md + 2 * a.alpha;
  const uint64_t* hP = mat + (size_t)a.alpha * a.L + 2 * a.L;
  const uint64_t* mat_sh = hP + a.alpha + a.L;
  const uint64_t* wlo = mat_sh + (size_t)a.alpha * a.L;
  const uint64_t* yP = a.yP + (size_t)i * a.yp_stride + (size_t)p * a.yp_pstride;
  // exact conversion: sum_u w_u (P/p_u) - v P, w_u = [y_u (P/p_u)^-1]_{p_u},
  // v = floor(sum_u w_u / p_u) (64.64 fixed point, resolved exactly near an
  // integer)
  for (uint32_t u = 0; u < a.alpha; ++u) {
    const PrimeDev pp = a.primes[a.spr[u]];
    const uint64_t* src = yP + (size_t)u * N;
    if (a.half) {
      // the inverse transform's column pass on this tile, then the scaling by N^-1
      stage_twiddles<LOG_N, LOG_M, LOG_K, true>(stw, a.itw + (size_t)a.spr[u] * N, tile);
#pragma unroll 8
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T)
        sm[idx + (idx >> 3)] = __ldg(src + S::gidx(tile, idx & (S::K - 1), idx >> LOG_K));
      __syncthreads();
      run_rounds<true, false, LOG_N, LOG_M, LOG_K, true>(sm, stw, pp.q);
    }
#pragma unroll 2
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
      const uint64_t y0 = a.half ? mul_shoup(sm[idx + (idx >> 3)], pp.n_inv, pp.n_inv_sh, pp.q)
                                 : __ldg(src + S::gidx(tile, idx & (S::K - 1), idx >> LOG_K));
      const uint64_t y = add_mod(y0, hP[u], pp.q);
      wv[(size_t)u * S::TILE + idx] = mul_shoup(y, a.md[2 * u], a.md[2 * u + 1], pp.q);
    }
    // the next limb's staging overwrites stw and sm: wait for every thread
    if (a.half) __syncthreads();
  }
#pragma unroll 2
  for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
    uint64_t fs = 0;
    uint32_t v = 0;
    if (a.alpha > 1) {
      for (uint32_t u = 0; u < a.alpha; ++u)
        frac_acc(wv[(size_t)u * S::TILE + idx], a.primes[a.spr[u]].one_sh, wlo[u], &fs, &v);
      if (frac_in_window(fs, a.alpha)) {
        const uint64_t* phat = wlo + a.alpha + 9 * (size_t)a.L;  // [alpha][8] words of P/p_u, then [8] of P
        v = exact_lift_multiple(wv + idx, S::TILE, a.alpha, phat, phat + 8 * (size_t)a.alpha, v);
      }
    }
    vv[idx] = v;
  }
  for (uint32_t t = 0; t < a.level; ++t) {
    const PrimeDev pr = a.primes[t];
    const uint64_t q2 = pr.q + pr.q, hQ = hP[a.alpha + t];
    const uint64_t* vP = wlo + a.alpha + a.L + (size_t)t * 8;  // v P mod q_t, v < 8
    stage_twiddles<LOG_N, LOG_M, LOG_K, true>(stw, a.tw + (size_t)t * N, tile);
    // Shoup products by (P/p_u) mod q_t (the dropped-prime count a
    // compile-time constant for the usual counts), then - v P - h
    if (a.alpha >= 2 && a.alpha <= 5) {
      if (a.alpha == 2) conv_sum_tile<S::TILE, S::T, 2>(sm, wv, mat + t, mat_sh + t, a.L, pr.q, vv, vP, hQ);
      else if (a.alpha == 3) conv_sum_tile<S::TILE, S::T, 3>(sm, wv, mat + t, mat_sh + t, a.L, pr.q, vv, vP, hQ);
      else if (a.alpha == 4) conv_sum_tile<S::TILE, S::T, 4>(sm, wv, mat + t, mat_sh + t, a.L, pr.q, vv, vP, hQ);
      else conv_sum_tile<S::TILE, S::T, 5>(sm, wv, mat + t, mat_sh + t, a.L, pr.q, vv, vP, hQ);
    } else {
#pragma unroll 2
      for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
        uint64_t acc = 0;  // kept in [0, 2q)
        for (uint32_t u = 0; u < a.alpha; ++u) {
          acc += mul_shoup_lazy(wv[(size_t)u * S::TILE + idx], mat[(size_t)u * a.L + t], mat_sh[(size_t)u * a.L + t],
                                pr.q);
          acc = acc >= q2 ? acc - q2 : acc;
        }
        acc = acc >= pr.q ? acc - pr.q : acc;
        acc = sub_mod(acc, vP[vv[idx]], pr.q);
        sm[idx + (idx >> 3)] = sub_mod(acc, hQ, pr.q);
      }
    }
    __syncthreads();
    if (pr.q < (1ull << 58)) run_rounds<false, true, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
    else run_rounds<false, false, LOG_N, LOG_M, LOG_K, true>(sm, stw, pr.q);
    uint64_t* out = a.conv + (((size_t)i * 2 + p) * a.level + t) * N;
#pragma unroll 8
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
      const uint32_t xx = idx >> LOG_K, k = idx & (S::K - 1);
      out[S::gidx(tile, k, xx)] = sm[idx + (idx >> 3)];
    }
  }
}

template <int LOG_N, int LOG_M, int LOG_K>
__global__ void __launch_bounds__((1 << (LOG_M + LOG_K)) / 8, 3) md_row_combine(MdArgs a) {
  using S = Shape<LOG_N, LOG_M, LOG_K, false>;
  constexpr uint32_t N = 1u << LOG_N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* stw = reinterpret_cast<ulonglong2*>(smem_raw);
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem_raw + sizeof(ulonglong2) * S::NTW);
  uint32_t b = blockIdx.x;
  const uint32_t tile = b % S::TILES;
  b /= S::TILES;
  const uint32_t t = b % a.level, i = b / a.level;
  const PrimeDev pr = a.primes[t];
  const uint64_t q = pr.q;
  const bool lazy = q < (1ull << 58);
  const uint64_t* pinv = a.md + 2 * a.alpha + (size_t)a.alpha * a.L;
  const uint64_t w = pinv[2 * t], wsh = pinv[2 * t + 1];
  const uint64_t dw = a.addw ? a.addw[2 * t] : 1, dwsh = a.addw ? a.addw[2 * t + 1] : 0;
  stage_twiddles<LOG_N, LOG_M, LOG_K, false>(stw, a.tw + (size_t)t * N, tile);
  constexpr int PER = S::TILE / S::T;
  for (uint32_t p = 0; p < 2; ++p) {
    const uint64_t* src = a.conv + (((size_t)i * 2 + p) * a.level + t) * N;
#pragma unroll 8
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)S::TILE; idx += S::T) {
      const uint32_t k = idx >> LOG_M, x = idx & (S::M - 1);
      sm[idx + (idx >> 3)] = __ldg(src + S::gidx(tile, k, x));
    }
    // the epilogue's operands are loaded before the transform so that their
    // latency overlaps its rounds
    const uint64_t* accq = cpoly(a.accq, i, p, t, N);
    const bool add = a.has_add >= 2 || (a.has_add == 1 && p == 0);
    const bool add_perm = (a.has_add == 1 || a.has_add == 3) && p == 0 && a.n_gal;  // part 0 through the automorphisms
    const bool add_plain = a.has_add == 3 || (add && !add_perm);                     // the addend as it is
    const uint64_t* ad = add ? cpoly(a.add, i, p, t, N) : nullptr;
    uint64_t av[PER], dv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * S::T;
      const uint32_t e = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
      av[u] = __ldg(accq + e);
      dv[u] = add_plain ? __ldg(ad + e) : 0;
    }
    if (add_perm)  // one automorphism at a time: the thread's PER gathers are independent loads
      for (uint32_t g = 0; g < a.n_gal; ++g) {
        uint64_t gv[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const uint32_t idx = threadIdx.x + u * S::T;
          const uint32_t e = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
          gv[u] = __ldg(ad + automorph_src(e, a.gal[g], LOG_N));
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) dv[u] = add_mod(dv[u], gv[u], q);
      }
    __syncthreads();
    if (lazy) run_rounds<false, true, LOG_N, LOG_M, LOG_K, false>(sm, stw, q);
    else run_rounds<false, false, LOG_N, LOG_M, LOG_K, false>(sm, stw, q);
    uint64_t* o = cpoly(a.out, i, p, t, N);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * S::T;
      const uint32_t e = S::gidx(tile, idx >> LOG_M, idx & (S::M - 1));
      const uint64_t v = sm[idx + (idx >> 3)];
      const uint64_t cv = lazy ? fwd_final<true>(v, pr) : fwd_final<false>(v, pr);
      uint64_t r = mul_shoup(sub_mod(av[u], cv, q), w, wsh, q);
      if (add) r = add_mod(r, a.addw ? mul_shoup(dv[u], dw, dwsh, q) : dv[u], q);
      o[e] = r;
    }
  }
}

// Shared memory of md_conv_col with nd dropped limbs.
template <int LOG_N, int M1, int K1>
size_t md_col_smem(uint32_t nd) {
  using SC = Shape<LOG_N, M1, K1, true>;
  return sizeof(ulonglong2) * SC::NTW + sizeof(uint64_t) * (SC::TILE + SC::TILE / 8) +
         (sizeof(uint64_t) * nd + sizeof(uint32_t)) * SC::TILE;
}

template <int LOG_N, int M1, int K1, int M2, int K2>
int md_fused_run(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  using SC = Shape<LOG_N, M1, K1, true>;
  using SR = Shape<LOG_N, M2, K2, false>;
  const size_t smc = md_col_smem<LOG_N, M1, K1>(a.alpha);
  const size_t smr = sizeof(ulonglong2) * SR::NTW + sizeof(uint64_t) * (SR::TILE + SR::TILE / 8);
  if (smc > kModupAllSmem) {  // too many special primes for this tile: the caller runs the unfused sequence
    *handled = false;
    if (a.half) return fail(HE_EINVAL, "md_fused: half-transformed input needs the fused kernels");
    return HE_OK;
  }
  *handled = true;
  static std::atomic<unsigned long long> attr_col{0}, attr_row{0};
  HE_TRY(set_smem_attr_once(attr_col, c->device, (const void*)md_conv_col<LOG_N, M1, K1>, kModupAllSmem));
  HE_TRY(set_smem_attr_once(attr_row, c->device, (const void*)md_row_combine<LOG_N, M2, K2>, smr));
  const double n = (double)(1u << LOG_N);
  const double polys = 2.0 * count * a.level;  // transformed limbs
  const char* nm_col = a.kind == 1 ? "rescale_ntt" : a.kind == 2 ? "moddown_rescale_ntt" : "moddown_ntt";
  const char* nm_row = a.kind == 1 ? "rescale_ntt_final" : a.kind == 2 ? "moddown_rescale_ntt_combine"
                                                                       : "moddown_ntt_combine";
  {
    const size_t blocks = (size_t)count * 2 * SC::TILES;
    // with a half-transformed input, also the dropped limbs' inverse column pass
    const double bfly = polys * n / 2 * M1 + (a.half ? 2.0 * count * a.alpha * n / 2 * M1 : 0.0);
    ProfScope prof(c, nm_col, bfly + polys * n * a.alpha, n * 8 * (2.0 * count * a.alpha + polys), 0.0, bfly);
    md_conv_col<LOG_N, M1, K1><<<(unsigned)blocks, SC::T, smc, c->stream>>>(a);
  }
  HE_CUDA(cudaGetLastError());
  {
    const size_t blocks = (size_t)count * a.level * SR::TILES;
    const double addw = a.has_add == 3 ? 1.5 * polys : a.has_add == 2 ? polys : a.has_add == 1 ? polys / 2 : 0.0;
    ProfScope prof(c, nm_row, polys * (n / 2 * M2 + 2 * n), n * 8 * (3.0 * polys + addw), 0.0, polys * n / 2 * M2);
    md_row_combine<LOG_N, M2, K2><<<(unsigned)blocks, SR::T, smr, c->stream>>>(a);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// Dynamic shared memory of ks_modup_col_all for these digits.
template <int LOG_N, int M1, int K1>
size_t ks_all_smem(const he_ctx* c, uint32_t beta, const uint32_t* cnt) {
  using SC = Shape<LOG_N, M1, K1, true>;
  uint32_t cnt_max = 0;
  for (uint32_t j = 0; j < beta; ++j) cnt_max = std::max(cnt_max, cnt[j]);
  (void)c;
  return sizeof(ulonglong2) * SC::NTW + sizeof(uint64_t) * (SC::TILE + SC::TILE / 8) +
         sizeof(uint64_t) * (size_t)cnt_max * SC::TILE;
}

// The ModUp + column-pass launch shared by the key switch and the hoisted
// rotate-and-sum.
template <int LOG_N, int M1, int K1>
int ks_modup_launch(he_ctx* c, const KsFusedArgs& a, uint32_t count) {
  using SC = Shape<LOG_N, M1, K1, true>;
  const size_t smc = sizeof(ulonglong2) * SC::NTW + sizeof(uint64_t) * (SC::TILE + SC::TILE / 8);
  static std::atomic<unsigned long long> attr_one{0}, attr_all{0};
  HE_TRY(set_smem_attr_once(attr_one, c->device, (const void*)ks_modup_col<LOG_N, M1, K1>, smc));
  HE_TRY(set_smem_attr_once(attr_all, c->device, (const void*)ks_modup_col_all<LOG_N, M1, K1>, kModupAllSmem));
  const double n = (double)(1u << LOG_N);
  double own = 0;  // limbs each ciphertext takes as they are
  for (uint32_t j = 0; j < a.beta; ++j) own += a.cnt[j];
  const double conv = (double)a.beta * a.nt - own;  // converted limbs per ciphertext
  double conv_products = 0;  // basis-conversion products (none when a digit is one limb)
  for (uint32_t j = 0; j < a.beta; ++j)
    if (a.cnt[j] > 1) conv_products += (double)(a.nt - a.cnt[j]) * a.cnt[j];
  // work = modular products: butterflies, conversion products
  {
    // with a half-transformed input the kernel also runs the inverse column pass of the level input limbs
    const double inv_bfly = a.half ? (double)a.level * n / 2 * M1 + (double)a.level * n : 0.0;
    const double bfly = count * (conv * n / 2 * M1 + (a.half ? (double)a.level * n / 2 * M1 : 0.0));
    ProfScope prof(c, "ks_modup_ntt", count * (conv * n / 2 * M1 + conv_products * n + inv_bfly),
                   count * n * 8 * (a.level + conv), 0.0, bfly);
    const size_t sma = ks_all_smem<LOG_N, M1, K1>(c, a.beta, a.cnt);
    if (a.half && sma > kModupAllSmem) return fail(HE_EINVAL, "ks_fused: half-transformed input needs the all-targets kernel");
    if (sma <= kModupAllSmem) {  // one CTA per digit and tile, all targets
      const size_t blocks = (size_t)count * a.beta * SC::TILES;
      ks_modup_col_all<LOG_N, M1, K1><<<(unsigned)blocks, SC::T, sma, c->stream>>>(a);
    } else {
      const size_t blocks = (size_t)count * a.beta * a.nt * SC::TILES;
      ks_modup_col<LOG_N, M1, K1><<<(unsigned)blocks, SC::T, smc, c->stream>>>(a);
    }
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// Dynamic shared memory of ks_row_rot (row tiles of half the row pass's
// tile: M2 x 2^(K2-1)) for beta digits of ct ciphertexts (and their part 0's
// tiles when c0).
template <int LOG_N, int M2, int K2>
size_t ks_rot_smem(uint32_t beta, uint32_t ct = 1, bool c0 = false) {
  using SR = Shape<LOG_N, M2, K2 - 1, false>;
  return sizeof(ulonglong2) * SR::NTW + sizeof(uint64_t) * (SR::TILE + SR::TILE / 8) * (beta + (c0 ? 1 : 0)) * ct;
}



// The hoisted rotate-and-sum's ModUp, column pass and row pass with the
// inner products of every rotation.  *handled = false (nothing launched)
// when the digits' tiles do not fit in shared memory.
inline uint32_t brev_host(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// Whether X -> X^gal maps every row tile of the hoisted row pass (2^LOG_K
// rows of 2^LOG_M evaluation points) onto itself.
template <int LOG_N, int LOG_M, int LOG_K>
bool rot_closed(uint64_t gal_inv) {
  for (uint32_t row = 0; row < (1u << (LOG_N - LOG_M)); ++row) {
    const uint32_t e = 2 * brev_host(row << LOG_M, LOG_N) + 1;
    const uint32_t e2 = (uint32_t)(((uint64_t)e * gal_inv) & ((2ull << LOG_N) - 1));
    const uint32_t orow = brev_host((e2 - 1) >> 1, LOG_N) >> LOG_M;
    if ((orow >> LOG_K) != (row >> LOG_K)) return false;
  }
  return true;
}

template <int LOG_N, int M1, int K1, int M2, int K2>
int ks_rot_run(he_ctx* c, const KsRotArgs& ra, uint32_t count, bool* handled, int* closed_out) {
  using SR = Shape<LOG_N, M2, K2 - 1, false>;
  const KsFusedArgs& a = ra.k;
  const size_t smr = ks_rot_smem<LOG_N, M2, K2>(a.beta);
  *handled = smr <= kRotSmemMax;
  if (!*handled) return HE_OK;
  static std::atomic<unsigned long long> attr1{0}, attr2{0}, attr4{0};
  HE_TRY(set_smem_attr_once(attr1, c->device, (const void*)ks_row_rot<LOG_N, M2, K2 - 1, 1>, kRotSmemMax));
  HE_TRY(set_smem_attr_once(attr2, c->device, (const void*)ks_row_rot<LOG_N, M2, K2 - 1, 2>, kRotSmemMax));
  HE_TRY(set_smem_attr_once(attr4, c->device, (const void*)ks_row_rot<LOG_N, M2, K2 - 1, 4>, kRotSmemMax));
  HE_TRY((ks_modup_launch<LOG_N, M1, K1>(c, a, count)));
  const double n = (double)(1u << LOG_N);
  double own = 0;
  for (uint32_t j = 0; j < a.beta; ++j) own += a.cnt[j];
  const double conv = (double)a.beta * a.nt - own;
  {
    KsRotArgs rc = ra;
    rc.count = count;
    rc.closed = ra.closed;  // 0 when the summed products could exceed 128 bits
    for (uint32_t r = 0; r < ra.nrot; ++r) rc.closed &= rot_closed<LOG_N, M2, K2 - 1>(ra.gal_inv[r]) ? 1 : 0;
    // work: the converted limbs' row-pass butterflies, one reduction per
    // accumulator residue, and the key products (split sums on the target
    // limbs whose primes allow them in a closed stage, as the kernel decides;
    // 128-bit multiply-accumulates on the others); bytes: the limbs read once,
    // one accumulator written (the rotations' products are summed into it),
    // each rotation's key read once per launch
    const uint32_t terms_bits = 32 - __builtin_clz(ra.nrot * a.beta);
    double split_limbs = 0, split_q = 0;
    for (uint32_t t = 0; t < a.nt && rc.closed; ++t) {
      const uint32_t k = 64 - __builtin_clzll(c->q[ks_prime(t, a.level, a.L)]), sb = (k + 1) / 2;
      if (2 * sb + 2 + terms_bits <= 64) {
        split_limbs += 1;
        split_q += t < a.level ? 1 : 0;
      }
    }
    // part 0 through the rotations: in closed stages whose limbs q_t all take
    // the split sums, when its tile fits beside the digits'
    if (!rc.closed || split_q < a.level || ks_rot_smem<LOG_N, M2, K2>(a.beta, 1, true) > kRotSmemMax)
      rc.c0 = nullptr;
    const bool c0 = rc.c0 != nullptr;
    *closed_out = rc.closed | (c0 ? 2 : 0);
    const double per_limb = count * 2.0 * ra.nrot * a.beta * n;
    const double macs = per_limb * (a.nt - split_limbs), mac3 = per_limb * split_limbs;
    // (with part 0: nrot additions and one 128-bit product per residue of its limbs, and those limbs read)
    const double c0_work = c0 ? count * (double)a.level * n : 0.0;
    ProfScope prof(c, "ks_ntt_rot_products", count * (conv * n / 2 * M2 + 2.0 * a.nt * n) + macs + mac3 + c0_work,
                   count * n * 8 * (conv + own + 2.0 * a.nt + (c0 ? a.level : 0)) +
                       8.0 * n * ra.nrot * a.beta * 2.0 * a.nt,
                   macs + c0_work, count * conv * n / 2 * M2, mac3);
    if (!rc.closed)
      HE_CUDA(cudaMemsetAsync(ra.k.acc, 0, sizeof(uint64_t) * count * 2 * a.nt * (1u << LOG_N), c->stream));
    // ciphertexts per CTA (closed stages only): the knob, else 2 when that
    // keeps as many warps resident per SM as 1 does (a 15-rotation stage of
    // 512 ciphertexts at N = 2^14, 16 warps either way: 9.3 ms against 10.1 ms
    // for 1 and 10.0 ms for 4; six digits at N = 2^16 would fall from 12 to 8
    // warps, slower)
    uint32_t ct = 1;
    if (rc.closed) {
      auto warps = [&](uint32_t k) {  // resident warps per SM with k ciphertexts per CTA
        const size_t sm = ks_rot_smem<LOG_N, M2, K2>(a.beta, k, c0) + 1024;  // + the runtime's reserve per CTA
        const size_t by_smem = c->smem_per_sm / sm, by_regs = 4 / k;
        return std::min(by_smem, by_regs) * k * (size_t)SR::T / 32;
      };
      const uint32_t want = c->ks_ct ? (uint32_t)c->ks_ct : 2u;
      for (uint32_t cand : {4u, 2u})
        if (ct == 1 && cand <= want && cand <= count && ks_rot_smem<LOG_N, M2, K2>(a.beta, cand, c0) <= kRotSmemMax &&
            (c->ks_ct || warps(cand) >= warps(1)))
          ct = cand;
    }
    const size_t blocks = (size_t)a.nt * ((count + ct - 1) / ct) * SR::TILES;
    const size_t sm = ks_rot_smem<LOG_N, M2, K2>(a.beta, ct, c0);
    if (ct == 4) ks_row_rot<LOG_N, M2, K2 - 1, 4><<<(unsigned)blocks, 4 * SR::T, sm, c->stream>>>(rc);
    else if (ct == 2) ks_row_rot<LOG_N, M2, K2 - 1, 2><<<(unsigned)blocks, 2 * SR::T, sm, c->stream>>>(rc);
    else ks_row_rot<LOG_N, M2, K2 - 1, 1><<<(unsigned)blocks, SR::T, sm, c->stream>>>(rc);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// Per ring size (ks_fused_n12.cu .. ks_fused_n16.cu: one translation unit
// each, so that the template instances compile in parallel): the launches
// for the tile shape c->ntt_shape.
#define HE_KS_FUSED_DECL(NN)                                                         \
  int ks_rot_n##NN(he_ctx* c, const KsRotArgs& a, uint32_t count, bool* handled, int* closed); \
  size_t ks_rot_smem_n##NN(const he_ctx* c, uint32_t beta);                          \
  int md_fused_n##NN(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled);     \
  size_t md_col_smem_n##NN(const he_ctx* c, uint32_t nd);                            \
  size_t ks_all_smem_n##NN(const he_ctx* c, uint32_t beta, const uint32_t* cnt);
HE_KS_FUSED_DECL(12)
HE_KS_FUSED_DECL(13)
HE_KS_FUSED_DECL(14)
HE_KS_FUSED_DECL(15)
HE_KS_FUSED_DECL(16)
#undef HE_KS_FUSED_DECL

}  // namespace he
