// he_common.cuh -- device arithmetic shared by the sm_103a kernels of the
// RNS-CKKS worker library (residue arithmetic of Li & Huang, KDD'20, Sec. 3).
//
// All residues are uint64 words in [0, q) with q < 2^61 (so that the lazy
// NTT range [0, 4q) fits a word).  Two reductions are used:
//  * Shoup's precomputed-quotient product for a known operand w (twiddles,
//    key-switch and rescale constants): w' = floor(w 2^64 / q),
//    a*w - umulhi(a, w')*q lies in [0, 2q) for every 64-bit a.
//  * Barrett (1986) for a product of two variable residues: k = bitlen(q),
//    mu = floor(2^(2k) / q); for x < 2^(2k), t = x >> (k-1),
//    qe = (t*mu) >> (k+1) undershoots floor(x/q) by at most 2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HE_MAX_PRIMES 64

struct PrimeDev {
  uint64_t q;
  uint64_t mu;        // Barrett constant floor(2^(2k)/q)
  uint32_t k;         // bit length of q
  uint32_t pad;
  uint64_t n_inv;     // N^-1 mod q
  uint64_t n_inv_sh;  // its Shoup companion
  uint64_t one_sh;    // Shoup companion of 1: floor(2^64 / q)
  uint64_t r64;       // 2^64 mod q
  uint64_t r64_sh;    // its Shoup companion
};

__device__ __forceinline__ uint64_t shoup_companion_dev(uint64_t w, uint64_t q) {
  return (uint64_t)(((unsigned __int128)w << 64) / q);
}

// a*w mod q in [0, 2q), any 64-bit a.
__device__ __forceinline__ uint64_t mul_shoup_lazy(uint64_t a, uint64_t w, uint64_t wsh, uint64_t q) {
  uint64_t qh = __umul64hi(a, wsh);
  return a * w - qh * q;
}

__device__ __forceinline__ uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t wsh, uint64_t q) {
  uint64_t r = mul_shoup_lazy(a, w, wsh, q);
  return r >= q ? r - q : r;
}

// (hi:lo) mod q for hi:lo < 2^(2k).
__device__ __forceinline__ uint64_t barrett_reduce128(uint64_t hi, uint64_t lo, const PrimeDev& p) {
  const uint32_t k = p.k;
  uint64_t t = (lo >> (k - 1)) | (hi << (65 - k));
  uint64_t plo = t * p.mu, phi = __umul64hi(t, p.mu);
  uint64_t qe = (plo >> (k + 1)) | (phi << (63 - k));
  uint64_t r = lo - qe * p.q;
  if (r >= p.q) r -= p.q;
  if (r >= p.q) r -= p.q;
  return r;
}

// a*b mod q for a, b < q.
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const PrimeDev& p) {
  return barrett_reduce128(__umul64hi(a, b), a * b, p);
}

// x mod q for any 64-bit x (x < 2^(2k) when k >= 32; hardware remainder otherwise).
__device__ __forceinline__ uint64_t reduce64(uint64_t x, const PrimeDev& p) {
  if (p.k >= 32) return barrett_reduce128(0, x, p);
  return x % p.q;
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
  uint64_t r = a + b;
  return r >= q ? r - q : r;
}

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
  return a >= b ? a - b : a + q - b;
}

// One term of v = floor(sum_k u_k / p_k) for u_k < p_k: u_k 2^64 / p_k in
// 64.64 fixed point from floor(2^128 / p_k) = (one_sh, wlo), at most 2 units
// of 2^-64 below the exact value; the fractional parts accumulate in *s and
// their carries (the integer part) in *v.
__device__ __forceinline__ void frac_acc(uint64_t u, uint64_t one_sh, uint64_t wlo, uint64_t* s, uint32_t* v) {
  const uint64_t t0 = u * one_sh;
  const uint64_t t = t0 + __umul64hi(u, wlo);
  *v += t < t0;
  *s += t;
  *v += *s < t;
}

// The fixed-point sum of frac_acc over a terms is at most 2a units of 2^-64
// below sum_k u_k / p_k = v + x/P (x in [0, P) the exact lift), so its integer
// part is v - 1 only when its fractional part fs lies within 2a units of the
// next integer.  Such an element (about 2a 2^-64 of uniform inputs) takes the
// exact test below.
__device__ __forceinline__ bool frac_in_window(uint64_t fs, uint32_t a) { return fs >= 0ull - 2ull * a; }

// Exact v for an element in that window: v = vc + 1 iff
// sum_k u_k (P/p_k) >= (vc + 1) P, compared as 8-word integers.  u_k at
// u[k * ustride]; phat = [a][8] words of P/p_k, pw = [8] words of P.
static __device__ __noinline__ uint32_t exact_lift_multiple(const uint64_t* u, size_t ustride, uint32_t a,
                                                            const uint64_t* phat, const uint64_t* pw, uint32_t vc) {
  uint64_t s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (uint32_t k = 0; k < a; ++k) {
    const uint64_t x = u[(size_t)k * ustride];
    uint64_t carry = 0;
    for (int w = 0; w < 8; ++w) {
      const uint64_t ph = phat[(size_t)k * 8 + w];
      uint64_t lo = x * ph, hi = __umul64hi(x, ph);
      lo += carry;
      hi += lo < carry;
      s[w] += lo;
      hi += s[w] < lo;
      carry = hi;
    }
  }
  const uint64_t m = (uint64_t)vc + 1;
  uint64_t t[8], carry = 0;
  for (int w = 0; w < 8; ++w) {
    uint64_t lo = m * pw[w], hi = __umul64hi(m, pw[w]);
    lo += carry;
    hi += lo < carry;
    t[w] = lo;
    carry = hi;
  }
  for (int w = 7; w >= 0; --w)
    if (s[w] != t[w]) return s[w] > t[w] ? vc + 1 : vc;
  return vc + 1;
}

// Signed integer to residue.
__device__ __forceinline__ uint64_t from_signed(int64_t x, const PrimeDev& p) {
  if (x >= 0) return reduce64((uint64_t)x, p);
  uint64_t r = reduce64((uint64_t)(-x), p);
  return r ? p.q - r : 0;
}

// (hi:lo) += a*b, the full 128-bit product (no reduction).
// Asynchronous global -> shared copies (cp.async, sm_80 and later): each
// thread's copies are grouped by commit; wait_group n returns when at most n
// of the thread's groups are still in flight (a barrier then makes every
// thread's copies visible).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// at most n groups in flight (n >= 7: at most 7, which waits for more than asked)
__device__ __forceinline__ void cp_async_wait_dyn(uint32_t n) {
  switch (n) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}

__device__ __forceinline__ void mac128(uint64_t& lo, uint64_t& hi, uint64_t a, uint64_t b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(lo), "+l"(hi) : "l"(a), "l"(b));
}

// (hi:lo) mod q for any 128-bit value: hi * (2^64 mod q) by a Shoup product
// (any 64-bit hi, result in [0, 2q)) plus lo mod q, corrected once.
__device__ __forceinline__ uint64_t reduce128_any(uint64_t hi, uint64_t lo, const PrimeDev& p) {
  const uint64_t q = p.q;
  uint64_t r = mul_shoup_lazy(hi, p.r64, p.r64_sh, q) + reduce64(lo, p);
  r = r >= q + q ? r - q - q : r;
  return r >= q ? r - q : r;
}

// Sums of products of residues below 2^k, k <= 2 sb, whose sums fit in 64
// bits (2 sb + 2 + bitlen(terms) <= 64; the fused key switch's key products):
// every residue is split as x = xh 2^sb + xl, and x w is summed as three
// 64-bit sums of 32 x 32 -> 64-bit products (Karatsuba):
//   S_ll = sum xl wl,  S_hh = sum xh wh,  S_s = sum (xl + xh)(wl + wh),
//   sum x w = S_ll + (S_s - S_ll - S_hh) 2^sb + S_hh 2^(2 sb),
// formed as one 128-bit value and reduced once per residue.  The same exact
// sum as the 128-bit multiply-accumulates, so the same residues.
struct Split3 {
  uint32_t l, h, s;
};
__device__ __forceinline__ Split3 split3(uint64_t x, uint32_t sb, uint32_t mask) {
  const uint32_t l = (uint32_t)x & mask, h = (uint32_t)(x >> sb);
  return Split3{l, h, l + h};
}
__device__ __forceinline__ void mac_split3(uint64_t& ll, uint64_t& hh, uint64_t& ss, const Split3& x,
                                           const Split3& w) {
  ll += (uint64_t)x.l * w.l;
  hh += (uint64_t)x.h * w.h;
  ss += (uint64_t)x.s * w.s;
}
// The sum as a 128-bit value (hi:lo).
__device__ __forceinline__ void split3_total(uint64_t ll, uint64_t hh, uint64_t ss, uint32_t sb, uint64_t& lo,
                                             uint64_t& hi) {
  const uint64_t mid = ss - ll - hh;  // sum (xl wh + xh wl), exact
  lo = ll;
  hi = 0;
  const uint64_t m_lo = mid << sb, m_hi = mid >> (64 - sb);  // 1 <= sb <= 31
  const uint64_t h_lo = hh << (2 * sb), h_hi = hh >> (64 - 2 * sb);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(m_lo), "l"(m_hi));
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(h_lo), "l"(h_hi));
}

// 128-bit word (w3:w2:w1:w0) mod q, by Horner on 64-bit halves:
// x = hi*2^64 + lo; hi*2^64 mod q = (hi mod q) * (2^64 mod q).
__device__ __forceinline__ uint64_t reduce_u128(uint64_t hi, uint64_t lo, const PrimeDev& p, uint64_t two64) {
  uint64_t h = reduce64(hi, p);
  uint64_t a = mul_mod(h, two64, p);
  uint64_t b = reduce64(lo, p);
  return add_mod(a, b, p.q);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (c0..c3), key
// (k0, k1); ten rounds of two multiply-xor boxes with a Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    uint4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// Random stream domains (counter word 3).
enum : uint32_t {
  DOM_S = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_EVK_A = 4, DOM_EVK_E = 5,
  DOM_ENC_V = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8, DOM_ENC_A = 9
};

__device__ __forceinline__ uint32_t brev_bits(uint32_t x, int bits) {
  return __brev(x) >> (32 - bits);
}

// The automorphism X -> X^gal (gal odd) in evaluation form: slot j of the
// result is slot automorph_src(j) of the input, where slot j holds the value at
// psi^(2 brv(j) + 1), so 2 brv(src) + 1 = (2 brv(j) + 1) * gal mod 2N.
__device__ __forceinline__ uint32_t automorph_src(uint32_t j, uint64_t gal, int log_n) {
  const uint32_t e = 2 * brev_bits(j, log_n) + 1;
  const uint32_t e2 = (e * (uint32_t)gal) & ((2u << log_n) - 1);  // 2N divides 2^32
  return brev_bits((e2 - 1) >> 1, log_n);
}
