// arith.cu -- residue-wise kernels of the ciphertext operations (Sec. 3:
// addition, multiplication, rescaling) and of hybrid key switching.
//
// Every kernel walks (ciphertext, limb, coefficient) with the coefficient
// index fastest, so a warp stays on one limb (one prime) and reads 2 x 64-bit
// words per thread through 128-bit accesses.  The flat index splits into
// (row, coefficient) by a shift (N is a power of two) and the row into
// (ciphertext, part, limb) by divisions that run in 32 bits whenever the row
// index fits, as it does for any batch of fewer than 2^31 limbs (rmod).
#include "he_internal.h"
#include "he_kernels.h"

namespace he {

// r mod d, and r <- r / d.
__device__ __forceinline__ uint32_t rmod(size_t& r, uint32_t d) {
  if (r <= 0xffffffffull) {
    const uint32_t r32 = (uint32_t)r, m = r32 % d;
    r = r32 / d;
    return m;
  }
  const uint32_t m = (uint32_t)(r % d);
  r /= d;
  return m;
}

// ---- tensor product: (a0 b0, a0 b1 + a1 b0, a1 b1) ---------------------------
__global__ void k_tensor(CtBatch A, CtBatch B, CtBatch D, uint64_t* d2, uint64_t d2_stride,
                         uint32_t level, uint32_t count, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    const size_t r = g >> (log_n - 1);
    size_t rq = r;
    const uint32_t t = rmod(rq, level), i = (uint32_t)rq;
    const PrimeDev pr = primes[t];
    const ulonglong2 a0 = *(const ulonglong2*)(cpoly(A, i, 0, t, n) + k);
    const ulonglong2 a1 = *(const ulonglong2*)(cpoly(A, i, 1, t, n) + k);
    const ulonglong2 b0 = *(const ulonglong2*)(cpoly(B, i, 0, t, n) + k);
    const ulonglong2 b1 = *(const ulonglong2*)(cpoly(B, i, 1, t, n) + k);
    ulonglong2 o0, o1, o2;
    o0.x = mul_mod(a0.x, b0.x, pr);
    o0.y = mul_mod(a0.y, b0.y, pr);
    o1.x = add_mod(mul_mod(a0.x, b1.x, pr), mul_mod(a1.x, b0.x, pr), pr.q);
    o1.y = add_mod(mul_mod(a0.y, b1.y, pr), mul_mod(a1.y, b0.y, pr), pr.q);
    o2.x = mul_mod(a1.x, b1.x, pr);
    o2.y = mul_mod(a1.y, b1.y, pr);
    *(ulonglong2*)(cpoly(D, i, 0, t, n) + k) = o0;
    *(ulonglong2*)(cpoly(D, i, 1, t, n) + k) = o1;
    *(ulonglong2*)(d2 + (size_t)i * d2_stride + (size_t)t * n + k) = o2;
  }
}

// ---- ModUp: approximate basis conversion of each digit ------------------------
// For digit j (limbs D_j = [lo, lo+cnt)) and coefficient k: u_a = x_a * inv_a
// mod q_a, then for every target limb t outside D_j (limbs < level, then the
// special primes): y_t = sum_a u_a * ((Q_j/q_a) mod p_t) mod p_t.
__global__ void k_modup(const uint64_t* xc, uint64_t xc_stride, uint64_t* ext, uint64_t ext_stride,
                        ModUpArgs m, uint32_t count, int log_n, const PrimeDev* primes,
                        const uint64_t* consts) {
  const uint32_t n = 1u << log_n;
  const uint32_t nt = m.level + m.alpha;
  const size_t total = (size_t)count * m.beta * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (n - 1));
    const size_t r = g >> log_n;
    size_t rq = r;
    const uint32_t j = rmod(rq, m.beta), i = (uint32_t)rq;
    const uint32_t lo = m.lo[j], cnt = m.cnt[j];
    const uint64_t* tab = consts + m.off[j];
    uint64_t u[HE_MAX_DIGIT];
    for (uint32_t a = 0; a < cnt; ++a) {
      const uint64_t qa = primes[lo + a].q;
      const uint64_t x = xc[(size_t)i * xc_stride + (size_t)(lo + a) * n + k];
      u[a] = mul_shoup(x, tab[2 * a], tab[2 * a + 1], qa);
    }
    const uint64_t* mat = tab + 2 * cnt;
    uint64_t* out = ext + (size_t)i * ext_stride + (size_t)j * nt * n;
    for (uint32_t t = 0; t < nt; ++t) {
      if (t >= lo && t < lo + cnt) continue;
      const uint32_t p = t < m.level ? t : m.L + t - m.level;
      const PrimeDev pr = primes[p];
      uint64_t y = 0;
      for (uint32_t a = 0; a < cnt; ++a)
        y = add_mod(y, mul_mod(reduce64(u[a], pr), mat[(size_t)a * m.np + p], pr), pr.q);
      out[(size_t)t * n + k] = y;
    }
  }
}

// ---- key-switching inner product --------------------------------------------
// acc_p[t] = sum_j ext_j[t] * evk[j][p][prime(t)]; on the digit's own limbs
// ext_j[t] is the input d itself (already in evaluation form).
__global__ void k_inner_product(const uint64_t* ext, uint64_t ext_stride, const uint64_t* d,
                                uint64_t d_stride, const uint64_t* evk, uint64_t* acc,
                                uint64_t acc_stride, uint32_t level, uint32_t alpha, uint32_t beta,
                                uint32_t L, uint32_t np, uint32_t count, int log_n,
                                const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const uint32_t nt = level + alpha;
  const size_t total = (size_t)count * nt * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    const size_t r = g >> (log_n - 1);
    size_t rq = r;
    const uint32_t t = rmod(rq, nt), i = (uint32_t)rq;
    const uint32_t p = t < level ? t : L + t - level;
    const PrimeDev pr = primes[p];
    uint64_t s0x = 0, s0y = 0, s1x = 0, s1y = 0;
    for (uint32_t j = 0; j < beta; ++j) {
      const uint32_t lo = j * alpha;
      const bool own = t >= lo && t < lo + alpha && t < level;
      const uint64_t* src = own ? d + (size_t)i * d_stride + (size_t)t * n
                                : ext + (size_t)i * ext_stride + ((size_t)j * nt + t) * n;
      const ulonglong2 x = *(const ulonglong2*)(src + k);
      const ulonglong2 kb = __ldg((const ulonglong2*)(evk + (((size_t)j * 2 + 0) * np + p) * n + k));
      const ulonglong2 ka = __ldg((const ulonglong2*)(evk + (((size_t)j * 2 + 1) * np + p) * n + k));
      s0x = add_mod(s0x, mul_mod(x.x, kb.x, pr), pr.q);
      s0y = add_mod(s0y, mul_mod(x.y, kb.y, pr), pr.q);
      s1x = add_mod(s1x, mul_mod(x.x, ka.x, pr), pr.q);
      s1y = add_mod(s1y, mul_mod(x.y, ka.y, pr), pr.q);
    }
    uint64_t* a0 = acc + (size_t)i * acc_stride + (size_t)t * n + k;
    uint64_t* a1 = acc + (size_t)i * acc_stride + ((size_t)nt + t) * n + k;
    *(ulonglong2*)a0 = make_ulonglong2(s0x, s0y);
    *(ulonglong2*)a1 = make_ulonglong2(s1x, s1y);
  }
}

// ---- hoisted rotate-and-sum (unfused form, any N) --------------------------------
// The inner products of several rotations sharing one decomposition, summed:
// ext holds the extended digits of d (evaluation form, d itself on each
// digit's own limbs) and rotation r uses them through its automorphism,
//   acc[i][p][t][e] = sum_r sum_j X_j[automorph_src(e, gal_r)] * evk_r[j][p][prime(t)][e],
// which permutes the evaluation points of every limb alike.
__global__ void k_inner_product_rot(const uint64_t* ext, uint64_t ext_stride, const uint64_t* d,
                                    uint64_t d_stride, RotSet rs, uint64_t* acc, uint64_t acc_stride,
                                    uint32_t level, uint32_t alpha, uint32_t beta, uint32_t L, uint32_t np,
                                    uint32_t count, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const uint32_t nt = level + alpha;
  const size_t total = (size_t)count * nt * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t e = (uint32_t)(g & (n - 1));
    const size_t r2 = g >> log_n;
    size_t r2q = r2;
    const uint32_t t = rmod(r2q, nt), i = (uint32_t)r2q;
    const uint32_t p = t < level ? t : L + t - level;
    const PrimeDev pr = primes[p];
    uint64_t s0 = 0, s1 = 0;
    for (uint32_t r = 0; r < rs.n; ++r) {
      const uint32_t src = automorph_src(e, rs.gal[r], log_n);
      const uint64_t* evk = rs.evk[r];
      for (uint32_t j = 0; j < beta; ++j) {
        const uint32_t lo = j * alpha;
        const bool own = t >= lo && t < lo + alpha && t < level;
        const uint64_t x = own ? d[(size_t)i * d_stride + (size_t)t * n + src]
                               : ext[(size_t)i * ext_stride + ((size_t)j * nt + t) * n + src];
        s0 = add_mod(s0, mul_mod(x, __ldg(evk + (((size_t)j * 2 + 0) * np + p) * n + e), pr), pr.q);
        s1 = add_mod(s1, mul_mod(x, __ldg(evk + (((size_t)j * 2 + 1) * np + p) * n + e), pr), pr.q);
      }
    }
    uint64_t* a = acc + (size_t)i * acc_stride;
    a[(size_t)t * n + e] = s0;
    a[((size_t)nt + t) * n + e] = s1;
  }
}

// Accumulators of both parts (limbs 0 .. nt-1, limb t over prime(t)) reduced
// to [0, q) from sums of a few residues.
__global__ void k_reduce_acc(uint64_t* acc, uint64_t acc_stride, uint32_t nt, uint32_t level, uint32_t L,
                             uint32_t count, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)count * 2 * nt * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t e = (uint32_t)(g & (n - 1));
    size_t r = g >> log_n;
    const uint32_t t = rmod(r, nt);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    uint64_t* a = acc + (size_t)i * acc_stride + ((size_t)p * nt + t) * n + e;
    *a = reduce64(*a, primes[t < level ? t : L + t - level]);
  }
}

// O = (A0 + sum_r kappa_r(A0), A1): the addend of a hoisted rotate-and-sum.
__global__ void k_add_automorphs(CtBatch A, CtBatch O, RotSet rs, uint32_t level, uint32_t count, int log_n,
                                 const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)count * 2 * level * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t e = (uint32_t)(g & (n - 1));
    size_t r = g >> log_n;
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q;
    const uint64_t* a = cpoly(A, i, p, t, n);
    uint64_t v = a[e];
    if (p == 0)
      for (uint32_t s = 0; s < rs.n; ++s) v = add_mod(v, a[automorph_src(e, rs.gal[s], log_n)], q);
    cpoly(O, i, p, t, n)[e] = v;
  }
}

// ---- ModDown conversion: BConv from P to each limb q_t (coefficient form) ----
// y (special limbs of the accumulator, coefficient form) plus h = (P-1)/2 ->
// conv[t] = sum_k [(y_k + h) * (P/p_k)^-1]_{p_k} * ((P/p_k) mod q_t) - h mod q_t:
// subtracting this from the accumulator divides by P with rounding (for one
// special prime it is the centered residue of the accumulator mod P).
__global__ void k_moddown_conv(const uint64_t* acc, uint64_t acc_stride, uint32_t nt, MdDrop dr, uint64_t* conv,
                               uint64_t conv_stride, uint32_t level, uint32_t L, uint32_t count, int log_n,
                               const PrimeDev* primes, const uint64_t* md) {
  const uint32_t n = 1u << log_n;
  const uint32_t alpha = dr.n;
  const size_t total = (size_t)count * 2 * n;
  const uint64_t* mat = md + 2 * alpha;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (n - 1));
    const size_t r = g >> log_n;
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    uint64_t u[HE_MAX_DIGIT];
    const uint64_t* hP = md + 2 * alpha + (size_t)alpha * L + 2 * L;
    const uint64_t* hQ = hP + alpha;
    const uint64_t* wlo = hQ + L + (size_t)alpha * L;
    const uint64_t* p_mod_q = wlo + alpha;
    // exact conversion: v = floor(sum_a u_a / p_a) multiples of P come off
    uint64_t fs = 0;
    uint32_t v = 0;
    for (uint32_t a = 0; a < alpha; ++a) {
      const PrimeDev& pp = primes[dr.pr[a]];
      const uint64_t y = add_mod(acc[(size_t)i * acc_stride + ((size_t)p * nt + dr.first + a) * n + k], hP[a], pp.q);
      u[a] = mul_shoup(y, md[2 * a], md[2 * a + 1], pp.q);
      if (alpha > 1) frac_acc(u[a], pp.one_sh, wlo[a], &fs, &v);
    }
    if (alpha > 1 && frac_in_window(fs, alpha)) {
      const uint64_t* phat = wlo + alpha + 9 * (size_t)L;  // [alpha][8] words of P/p_a, then [8] of P
      v = exact_lift_multiple(u, 1, alpha, phat, phat + 8 * (size_t)alpha, v);
    }
    uint64_t* out = conv + (size_t)i * conv_stride + (size_t)p * level * n;
    for (uint32_t t = 0; t < level; ++t) {
      const PrimeDev pr = primes[t];
      uint64_t s = 0;
      for (uint32_t a = 0; a < alpha; ++a)
        s = add_mod(s, mul_mod(reduce64(u[a], pr), mat[(size_t)a * L + t], pr), pr.q);
      if (v) s = sub_mod(s, reduce64((uint64_t)v * p_mod_q[t], pr), pr.q);
      out[(size_t)t * n + k] = sub_mod(s, hQ[t], pr.q);
    }
  }
}

// ---- ModDown finish: out = add + (acc_Q - conv) * P^-1 ----------------------
// has_add: 0 no addend, 1 addend on part 0 only, 2 on both parts; addw (if
// set): the addend times these Shoup pairs per limb.  acc has nt limbs per part.
__global__ void k_ks_combine(const uint64_t* acc, uint64_t acc_stride, uint32_t nt, const uint64_t* conv,
                             uint64_t conv_stride, CtBatch add, int has_add, const uint64_t* addw, CtBatch out,
                             uint32_t level, uint32_t count, int log_n, const PrimeDev* primes,
                             const uint64_t* pinv) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q;
    const uint64_t w = pinv[2 * t], wsh = pinv[2 * t + 1];
    const ulonglong2 a = *(const ulonglong2*)(acc + (size_t)i * acc_stride + ((size_t)p * nt + t) * n + k);
    const ulonglong2 c = *(const ulonglong2*)(conv + (size_t)i * conv_stride + ((size_t)p * level + t) * n + k);
    ulonglong2 o;
    o.x = mul_shoup(sub_mod(a.x, c.x, q), w, wsh, q);
    o.y = mul_shoup(sub_mod(a.y, c.y, q), w, wsh, q);
    if (has_add == 2 || (has_add == 1 && p == 0)) {
      ulonglong2 d = *(const ulonglong2*)(cpoly(add, i, p, t, n) + k);
      if (addw) {
        d.x = mul_shoup(d.x, addw[2 * t], addw[2 * t + 1], q);
        d.y = mul_shoup(d.y, addw[2 * t], addw[2 * t + 1], q);
      }
      o.x = add_mod(o.x, d.x, q);
      o.y = add_mod(o.y, d.y, q);
    }
    *(ulonglong2*)(cpoly(out, i, p, t, n) + k) = o;
  }
}

// acc limb l (both parts) += P_l * d_l: the merged ModDown's dropped limb
// q_l holds V = acc + P d (P d vanishes on the special primes).
__global__ void k_add_pd(uint64_t* acc, uint64_t acc_stride, uint32_t nt, CtBatch d, uint32_t l, uint64_t Pl,
                         uint64_t Pl_sh, uint32_t count, int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)count * 2 * n;
  const uint64_t q = primes[l].q;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (n - 1));
    const size_t r = g >> log_n;
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    uint64_t* a = acc + (size_t)i * acc_stride + ((size_t)p * nt + l) * n + k;
    *a = add_mod(*a, mul_shoup(cpoly(d, i, p, l, n)[k], Pl, Pl_sh, q), q);
  }
}

// ---- rescale ------------------------------------------------------------------
// last: coefficient form of limb l-1 of both parts [count][2][N].  corr[t] =
// (centered last) mod q_t for t < l-1, coefficient form.
__global__ void k_rescale_corr(const uint64_t* last, uint64_t* corr, uint32_t level, uint32_t count,
                               int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const uint32_t lt = level - 1;
  const uint64_t ql = primes[lt].q, h = (ql - 1) >> 1;
  const size_t total = (size_t)count * 2 * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint64_t x = last[g];
    const size_t ip = g >> log_n;
    const uint32_t k = (uint32_t)(g & (n - 1));
    const bool neg = x > h;
    const uint64_t mag = neg ? ql - x : x;
    uint64_t* out = corr + ip * (size_t)lt * n + k;
    for (uint32_t t = 0; t < lt; ++t) {
      const PrimeDev pr = primes[t];
      const uint64_t m = reduce64(mag, pr);
      out[(size_t)t * n] = (neg && m) ? pr.q - m : m;
    }
  }
}

// out_t = (in_t - corr_t) * q_{l-1}^-1 for t < l-1.
__global__ void k_rescale_final(CtBatch in, const uint64_t* corr, CtBatch out, uint32_t level,
                                uint32_t count, int log_n, const PrimeDev* primes, const uint64_t* rs) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const uint32_t lt = level - 1;
  const size_t total = (size_t)count * 2 * lt * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, lt);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q, w = rs[2 * t], wsh = rs[2 * t + 1];
    const ulonglong2 a = *(const ulonglong2*)(cpoly(in, i, p, t, n) + k);
    const ulonglong2 c = *(const ulonglong2*)(corr + (((size_t)i * 2 + p) * lt + t) * n + k);
    ulonglong2 o;
    o.x = mul_shoup(sub_mod(a.x, c.x, q), w, wsh, q);
    o.y = mul_shoup(sub_mod(a.y, c.y, q), w, wsh, q);
    *(ulonglong2*)(cpoly(out, i, p, t, n) + k) = o;
  }
}

// ---- automorphism in evaluation form: out[j] = in[j'] with
// 2 brv(j') + 1 = (2 brv(j) + 1) * g mod 2N -------------------------------------
__global__ void k_automorph(CtBatch in, CtBatch out, uint32_t nparts, uint32_t level, uint64_t gal,
                            uint32_t count, int log_n) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)count * nparts * level * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(g & (n - 1));
    size_t r = g >> log_n;
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, nparts), i = (uint32_t)rq;
    cpoly(out, i, p, t, n)[j] = cpoly(in, i, p, t, n)[automorph_src(j, gal, log_n)];
  }
}

// ---- circuit glue --------------------------------------------------------------
// op 0: a + b, 1: a - b
__global__ void k_addsub(CtBatch A, CtBatch B, CtBatch O, int op, uint32_t level, uint32_t count,
                         int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q;
    const ulonglong2 a = *(const ulonglong2*)(cpoly(A, i, p, t, n) + k);
    const ulonglong2 b = *(const ulonglong2*)(cpoly(B, i, p, t, n) + k);
    ulonglong2 o;
    if (op == 0) { o.x = add_mod(a.x, b.x, q); o.y = add_mod(a.y, b.y, q); }
    else { o.x = sub_mod(a.x, b.x, q); o.y = sub_mod(a.y, b.y, q); }
    *(ulonglong2*)(cpoly(O, i, p, t, n) + k) = o;
  }
}

// Multiply both parts by per-limb constants (Shoup pairs in kc).
__global__ void k_mul_const(CtBatch A, CtBatch O, LimbConsts kc, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q;
    const ulonglong2 a = *(const ulonglong2*)(cpoly(A, i, p, t, n) + k);
    ulonglong2 o;
    o.x = mul_shoup(a.x, kc.w[t], kc.wsh[t], q);
    o.y = mul_shoup(a.y, kc.w[t], kc.wsh[t], q);
    *(ulonglong2*)(cpoly(O, i, p, t, n) + k) = o;
  }
}

// Add per-limb constants to every evaluation of part 0; copy part 1.
__global__ void k_add_const(CtBatch A, CtBatch O, LimbConsts kc, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const uint64_t q = primes[t].q;
    ulonglong2 a = *(const ulonglong2*)(cpoly(A, i, p, t, n) + k);
    if (p == 0) { a.x = add_mod(a.x, kc.w[t], q); a.y = add_mod(a.y, kc.w[t], q); }
    *(ulonglong2*)(cpoly(O, i, p, t, n) + k) = a;
  }
}

// Multiply both parts by a plaintext in evaluation form pt[level][N].
__global__ void k_mul_plain(CtBatch A, const uint64_t* pt, CtBatch O, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    const PrimeDev pr = primes[t];
    const ulonglong2 a = *(const ulonglong2*)(cpoly(A, i, p, t, n) + k);
    const ulonglong2 b = *(const ulonglong2*)(pt + (size_t)t * n + k);
    ulonglong2 o;
    o.x = mul_mod(a.x, b.x, pr);
    o.y = mul_mod(a.y, b.y, pr);
    *(ulonglong2*)(cpoly(O, i, p, t, n) + k) = o;
  }
}

// Copy limbs [0, level) of both parts (level drop / re-layout).
__global__ void k_copy_limbs(CtBatch A, CtBatch O, uint32_t level, uint32_t count, int log_n) {
  const uint32_t n = 1u << log_n, half = n >> 1;
  const size_t total = (size_t)count * 2 * level * half;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g & (half - 1)) * 2;
    size_t r = g >> (log_n - 1);
    const uint32_t t = rmod(r, level);
    size_t rq = r;
    const uint32_t p = rmod(rq, 2), i = (uint32_t)rq;
    *(ulonglong2*)(cpoly(O, i, p, t, n) + k) = *(const ulonglong2*)(cpoly(A, i, p, t, n) + k);
  }
}

}  // namespace he
