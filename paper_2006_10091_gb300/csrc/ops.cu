// ops.cu -- batched ciphertext operations: hybrid key switching, the
// multiplication of Sec. 3 (tensor, relinearise, rescale), rotation, and the
// circuit glue, each as a fixed sequence of kernel launches over a batch of
// ciphertexts that share level and layout.
//
// Key switching at level l with digits D_j = [j*alpha, min((j+1)*alpha, l)):
//   1. d to coefficient form (inverse NTT, l limbs);
//   2. ModUp every digit to the l limbs and alpha special primes (approximate
//      basis conversion, coefficient form), then forward NTT of the converted
//      limbs (the digit's own limbs are taken from d as they are);
//   3. inner product with the switching key, two accumulators over l + alpha limbs;
//   4. ModDown: inverse NTT of the special limbs (the fused path runs only
//      its row pass here; the conversion kernel does the column pass),
//      conversion of (y + h) to each q_t minus h (h = (P-1)/2, so that the
//      division by P rounds), forward NTT, out_t = (acc_t - conv_t) * P^-1
//      (+ an optional addend).
#include "he_ops.h"

namespace he {
bool ks_converts_per_digit(const he_ctx* c, uint32_t level);
bool md_half_ok(const he_ctx* c, uint32_t nd);
int ntt2_inverse_rows(he_ctx* c, const PolyBatch& b);
int md_fused(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, int add_mode,
             uint64_t add_gal, CtBatch out, uint32_t level, uint32_t count, bool half, bool* handled);
int rs_fused(he_ctx* c, CtBatch in, const uint64_t* last, uint64_t* conv, CtBatch out, uint32_t level,
             uint32_t count, bool half, bool* handled);
bool ks_rot_fits(const he_ctx* c, uint32_t level, uint32_t nrot);
int ks_rot(he_ctx* c, const uint64_t* d, uint64_t d_stride, const uint64_t* d2c, uint64_t* ext, uint64_t* acc,
           const RotSet& rs, uint32_t level, uint32_t count, bool half, bool* handled, bool* unreduced,
           uint64_t in_gal = 0, const uint64_t* c0 = nullptr, uint64_t c0_stride = 0, bool* c0_added = nullptr);
int md_fused_gals(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, int add_mode,
                  const uint64_t* gals, uint32_t n_gal, CtBatch out, uint32_t level, uint32_t count, bool half,
                  bool* handled);
int md_fused_rescale(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, CtBatch out,
                     uint32_t level, uint32_t count, bool half, bool* handled);
}

namespace he {

unsigned grid_for(size_t work) {
  size_t b = (work + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)(b ? b : 1);
}

static PolyBatch pb(const uint64_t* src, uint64_t* dst, uint64_t src_stride, uint64_t dst_stride,
                    uint32_t npolys, uint32_t nl, uint32_t limb0, uint32_t level) {
  PolyBatch b;
  b.src = src;
  b.dst = dst;
  b.src_stride = src_stride;
  b.dst_stride = dst_stride;
  b.npolys = npolys;
  b.nl = nl;
  b.limb0 = limb0;
  b.level = level;
  b.skip_alpha = 0;
  b.skip_beta = 1;
  return b;
}

size_t ks_words(const he_ctx* c, uint32_t level, uint32_t count) {
  const size_t n = c->n, a = c->alpha, beta = (level + a - 1) / a, nt = level + a;
  return count * n * (level + beta * nt + 2 * nt + 2 * level) + 4 * 32;
}

size_t rescale_words(const he_ctx* c, uint32_t level, uint32_t count) {
  return (size_t)count * c->n * (2 + 2 * (level - 1)) + 2 * 32;
}

size_t mul_words(const he_ctx* c, uint32_t level, uint32_t count, bool rescale) {
  size_t w = (size_t)count * c->n * (3 * level) + ks_words(c, level, count) + 2 * 32;
  if (rescale) w += (size_t)count * c->n * 2 * level + rescale_words(c, level, count) + 32;
  return w;
}

size_t rot_words(const he_ctx* c, uint32_t level, uint32_t count) {
  return (size_t)count * c->n * 2 * level + ks_words(c, level, count) + 32;
}

const uint64_t* galois_key(const he_ctx* c, uint64_t gal) {
  auto it = c->gal.find(gal);
  return it == c->gal.end() ? nullptr : it->second;
}

// ModUp and the NTT of the converted limbs as separate kernels (any N):
// ext = count x [beta][nt][N], evaluation form (a digit's own limbs unset).
static int modup_unfused(he_ctx* c, const uint64_t* d2c, uint64_t* ext, uint32_t level, uint32_t count) {
  const uint32_t n = c->n, alpha = c->alpha, L = c->L, np = c->np;
  const uint32_t nt = level + alpha, beta = (level + alpha - 1) / alpha;
  ModUpArgs m;
  m.level = level;
  m.alpha = alpha;
  m.beta = beta;
  m.L = L;
  m.np = np;
  for (uint32_t j = 0; j < beta; ++j) {
    const ModUpConst& mc = c->modup[level][j];
    m.lo[j] = mc.lo;
    m.cnt[j] = mc.cnt;
    m.off[j] = mc.off;
  }
  {
    ProfScope prof(c, "modup", (double)count * beta * n * (double)(nt * alpha), (double)count * n * 8 * (level + (double)beta * nt));
    k_modup<<<grid_for((size_t)count * beta * n), 256, 0, c->stream>>>(
        d2c, (size_t)level * n, ext, (size_t)beta * nt * n, m, count, c->log_n, c->d_primes, c->d_modup);
  }
  HE_CUDA(cudaGetLastError());
  PolyBatch e = pb(ext, ext, (size_t)nt * n, (size_t)nt * n, count * beta, nt, 0, level);
  e.skip_alpha = alpha;
  e.skip_beta = beta;
  return ntt_forward(c, e);
}

// ModUp, NTT of the converted limbs and the key inner product as separate
// kernels (any N).
static int ks_unfused_middle(he_ctx* c, const uint64_t* d, uint64_t d_stride, const uint64_t* d2c, uint64_t* ext,
                             uint64_t* acc, const uint64_t* evk, uint32_t level, uint32_t count) {
  const uint32_t n = c->n, alpha = c->alpha, L = c->L, np = c->np;
  const uint32_t nt = level + alpha, beta = (level + alpha - 1) / alpha;
  HE_TRY(modup_unfused(c, d2c, ext, level, count));
  // 3. inner product with the key
  {
    ProfScope prof(c, "inner_product", 2.0 * count * beta * nt * n, (double)n * 8 * ((double)count * beta * nt + 2.0 * beta * nt * count + 2.0 * count * nt));
    k_inner_product<<<grid_for((size_t)count * nt * n / 2), 256, 0, c->stream>>>(
        ext, (size_t)beta * nt * n, d, d_stride, evk, acc, (size_t)2 * nt * n, level, alpha, beta, L, np,
        count, c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// The ModDown of a key switch as separate kernels: conversion of the dropped
// limbs (already in coefficient form), NTT, combine (add_mode 0 none, 1 part
// 0, 2 both parts; addw scales the addend).  `merged`: the dropped limbs are
// q_{level-1} and the special primes (the ModDown merged with the rescale;
// out has level - 1 limbs), else the special primes.
static int moddown_unfused(he_ctx* c, const uint64_t* acc, uint64_t* conv, CtBatch add, int add_mode, CtBatch out,
                           uint32_t level, uint32_t count, bool merged = false) {
  const uint32_t n = c->n, alpha = c->alpha, L = c->L, nt = level + alpha;
  const uint32_t lt = merged ? level - 1 : level;  // target limbs
  MdDrop dr;
  dr.n = merged ? alpha + 1 : alpha;
  dr.first = lt;
  for (uint32_t u = 0; u < dr.n; ++u) dr.pr[u] = merged ? (u == 0 ? level - 1 : L + u - 1) : L + u;
  const uint64_t* md = merged ? c->d_mdrs + (size_t)level * c->mdrs_words : c->d_moddown;
  const uint64_t* addw = merged ? c->d_rescale + (size_t)(level - 1) * L * 2 : nullptr;
  {
    ProfScope prof(c, "moddown_conv", 2.0 * count * n * dr.n * (lt + 1), (double)count * 2 * n * 8 * (dr.n + lt));
    k_moddown_conv<<<grid_for((size_t)count * 2 * n), 256, 0, c->stream>>>(
        acc, (size_t)2 * nt * n, nt, dr, conv, (size_t)2 * lt * n, lt, L, count, c->log_n, c->d_primes, md);
  }
  HE_CUDA(cudaGetLastError());
  HE_TRY(ntt_forward(c, pb(conv, conv, (size_t)lt * n, (size_t)lt * n, count * 2, lt, 0, lt)));
  const uint64_t* pinv = md + 2 * dr.n + (size_t)dr.n * L;
  {
    ProfScope prof(c, "ks_combine", 2.0 * count * lt * n, (double)count * 2 * lt * n * 8 * (add_mode ? 4 : 3));
    k_ks_combine<<<grid_for((size_t)count * 2 * lt * n / 2), 256, 0, c->stream>>>(
        acc, (size_t)2 * nt * n, nt, conv, (size_t)2 * lt * n, add, add_mode, addw, out, lt, count, c->log_n,
        c->d_primes, pinv);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int keyswitch_batch(he_ctx* c, const uint64_t* d, uint64_t d_stride, uint32_t level, uint32_t count,
                    const uint64_t* evk, CtBatch add, int add_mode, CtBatch out, Arena& ar, uint64_t gal,
                    bool merged) {
  if (merged && (gal || add_mode != 2 || level < 2 || !c->d_mdrs))
    return fail(HE_EINVAL, "keyswitch_batch: the merged rescale takes (d0, d1) as addend, level >= 2");
  const uint32_t n = c->n, alpha = c->alpha, L = c->L, np = c->np;
  const uint32_t nt = level + alpha, beta = (level + alpha - 1) / alpha;
  uint64_t* d2c = ar.take<uint64_t>((size_t)count * level * n);
  uint64_t* ext = ar.take<uint64_t>((size_t)count * beta * nt * n);
  uint64_t* acc = ar.take<uint64_t>((size_t)count * 2 * nt * n);
  uint64_t* conv = ar.take<uint64_t>((size_t)count * 2 * level * n);
  if (!d2c || !ext || !acc || !conv) return fail(HE_ENOMEM, "key switch scratch too small");
  // 1. coefficient form (when each digit is converted in one CTA, only the
  //    inverse transform's row pass here; the conversion kernel finishes it)
  const bool fits = ks_rot_fits(c, level, 1);
  if (gal && !fits) return fail(HE_EINVAL, "keyswitch_batch: automorphism needs the fused kernels");
  const bool half = fits && ks_converts_per_digit(c, level);
  {
    PolyBatch b = pb(d, d2c, d_stride, (size_t)level * n, count, level, 0, level);
    b.gal = gal;
    HE_TRY(half ? ntt2_inverse_rows(c, b) : ntt_inverse(c, b));
  }
  // 2-3. ModUp + NTT + inner product, fused where N has compiled shapes and
  //      the digits' tiles fit in shared memory (the hoisted row kernel with
  //      one rotation by the identity; d read through X -> X^gal)
  bool fused = false;
  if (fits) {
    RotSet rs;
    rs.n = 1;
    rs.gal[0] = 1;
    rs.evk[0] = evk;
    bool unreduced = false;
    HE_TRY(ks_rot(c, d, d_stride, d2c, ext, acc, rs, level, count, half, &fused, &unreduced, gal));
  }
  if (!fused) {
    if (half || gal) return fail(HE_ECUDA, "keyswitch_batch: fused kernels declined");
    HE_TRY(ks_unfused_middle(c, d, d_stride, d2c, ext, acc, evk, level, count));
  }
  // 4. ModDown
  return moddown_batch(c, acc, conv, level, count, add, add_mode, out, ar, gal, merged);
}

// Step 4 of the key switch on acc (count x [2][level + alpha][N], evaluation
// form; its dropped limbs are overwritten), with conv (count x [2][level][N])
// as scratch.
int moddown_batch(he_ctx* c, uint64_t* acc, uint64_t* conv, uint32_t level, uint32_t count, CtBatch add,
                  int add_mode, CtBatch out, Arena& ar, uint64_t gal, bool merged) {
  const uint32_t n = c->n, alpha = c->alpha, nt = level + alpha;
  if (merged) {  // divide P (d0, d1) + acc by P q_{level-1}: its dropped limbs are acc's last alpha + 1
    const uint32_t lo = level - 1;
    {
      ProfScope prof(c, "elementwise", (double)count * 2 * n, (double)count * 2 * n * 24);
      k_add_pd<<<grid_for((size_t)count * 2 * n), 256, 0, c->stream>>>(
          acc, (size_t)2 * nt * n, nt, add, lo, c->P_mod_q[lo], h_shoup(c->P_mod_q[lo], c->q[lo]), count, c->log_n,
          c->d_primes);
    }
    HE_CUDA(cudaGetLastError());
    // the dropped limbs to coefficient form (only the row pass when the
    // fused conversion kernel finishes the transform)
    const bool mh = md_half_ok(c, alpha + 1);
    const PolyBatch bd = pb(acc + (size_t)lo * n, acc + (size_t)lo * n, (size_t)nt * n, (size_t)nt * n, count * 2,
                            alpha + 1, lo, level);
    HE_TRY(mh ? ntt2_inverse_rows(c, bd) : ntt_inverse(c, bd));
    bool done = false;
    HE_TRY(md_fused_rescale(c, acc, (size_t)2 * nt * n, conv, add, out, level, count, mh, &done));
    if (done) return HE_OK;
    return moddown_unfused(c, acc, conv, add, 2, out, level, count, true);
  }
  const bool mh = md_half_ok(c, alpha);
  {
    const PolyBatch bd = pb(acc + (size_t)level * n, acc + (size_t)level * n, (size_t)nt * n, (size_t)nt * n,
                            count * 2, alpha, level, level);
    HE_TRY(mh ? ntt2_inverse_rows(c, bd) : ntt_inverse(c, bd));
  }
  bool md_done = false;
  HE_TRY(md_fused(c, acc, (size_t)2 * nt * n, conv, add, add_mode, gal, out, level, count, mh, &md_done));
  if (md_done) return HE_OK;
  if (gal && add_mode) {  // the unfused combine reads its addend as it is: permute part 0 first
    uint64_t* pa = ar.take<uint64_t>((size_t)count * level * n);
    if (!pa) return fail(HE_ENOMEM, "key switch scratch too small");
    CtBatch P{pa, (size_t)level * n, level, 0};
    k_automorph<<<grid_for((size_t)count * level * n), 256, 0, c->stream>>>(add, P, 1, level, gal, count, c->log_n);
    HE_CUDA(cudaGetLastError());
    add = P;
  }
  return moddown_unfused(c, acc, conv, add, add_mode, out, level, count);
}

int rescale_batch(he_ctx* c, CtBatch in, uint32_t level, uint32_t count, CtBatch out, Arena& ar) {
  const uint32_t n = c->n, lt = level - 1;
  if (level < 2) return fail(HE_ELEVEL, "rescale needs two limbs");
  uint64_t* last = ar.take<uint64_t>((size_t)count * 2 * n);
  uint64_t* corr = ar.take<uint64_t>((size_t)count * 2 * lt * n);
  if (!last || !corr) return fail(HE_ENOMEM, "rescale scratch too small");
  const bool mh = md_half_ok(c, 1);  // the fused kernel finishes the inverse transform
  for (uint32_t p = 0; p < 2; ++p) {
    const PolyBatch bd = pb(in.base + ((size_t)p * in.cap + lt) * n, last + (size_t)p * n, in.stride, 2ull * n,
                            count, 1, lt, c->L);
    HE_TRY(mh ? ntt2_inverse_rows(c, bd) : ntt_inverse(c, bd));
  }
  bool fused = false;  // correction, NTT and division fused like ModDown's
  HE_TRY(rs_fused(c, in, last, corr, out, level, count, mh, &fused));
  if (fused) return HE_OK;
  {
    ProfScope prof(c, "rescale", (double)count * 2 * n * lt, (double)count * 2 * n * 8 * (1 + lt));
    k_rescale_corr<<<grid_for((size_t)count * 2 * n), 256, 0, c->stream>>>(last, corr, level, count,
                                                                            c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  HE_TRY(ntt_forward(c, pb(corr, corr, (size_t)lt * n, (size_t)lt * n, count * 2, lt, 0, c->L)));
  {
    ProfScope prof(c, "rescale", (double)count * 2 * lt * n, (double)count * 2 * lt * n * 8 * 3);
    k_rescale_final<<<grid_for((size_t)count * 2 * lt * n / 2), 256, 0, c->stream>>>(
        in, corr, out, level, count, c->log_n, c->d_primes, c->d_rescale + (size_t)lt * c->L * 2);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int mul_relin_batch(he_ctx* c, CtBatch A, CtBatch B, uint32_t level, uint32_t count, CtBatch out,
                    bool rescale, Arena& ar) {
  const uint32_t n = c->n;
  uint64_t* d01 = ar.take<uint64_t>((size_t)count * 2 * level * n);
  uint64_t* d2 = ar.take<uint64_t>((size_t)count * level * n);
  if (!d01 || !d2) return fail(HE_ENOMEM, "multiplication scratch too small");
  CtBatch D{d01, (size_t)2 * level * n, level, 0};
  {
    ProfScope prof(c, "tensor", 4.0 * count * level * n, (double)count * level * n * 8 * 7);
    k_tensor<<<grid_for((size_t)count * level * n / 2), 256, 0, c->stream>>>(
        A, B, D, d2, (size_t)level * n, level, count, c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  // with the rescale: the key switch's ModDown and the rescale as one division by P q_{level-1}
  return keyswitch_batch(c, d2, (size_t)level * n, level, count, c->d_rlk, D, 2, out, ar, 0, rescale);
}

int rotate_batch(he_ctx* c, CtBatch A, uint32_t level, uint32_t count, uint64_t gal, CtBatch out,
                 Arena& ar) {
  const uint32_t n = c->n;
  const uint64_t* key = galois_key(c, gal);
  if (!key) return fail(HE_ENOKEY, "no Galois key for this rotation");
  // With the fused kernels the automorphism is applied as the key switch
  // reads its input and addend, unless the output overlaps the input.
  const char* a_lo = (const char*)A.base;
  const char* a_hi = a_lo + sizeof(uint64_t) * ((size_t)(count - 1) * A.stride + (size_t)2 * A.cap * n);
  const char* o_lo = (const char*)out.base;
  const char* o_hi = o_lo + sizeof(uint64_t) * ((size_t)(count - 1) * out.stride + (size_t)2 * out.cap * n);
  if (ks_rot_fits(c, level, 1) && (o_hi <= a_lo || a_hi <= o_lo))
    return keyswitch_batch(c, A.base + (size_t)A.cap * n, A.stride, level, count, key, A, 1, out, ar, gal);
  uint64_t* t = ar.take<uint64_t>((size_t)count * 2 * level * n);
  if (!t) return fail(HE_ENOMEM, "rotation scratch too small");
  CtBatch T{t, (size_t)2 * level * n, level, 0};
  {
    ProfScope prof(c, "automorph", 0.0, (double)count * 2 * level * n * 16);
    k_automorph<<<grid_for((size_t)count * 2 * level * n), 256, 0, c->stream>>>(A, T, 2, level, gal, count,
                                                                                 c->log_n);
  }
  HE_CUDA(cudaGetLastError());
  return keyswitch_batch(c, t + (size_t)level * n, (size_t)2 * level * n, level, count, key, T, 1, out, ar);
}

// out = A + sum_r rotate(A, gal_r) with one decomposition of A's second part
// and one ModDown for all rotations (hoisting): iNTT of A1, ModUp + NTT
// once, the inner product of the permuted digits with each rotation's key,
// the sum of those products, ModDown, plus A0 + sum_r kappa_r(A0) and A1.
// out must not overlap A.
int rotsum_batch(he_ctx* c, CtBatch A, uint32_t level, uint32_t count, const uint64_t* gals, uint32_t nrot,
                 CtBatch out, Arena& ar) {
  if (nrot < 1 || nrot > HE_MAX_ROT) return fail(HE_EINVAL, "rotate-and-sum: 1 to 16 rotations per stage");
  RotSet rs;
  rs.n = nrot;
  for (uint32_t r = 0; r < nrot; ++r) {
    if (gals[r] == 1) return fail(HE_EINVAL, "rotate-and-sum: a rotation by 0 slots");
    rs.gal[r] = gals[r];
    rs.evk[r] = galois_key(c, gals[r]);
    if (!rs.evk[r]) return fail(HE_ENOKEY, "no Galois key for this rotation");
  }
  const uint32_t n = c->n, alpha = c->alpha, L = c->L, np = c->np;
  const uint32_t nt = level + alpha, beta = (level + alpha - 1) / alpha;
  const char* a_lo = (const char*)A.base;
  const char* a_hi = a_lo + sizeof(uint64_t) * ((size_t)(count - 1) * A.stride + (size_t)2 * A.cap * n);
  const char* o_lo = (const char*)out.base;
  const char* o_hi = o_lo + sizeof(uint64_t) * ((size_t)(count - 1) * out.stride + (size_t)2 * out.cap * n);
  if (!(o_hi <= a_lo || a_hi <= o_lo)) return fail(HE_EINVAL, "rotate-and-sum: output overlaps the input");
  const uint64_t acc_stride = (uint64_t)2 * nt * n;
  uint64_t* d2c = ar.take<uint64_t>((size_t)count * level * n);
  uint64_t* ext = ar.take<uint64_t>((size_t)count * beta * nt * n);
  uint64_t* acc = ar.take<uint64_t>((size_t)count * acc_stride);
  uint64_t* conv = ar.take<uint64_t>((size_t)count * 2 * level * n);
  if (!d2c || !ext || !acc || !conv) return fail(HE_ENOMEM, "rotate-and-sum scratch too small");
  const uint64_t* d = A.base + (size_t)A.cap * n;
  const bool fits = ks_rot_fits(c, level, nrot);
  const bool half = fits && ks_converts_per_digit(c, level);
  {
    const PolyBatch b = pb(d, d2c, A.stride, (size_t)level * n, count, level, 0, level);
    HE_TRY(half ? ntt2_inverse_rows(c, b) : ntt_inverse(c, b));
  }
  // the fused kernel also adds P sum_r kappa_r(A0) to the accumulator where it
  // can (c0_added): the ModDown then adds A0 and A1 as they are
  bool fused = false, unreduced = false, c0_added = false;
  if (fits)
    HE_TRY(ks_rot(c, d, A.stride, d2c, ext, acc, rs, level, count, half, &fused, &unreduced, 0, A.base, A.stride,
                  &c0_added));
  if (!fused) {
    if (half) return fail(HE_ECUDA, "rotate-and-sum: fused kernels declined a half-transformed input");
    HE_TRY(modup_unfused(c, d2c, ext, level, count));
    {
      ProfScope prof(c, "inner_product", 2.0 * nrot * count * beta * nt * n,
                     (double)n * 8 * ((double)count * beta * nt * (1 + 2.0 * nrot) + 2.0 * count * nt));
      k_inner_product_rot<<<grid_for((size_t)count * nt * n), 256, 0, c->stream>>>(
          ext, (size_t)beta * nt * n, d, A.stride, rs, acc, acc_stride, level, alpha, beta, L, np, count, c->log_n,
          c->d_primes);
    }
    HE_CUDA(cudaGetLastError());
  }
  if (unreduced) {  // sums of nrot residues from the rows the rotations moved between CTAs
    ProfScope prof(c, "elementwise", 0.0, (double)count * 2 * nt * n * 16);
    k_reduce_acc<<<grid_for((size_t)count * 2 * nt * n), 256, 0, c->stream>>>(acc, acc_stride, nt, level, L, count,
                                                                              c->log_n, c->d_primes);
    HE_CUDA(cudaGetLastError());
  }
  // ModDown of the summed inner products, plus A0 + sum_r kappa_r(A0) and A1
  const bool mh = md_half_ok(c, alpha);
  {
    const PolyBatch bd = pb(acc + (size_t)level * n, acc + (size_t)level * n, (size_t)nt * n, (size_t)nt * n,
                            count * 2, alpha, level, level);
    HE_TRY(mh ? ntt2_inverse_rows(c, bd) : ntt_inverse(c, bd));
  }
  bool md_done = false;
  HE_TRY(md_fused_gals(c, acc, acc_stride, conv, A, c0_added ? 2 : 3, gals, c0_added ? 0 : nrot, out, level, count,
                       mh, &md_done));
  if (md_done) return HE_OK;
  if (c0_added) return moddown_unfused(c, acc, conv, A, 2, out, level, count);
  uint64_t* sa = ar.take<uint64_t>((size_t)count * 2 * level * n);
  if (!sa) return fail(HE_ENOMEM, "rotate-and-sum scratch too small");
  const CtBatch S{sa, (uint64_t)2 * level * n, level, 0};
  k_add_automorphs<<<grid_for((size_t)count * 2 * level * n), 256, 0, c->stream>>>(A, S, rs, level, count, c->log_n,
                                                                                   c->d_primes);
  HE_CUDA(cudaGetLastError());
  return moddown_unfused(c, acc, conv, S, 2, out, level, count);
}

size_t rotsum_words(const he_ctx* c, uint32_t level, uint32_t count) {
  const size_t n = c->n, a = c->alpha, beta = (level + a - 1) / a, nt = level + a;
  return count * n * (level + beta * nt + 2 * nt + 2 * level + 2 * level) + 6 * 32;
}

int addsub_batch(he_ctx* c, CtBatch A, CtBatch B, CtBatch O, int op, uint32_t level, uint32_t count) {
  {
    ProfScope prof(c, "elementwise", 0.0, (double)count * 2 * level * c->n * 24);
    k_addsub<<<grid_for((size_t)count * 2 * level * c->n / 2), 256, 0, c->stream>>>(A, B, O, op, level, count,
                                                                                    c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

static LimbConsts int_consts(const he_ctx* c, int64_t k, uint32_t level) {
  LimbConsts kc;
  for (uint32_t t = 0; t < level; ++t) {
    const uint64_t q = c->q[t];
    const __int128 r = (__int128)k % (__int128)q;
    const uint64_t v = (uint64_t)(r < 0 ? r + q : r);
    kc.w[t] = v;
    kc.wsh[t] = h_shoup(v, q);
  }
  return kc;
}

int mul_int_batch(he_ctx* c, CtBatch A, CtBatch O, int64_t k, uint32_t level, uint32_t count) {
  {
    ProfScope prof(c, "elementwise", 0.0, (double)count * 2 * level * c->n * 16);
    k_mul_const<<<grid_for((size_t)count * 2 * level * c->n / 2), 256, 0, c->stream>>>(
        A, O, int_consts(c, k, level), level, count, c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int add_int_batch(he_ctx* c, CtBatch A, CtBatch O, int64_t k, uint32_t level, uint32_t count) {
  {
    ProfScope prof(c, "elementwise", 0.0, (double)count * 2 * level * c->n * 16);
    k_add_const<<<grid_for((size_t)count * 2 * level * c->n / 2), 256, 0, c->stream>>>(
        A, O, int_consts(c, k, level), level, count, c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int copy_batch(he_ctx* c, CtBatch A, CtBatch O, uint32_t level, uint32_t count) {
  {
    ProfScope prof(c, "elementwise", 0.0, (double)count * 2 * level * c->n * 16);
    k_copy_limbs<<<grid_for((size_t)count * 2 * level * c->n / 2), 256, 0, c->stream>>>(A, O, level, count,
                                                                                        c->log_n);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

__global__ void k_accumulate(CtBatch in, uint32_t count, CtBatch acc, uint32_t level, int log_n,
                             const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)2 * level * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(g % n);
    const size_t r = g / n;
    const uint32_t t = (uint32_t)(r % level), p = (uint32_t)(r / level);
    const uint64_t q = primes[t].q;
    uint64_t* a = acc.base + ((size_t)p * acc.cap + t) * n + k;
    uint64_t s = *a;
    for (uint32_t i = 0; i < count; ++i)
      s = add_mod(s, in.base[(size_t)i * in.stride + ((size_t)p * in.cap + t) * n + k], q);
    *a = s;
  }
}

int accumulate_batch(he_ctx* c, CtBatch in, uint32_t count, CtBatch acc, uint32_t level) {
  {
    ProfScope prof(c, "elementwise", 0.0, (double)(count + 2) * 2 * level * c->n * 8);
    k_accumulate<<<grid_for((size_t)2 * level * c->n), 256, 0, c->stream>>>(in, count, acc, level, c->log_n,
                                                                            c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// acc += sum over i < count of tensor(A_i, B_i): the three parts
// (a0 b0, a0 b1 + a1 b0, a1 b1) of each product summed into the three-part
// accumulator acc [3][level][N] (limbs below level of A and B).  A CTA of
// kTaSlices warps takes 32 consecutive coefficients (one per lane, coalesced
// loads); warp w sums the products of ciphertexts w, w + kTaSlices, ..., and
// the slices' sums are added in shared memory (modular sums are exact, so
// the order does not change a residue).
constexpr int kTaSlices = 8;

__global__ void __launch_bounds__(32 * kTaSlices) k_tensor_acc(CtBatch A, CtBatch B, uint32_t count, uint64_t* acc,
                                                             uint32_t level, int log_n, const PrimeDev* primes) {
  __shared__ uint64_t part[3][kTaSlices][32];
  const uint32_t n = 1u << log_n;
  const uint32_t lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const size_t total = (size_t)level * n;
  for (size_t base = (size_t)blockIdx.x * 32; base < total; base += (size_t)gridDim.x * 32) {
    const size_t g = base + lane;
    const bool in = g < total;
    uint64_t s0 = 0, s1 = 0, s2 = 0;
    uint32_t k = 0, t = 0;
    PrimeDev pr{};
    if (in) {
      k = (uint32_t)(g & (n - 1));
      t = (uint32_t)(g >> log_n);
      pr = primes[t];
      for (uint32_t i = slice; i < count; i += kTaSlices) {
        const uint64_t x0 = __ldg(cpoly(A, i, 0, t, n) + k), x1 = __ldg(cpoly(A, i, 1, t, n) + k);
        const uint64_t y0 = __ldg(cpoly(B, i, 0, t, n) + k), y1 = __ldg(cpoly(B, i, 1, t, n) + k);
        s0 = add_mod(s0, mul_mod(x0, y0, pr), pr.q);
        s1 = add_mod(s1, add_mod(mul_mod(x0, y1, pr), mul_mod(x1, y0, pr), pr.q), pr.q);
        s2 = add_mod(s2, mul_mod(x1, y1, pr), pr.q);
      }
    }
    part[0][slice][lane] = s0;
    part[1][slice][lane] = s1;
    part[2][slice][lane] = s2;
    __syncthreads();
    if (in && slice < 3) {  // warps 0, 1, 2 finish parts 0, 1, 2
      uint64_t* ap = acc + (size_t)slice * level * n + (size_t)t * n + k;
      uint64_t s = *ap;
#pragma unroll
      for (int w = 0; w < kTaSlices; ++w) s = add_mod(s, part[slice][w][lane], pr.q);
      *ap = s;
    }
    __syncthreads();
  }
}

int tensor_acc_batch(he_ctx* c, CtBatch A, CtBatch B, uint32_t count, uint64_t* acc, uint32_t level) {
  {
    ProfScope prof(c, "tensor", 4.0 * count * level * c->n, (double)(4 * count + 6) * level * c->n * 8);
    const size_t groups = ((size_t)level * c->n + 31) / 32;  // CTAs of 32 coefficients
    k_tensor_acc<<<(unsigned)std::min<size_t>(groups, 152 * 32), 32 * kTaSlices, 0, c->stream>>>(
        A, B, count, acc, level, c->log_n, c->d_primes);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// Relinearise three-part ciphertexts D (count x [3][level][N] at d_stride)
// and rescale, as one division by P q_{level-1} of P (d0, d1) + the inner
// products of d2 (out: level - 1 limbs).
int relin_rescale_batch(he_ctx* c, uint64_t* D, uint64_t d_stride, uint32_t level, uint32_t count, CtBatch out,
                        Arena& ar) {
  const CtBatch D01{D, d_stride, level, 0};
  return keyswitch_batch(c, D + (size_t)2 * level * c->n, d_stride, level, count, c->d_rlk, D01, 2, out, ar, 0,
                         true);
}

}  // namespace he
