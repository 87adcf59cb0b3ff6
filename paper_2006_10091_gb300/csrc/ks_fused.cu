// ks_fused.cu -- entry points of the fused key-switching kernels (kernels in
// ks_fused.cuh, instantiated per ring size in ks_fused_n12.cu .. n16.cu).
#include <algorithm>

#include "ks_fused.cuh"

namespace he {

// The arguments shared by the fused ModUp and row kernels.
static KsFusedArgs ks_args(he_ctx* c, const uint64_t* d, uint64_t d_stride, const uint64_t* d2c, uint64_t* ext,
                           uint64_t* acc, const uint64_t* evk, uint32_t level, uint64_t gal, bool half) {
  KsFusedArgs a;
  a.gal = gal;
  a.half = half ? 1 : 0;
  a.itw = reinterpret_cast<const ulonglong2*>(c->d_itw);
  a.d = d;
  a.d2c = d2c;
  a.ext = ext;
  a.acc = acc;
  a.evk = evk;
  a.d_stride = d_stride;
  a.level = level;
  a.alpha = (uint32_t)c->alpha;
  a.beta = (level + a.alpha - 1) / a.alpha;
  a.L = (uint32_t)c->L;
  a.np = (uint32_t)c->np;
  a.nt = level + a.alpha;
  a.primes = c->d_primes;
  a.tw = reinterpret_cast<const ulonglong2*>(c->d_tw);
  a.consts = c->d_modup;
  for (uint32_t j = 0; j < a.beta; ++j) {
    const ModUpConst& mc = c->modup[level][j];
    a.lo[j] = mc.lo;
    a.cnt[j] = mc.cnt;
    a.off[j] = mc.off;
  }
  return a;
}

// Inverse of an odd Galois element modulo 2N (Newton's iteration for the
// inverse modulo 2^64, then reduced).
static uint64_t gal_inverse(uint64_t gal, int log_n) {
  uint64_t x = gal;  // correct to 3 bits
  for (int i = 0; i < 5; ++i) x *= 2 - gal * x;
  return x & ((2ull << log_n) - 1);
}

bool ks_rot_fits(const he_ctx* c, uint32_t level, uint32_t nrot) {
  if (!ks_fusable(c)) return false;
  // rows moved between CTAs are summed as nrot unreduced residues in 64 bits
  uint64_t qmax = 0;
  for (uint32_t t = 0; t < level; ++t) qmax = std::max(qmax, c->q[t]);
  for (uint32_t u = 0; u < (uint32_t)c->alpha; ++u) qmax = std::max(qmax, c->q[c->L + u]);
  if (qmax > ~0ull / nrot) return false;
  const uint32_t beta = (level + (uint32_t)c->alpha - 1) / (uint32_t)c->alpha;
  size_t smem = 0;
  switch (c->log_n) {
    case 12: smem = ks_rot_smem_n12(c, beta); break;
    case 13: smem = ks_rot_smem_n13(c, beta); break;
    case 14: smem = ks_rot_smem_n14(c, beta); break;
    case 15: smem = ks_rot_smem_n15(c, beta); break;
    default: smem = ks_rot_smem_n16(c, beta); break;
  }
  return smem <= kRotSmemMax;
}

// ModUp -> NTT -> the summed inner products of every rotation of a hoisted
// rotate-and-sum, fused, into one accumulator; *unreduced when it holds sums
// of rs.n residues (the rotations moved rows between CTAs).
int ks_rot(he_ctx* c, const uint64_t* d, uint64_t d_stride, const uint64_t* d2c, uint64_t* ext, uint64_t* acc,
           const RotSet& rs, uint32_t level, uint32_t count, bool half, bool* handled, bool* unreduced,
           uint64_t in_gal, const uint64_t* c0, uint64_t c0_stride, bool* c0_added) {
  *handled = false;
  *unreduced = false;
  if (c0_added) *c0_added = false;
  if (!ks_rot_fits(c, level, rs.n)) return HE_OK;
  KsRotArgs ra;
  ra.k = ks_args(c, d, d_stride, d2c, ext, acc, nullptr, level, in_gal, half);
  ra.nrot = rs.n;
  ra.count = count;
  ra.c0 = c0;
  ra.c0_stride = c0_stride;
  // the summed path adds nrot * beta products below q^2 in 128 bits (the
  // other path beta of them)
  uint32_t bits = 0;
  for (uint32_t t = 0; t < level; ++t) bits = std::max(bits, (uint32_t)(64 - __builtin_clzll(c->q[t])));
  for (uint32_t u = 0; u < (uint32_t)c->alpha; ++u) bits = std::max(bits, (uint32_t)(64 - __builtin_clzll(c->q[c->L + u])));
  const uint32_t nprod = rs.n * ((level + (uint32_t)c->alpha - 1) / (uint32_t)c->alpha);
  ra.closed = 2 * bits + (32 - __builtin_clz(nprod)) <= 128 ? 1 : 0;
  for (uint32_t r = 0; r < rs.n; ++r) {
    ra.gal[r] = rs.gal[r];
    ra.gal_inv[r] = gal_inverse(rs.gal[r], c->log_n);
    ra.evk[r] = rs.evk[r];
  }
  int closed = 0, rc;
  switch (c->log_n) {
    case 12: rc = ks_rot_n12(c, ra, count, handled, &closed); break;
    case 13: rc = ks_rot_n13(c, ra, count, handled, &closed); break;
    case 14: rc = ks_rot_n14(c, ra, count, handled, &closed); break;
    case 15: rc = ks_rot_n15(c, ra, count, handled, &closed); break;
    default: rc = ks_rot_n16(c, ra, count, handled, &closed); break;
  }
  *unreduced = *handled && !(closed & 1);
  if (c0_added) *c0_added = *handled && (closed & 2);
  return rc;
}

}  // namespace he

namespace he {

// Conversion -> NTT -> combine of keyswitch_batch's ModDown, fused.  acc's P
// limbs must already be in coefficient form.  Sets *handled when N has
// compiled shapes (the same ones as the NTT and ModUp).
static int md_dispatch(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled);

int md_fused_gals(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, int add_mode,
                  const uint64_t* gals, uint32_t n_gal, CtBatch out, uint32_t level, uint32_t count, bool half,
                  bool* handled) {
  *handled = false;
  if (!ks_fusable(c) || n_gal > HE_MAX_ROT) {
    if (half) return fail(HE_EINVAL, "md_fused: half-transformed input needs the fused kernels");
    return HE_OK;
  }
  const uint32_t nt = level + (uint32_t)c->alpha;
  MdArgs a;
  a.n_gal = n_gal;
  for (uint32_t g = 0; g < n_gal; ++g) a.gal[g] = gals[g];
  a.yP = acc + (size_t)level * c->n;
  a.yp_stride = acc_stride;
  a.yp_pstride = (uint64_t)nt * c->n;
  a.accq = CtBatch{const_cast<uint64_t*>(acc), acc_stride, nt, 0};
  for (uint32_t u = 0; u < (uint32_t)c->alpha; ++u) a.spr[u] = (uint32_t)c->L + u;
  a.kind = 0;
  a.addw = nullptr;
  a.conv = conv;
  a.add = add;
  a.out = out;
  a.has_add = add_mode;
  a.level = level;
  a.alpha = (uint32_t)c->alpha;
  a.L = (uint32_t)c->L;
  a.primes = c->d_primes;
  a.tw = reinterpret_cast<const ulonglong2*>(c->d_tw);
  a.itw = reinterpret_cast<const ulonglong2*>(c->d_itw);
  a.half = half;
  a.md = c->d_moddown;
  return md_dispatch(c, a, count, handled);
}

int md_fused(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, int add_mode,
             uint64_t add_gal, CtBatch out, uint32_t level, uint32_t count, bool half, bool* handled) {
  return md_fused_gals(c, acc, acc_stride, conv, add, add_mode, &add_gal, add_gal ? 1 : 0, out, level, count, half,
                       handled);
}

// The ModDown of a multiplication's relinearisation merged with its rescale:
// acc's limbs level-1 .. level+alpha-1 (q_{level-1}, then the special primes;
// q_{level-1}'s already holds acc + P d) in coefficient form are converted
// to the level-1 remaining limbs, and out_t = (acc_t - NTT(conv_t)) (P q_{level-1})^-1
// + d_t q_{level-1}^-1 (the addend d on both parts).
int md_fused_rescale(he_ctx* c, const uint64_t* acc, uint64_t acc_stride, uint64_t* conv, CtBatch add, CtBatch out,
                     uint32_t level, uint32_t count, bool half, bool* handled) {
  *handled = false;
  if (!ks_fusable(c) || !c->d_mdrs || level < 2) {
    if (half) return fail(HE_EINVAL, "md_fused: half-transformed input needs the fused kernels");
    return HE_OK;
  }
  const uint32_t nt = level + (uint32_t)c->alpha, lo = level - 1;
  MdArgs a;
  a.n_gal = 0;
  a.yP = acc + (size_t)lo * c->n;
  a.yp_stride = acc_stride;
  a.yp_pstride = (uint64_t)nt * c->n;
  a.accq = CtBatch{const_cast<uint64_t*>(acc), acc_stride, nt, 0};
  a.spr[0] = lo;
  for (uint32_t u = 0; u < (uint32_t)c->alpha; ++u) a.spr[1 + u] = (uint32_t)c->L + u;
  a.kind = 2;
  a.addw = c->d_rescale + (size_t)lo * c->L * 2;
  a.conv = conv;
  a.add = add;
  a.out = out;
  a.has_add = 2;
  a.level = lo;
  a.alpha = (uint32_t)c->alpha + 1;
  a.L = (uint32_t)c->L;
  a.primes = c->d_primes;
  a.tw = reinterpret_cast<const ulonglong2*>(c->d_tw);
  a.itw = reinterpret_cast<const ulonglong2*>(c->d_itw);
  a.half = half;
  a.md = c->d_mdrs + (size_t)level * c->mdrs_words;
  return md_dispatch(c, a, count, handled);
}

// Rescale by q_{l-1} as a ModDown by that one prime, fused the same way.
// last: the dropped limb of both parts in coefficient form, count x [2][N].
int rs_fused(he_ctx* c, CtBatch in, const uint64_t* last, uint64_t* conv, CtBatch out, uint32_t level,
             uint32_t count, bool half, bool* handled) {
  *handled = false;
  if (!ks_fusable(c) || level < 2) {
    if (half) return fail(HE_EINVAL, "md_fused: half-transformed input needs the fused kernels");
    return HE_OK;
  }
  const uint32_t lt = level - 1;
  MdArgs a;
  a.n_gal = 0;
  a.yP = last;
  a.yp_stride = 2ull * c->n;
  a.yp_pstride = c->n;
  a.accq = in;
  a.spr[0] = lt;
  a.kind = 1;
  a.addw = nullptr;
  a.conv = conv;
  a.add = out;
  a.out = out;
  a.has_add = 0;
  a.level = lt;
  a.alpha = 1;
  a.L = (uint32_t)c->L;
  a.primes = c->d_primes;
  a.tw = reinterpret_cast<const ulonglong2*>(c->d_tw);
  a.itw = reinterpret_cast<const ulonglong2*>(c->d_itw);
  a.half = half;
  a.md = c->d_rescale_md + (size_t)lt * c->rescale_md_words;
  return md_dispatch(c, a, count, handled);
}

static int md_dispatch(he_ctx* c, const MdArgs& a, uint32_t count, bool* handled) {
  switch (c->log_n) {
    case 12: return md_fused_n12(c, a, count, handled);
    case 13: return md_fused_n13(c, a, count, handled);
    case 14: return md_fused_n14(c, a, count, handled);
    case 15: return md_fused_n15(c, a, count, handled);
    default: return md_fused_n16(c, a, count, handled);
  }
}

}  // namespace he

namespace he {

// Whether the fused ModDown (or rescale) with nd dropped limbs runs, so that
// its conversion kernel can finish the dropped limbs' inverse transform
// (the caller then runs only its row pass).
bool md_half_ok(const he_ctx* c, uint32_t nd) {
  if (!ks_fusable(c)) return false;
  size_t smem = 0;
  switch (c->log_n) {
    case 12: smem = md_col_smem_n12(c, nd); break;
    case 13: smem = md_col_smem_n13(c, nd); break;
    case 14: smem = md_col_smem_n14(c, nd); break;
    case 15: smem = md_col_smem_n15(c, nd); break;
    default: smem = md_col_smem_n16(c, nd); break;
  }
  return smem <= kModupAllSmem;
}

// Whether the fused key switch at this level converts each digit in one CTA
// (then it can finish the inverse transform of its input itself).
bool ks_converts_per_digit(const he_ctx* c, uint32_t level) {
  if (!ks_fusable(c)) return false;
  const uint32_t alpha = (uint32_t)c->alpha, beta = (level + alpha - 1) / alpha;
  uint32_t cnt[HE_MAX_PRIMES];
  for (uint32_t j = 0; j < beta; ++j) cnt[j] = c->modup[level][j].cnt;
  size_t smem = 0;
  switch (c->log_n) {
    case 12: smem = ks_all_smem_n12(c, beta, cnt); break;
    case 13: smem = ks_all_smem_n13(c, beta, cnt); break;
    case 14: smem = ks_all_smem_n14(c, beta, cnt); break;
    case 15: smem = ks_all_smem_n15(c, beta, cnt); break;
    default: smem = ks_all_smem_n16(c, beta, cnt); break;
  }
  return smem <= kModupAllSmem;
}

}  // namespace he
