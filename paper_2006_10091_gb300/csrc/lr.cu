// lr.cu -- the encrypted logistic-regression gradient step of a worker
// (Sec. 4: Eq. 5-8 with a Table 2 polynomial; Algorithm 1 line 7).
//
// Packing: each data ciphertext holds g samples interleaved, slot g*f + s =
// y_s * x_{s,f}; W holds w_f in slots g*f + s for every s.  Because slot
// rotations are cyclic over all N/2 slots, summing rotations by g, 2g, ...,
// N/4 leaves in every slot g*f + s the full inner product m_s = w . z_s of
// its own sample, so no mask is needed before the polynomial.  After the
// polynomial, rotations by 1, 2, ..., g/2 collect the per-feature sum on
// slots = 0 mod g, a 0/1 mask keeps those, and rotations by -1, ..., -g/2
// copy it back to all g slots.
//
// Op sequence and scale plan (doubles, same order as the CPU oracle; l0 the
// input level, q[i] the limb primes):
//   U  = HMult(Z_k, W)                      sU = sZ*sW/q[l0-1]
//   M  = U + rot(U, g) + ... (log2 F doublings)
//   T  = HMult(M, M)                        sT = sU*sU/q[l0-2]
//   sS = ((sW*q[l0-5])*q[l0-4]) / (mask_scale*sZ)
//   A  = rescale(M * round(c3*lr*sigA)),    sigA = ((sS*q[l0-3])/sT * q[l0-2])/sU
//   C  = HMult(T, A)
//   B  = rescale(M * round(c1*lr*sigB)),    sigB = (sS*q[l0-2])/sU, dropped one level
//   Q  = rescale(T * round(c2*lr*sigQ)),    sigQ = (sS*q[l0-3])/sT   (c2 != 0)
//   S  = C + B (+ Q) + round(c0*lr*scale(C))
//   G  = sum_k HMult(S, drop(Z_k))
//   H  = G + rot(G, 1) + ... ;  R = rescale(H (x) mask) ;  R += rot(R, -1) + ...
//   W' = drop(W) + R                        (scale sW, level l0-5)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "he_ops.h"

namespace he {

static bool scales_eq(double a, double b) { return fabs(a / b - 1.0) < ldexp(1.0, -40); }

static int ilog2u(uint32_t v) {
  int r = 0;
  while ((1u << r) < v) ++r;
  return r;
}

// Device coefficients of the 0/1 mask (1 on slots = 0 mod g) at mask_scale,
// encoded once per (g, scale) and kept in the context.
static int lr_mask(he_ctx* c, uint32_t g, double ms, const int64_t** out) {
  auto key = std::make_pair(g, ms);
  auto it = c->lr_masks.find(key);
  if (it != c->lr_masks.end()) {
    *out = it->second;
    return HE_OK;
  }
  const size_t n = c->n, nh = n / 2;
  int64_t* d = nullptr;
  HE_CUDA(cudaStreamSynchronize(c->stream));  // the workspace may still be in use
  HE_CUDA(cudaMalloc(&d, sizeof(int64_t) * n));
  c->lr_masks[key] = d;
  HE_TRY(ws_reserve(c, sizeof(double2) * 2 * n + sizeof(double) * nh + 4096));
  char* w = (char*)c->ws.ptr;
  double2* fft = (double2*)w;
  double* z = (double*)(fft + 2 * n);
  int* ovf = (int*)(z + nh);
  std::vector<double> host(nh, 0.0);
  for (size_t j = 0; j < nh; j += g) host[j] = 1.0;
  HE_CUDA(cudaMemcpy(z, host.data(), sizeof(double) * nh, cudaMemcpyHostToDevice));
  HE_CUDA(cudaMemset(ovf, 0, sizeof(int)));
  HE_TRY(encode_dev(c, z, nh, ms, d, fft, ovf));
  int flag = 0;
  HE_CUDA(cudaMemcpyAsync(&flag, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  if (flag) return fail(HE_EINVAL, "mask coefficient beyond int64");
  *out = d;
  return HE_OK;
}

static bool to_int(double v, int64_t* out) {
  if (!(fabs(v) < 9.2e18)) return false;
  *out = (int64_t)llround(v);
  return true;
}

struct LrPlan {
  uint32_t l0, g, logF, logg;
  double sZ, sW, sU, sT, sS, sigA, sigB, sigQ, sA_out, sC, sB, sQ, sG, sR;
  int64_t kA, kB, kQ, k0;
  bool has_c2;
};

static int lr_plan(const he_ctx* c, uint32_t l0, double sZ, double sW, const he_lr_config* cfg, LrPlan* p) {
  const std::vector<uint64_t>& q = c->q;
  p->l0 = l0;
  p->g = cfg->g;
  p->logF = (uint32_t)ilog2u((uint32_t)(c->n / 2) / cfg->g);
  p->logg = (uint32_t)ilog2u(cfg->g);
  p->sZ = sZ;
  p->sW = sW;
  const double lr = cfg->lr, ms = cfg->mask_scale;
  p->sU = sZ * sW / (double)q[l0 - 1];
  p->sT = p->sU * p->sU / (double)q[l0 - 2];
  p->sS = ((sW * (double)q[l0 - 5]) * (double)q[l0 - 4]) / (ms * sZ);
  const double sA = (p->sS * (double)q[l0 - 3]) / p->sT;
  p->sigA = (sA * (double)q[l0 - 2]) / p->sU;
  p->sigB = (p->sS * (double)q[l0 - 2]) / p->sU;
  p->sigQ = (p->sS * (double)q[l0 - 3]) / p->sT;
  if (!to_int(cfg->coeffs[3] * lr * p->sigA, &p->kA) || !to_int(cfg->coeffs[1] * lr * p->sigB, &p->kB) ||
      !to_int(cfg->coeffs[2] * lr * p->sigQ, &p->kQ))
    return fail(HE_EINVAL, "polynomial coefficient beyond int64 at its scale");
  p->sA_out = (p->sU * p->sigA) / (double)q[l0 - 2];
  p->sC = p->sT * p->sA_out / (double)q[l0 - 3];
  p->sB = (p->sU * p->sigB) / (double)q[l0 - 2];
  if (!scales_eq(p->sC, p->sB)) return fail(HE_ESCALE, "linear term scale mismatch");
  p->has_c2 = cfg->coeffs[2] != 0.0;
  p->sQ = (p->sT * p->sigQ) / (double)q[l0 - 3];
  if (p->has_c2 && !scales_eq(p->sC, p->sQ)) return fail(HE_ESCALE, "quadratic term scale mismatch");
  if (!to_int(cfg->coeffs[0] * lr * p->sC, &p->k0)) return fail(HE_EINVAL, "constant beyond int64");
  p->sG = p->sC * sZ / (double)q[l0 - 4];
  p->sR = (p->sG * ms) / (double)q[l0 - 5];
  if (!scales_eq(p->sR, sW)) return fail(HE_ESCALE, "output scale mismatch");
  return HE_OK;
}

// Per-ciphertext words of the circuit's intermediates at input level l0.
static size_t lr_ct_words(const he_ctx* c, uint32_t l0) {
  const size_t n = c->n;
  // U, T, A, C, B, Q, Gk, tmp, Zc copy
  return n * 2 * ((l0 - 1) + (l0 - 2) + (l0 - 2) + (l0 - 3) + (l0 - 2) + (l0 - 3) + (l0 - 4) + (l0 - 1) + l0);
}

static size_t lr_op_words(const he_ctx* c, uint32_t l0, uint32_t chunk) {
  size_t w = mul_words(c, l0, chunk, true);
  w = std::max(w, rot_words(c, l0 - 1, chunk));
  w = std::max(w, rescale_words(c, l0 - 1, chunk));
  return w + 64;
}

}  // namespace he

using namespace he;

extern "C" int he_lr_gradient_step(he_ctx* c, const he_ct* Z, size_t nZ, const he_ct* W, const he_lr_config* cfg,
                                   he_ct* W_out) {
  if (!c || !Z || !W || !cfg || !W_out || !W_out->data || !W->data) return fail(HE_EINVAL, "he_lr_gradient_step: null argument");
  if (nZ == 0) return fail(HE_EINVAL, "he_lr_gradient_step: no data ciphertexts");
  const uint32_t n = c->n;
  const uint32_t l0 = W->level;
  if (l0 < 6 || l0 > (uint32_t)c->L || W->cap < l0) return fail(HE_ELEVEL, "the step needs inputs at level >= 6");
  for (size_t k = 0; k < nZ; ++k) {
    if (!Z[k].data || Z[k].level != l0 || Z[k].cap < l0) return fail(HE_EINVAL, "data and weights must share one level");
    if ((uintptr_t)Z[k].data & 15) return fail(HE_EINVAL, "ciphertext data must be 16-byte aligned");
    if (!scales_eq(Z[k].scale, Z[0].scale)) return fail(HE_ESCALE, "data ciphertexts at different scales");
  }
  const uint32_t g = cfg->g;
  if (g < 1 || (g & (g - 1)) || g > n / 2) return fail(HE_EINVAL, "g must be a power of two <= N/2");
  if (!(cfg->mask_scale > 0.0)) return fail(HE_EINVAL, "mask_scale must be positive");
  if (W_out->cap < l0 - 5) return fail(HE_EINVAL, "output capacity too small");
  if (((uintptr_t)W->data & 15) || ((uintptr_t)W_out->data & 15)) return fail(HE_EINVAL, "ciphertext data must be 16-byte aligned");
  LrPlan P;
  HE_TRY(lr_plan(c, l0, Z[0].scale, W->scale, cfg, &P));
  std::vector<uint64_t> gal_in, gal_up, gal_down;
  for (uint32_t t = 0; t < P.logF; ++t) gal_in.push_back(h_galois_elt(c->log_n, (int32_t)(g << t)));
  for (uint32_t t = 0; t < P.logg; ++t) {
    gal_up.push_back(h_galois_elt(c->log_n, (int32_t)(1u << t)));
    gal_down.push_back(h_galois_elt(c->log_n, -(int32_t)(1u << t)));
  }
  for (auto* v : {&gal_in, &gal_up, &gal_down})
    for (uint64_t e : *v)
      if (e != 1 && !galois_key(c, e)) return fail(HE_ENOKEY, "missing Galois key for the step's rotations");
  const int64_t* mask = nullptr;
  HE_TRY(lr_mask(c, g, cfg->mask_scale, &mask));

  // chunk of data ciphertexts processed together
  const size_t per = (lr_ct_words(c, l0) + lr_op_words(c, l0, 1)) * sizeof(uint64_t);
  size_t chunk = std::max<size_t>(1, c->chunk_bytes / per);
  chunk = std::min(chunk, nZ);
  const size_t fixed = (size_t)n * 2 * ((l0 - 4) + 2 * (l0 - 4)) + lr_op_words(c, l0 - 4, 1) + 64;
  const size_t total_words = fixed + chunk * lr_ct_words(c, l0) + lr_op_words(c, l0, (uint32_t)chunk) + 1024;
  HE_TRY(ws_reserve(c, total_words * sizeof(uint64_t)));
  Arena base;
  base.base = (char*)c->ws.ptr;
  base.size = c->ws.size;
  const size_t C = chunk;
  auto ctbuf = [&](size_t count, uint32_t cap) -> CtBatch {
    uint64_t* p = base.take<uint64_t>(count * 2 * cap * n);
    return CtBatch{p, (uint64_t)2 * cap * n, cap, 0};
  };
  CtBatch G = ctbuf(1, l0 - 4), H1 = ctbuf(1, l0 - 4), R = ctbuf(1, l0 - 4);
  CtBatch U = ctbuf(C, l0 - 1), T = ctbuf(C, l0 - 2), A = ctbuf(C, l0 - 2), Cc = ctbuf(C, l0 - 3);
  CtBatch B = ctbuf(C, l0 - 2), Q = ctbuf(C, l0 - 3), Gk = ctbuf(C, l0 - 4), Tmp = ctbuf(C, l0 - 1);
  CtBatch Zcopy = ctbuf(C, l0);
  if (!G.base || !Zcopy.base) return fail(HE_ENOMEM, "step scratch too small");
  Arena ops;
  ops.base = base.base + base.off;
  ops.size = base.size - base.off;
  auto fresh = [&]() {
    ops.off = 0;
    return ops;
  };
  HE_CUDA(cudaMemsetAsync(G.base, 0, sizeof(uint64_t) * 2 * (l0 - 4) * n, c->stream));
  CtBatch Zall;
  const bool zu = uniform_view(Z, nZ, &Zall);
  const CtBatch Wb{W->data, 0, W->cap, 0};
  for (size_t k0 = 0; k0 < nZ; k0 += C) {
    const uint32_t m = (uint32_t)std::min(C, nZ - k0);
    CtBatch Zc;
    if (zu) {
      Zc = Zall;
      Zc.base += k0 * Zall.stride;
    } else {
      Zc = Zcopy;
      for (uint32_t i = 0; i < m; ++i) {
        CtBatch src{Z[k0 + i].data, 0, Z[k0 + i].cap, 0}, dst = Zcopy;
        dst.base += (size_t)i * Zcopy.stride;
        HE_TRY(copy_batch(c, src, dst, l0, 1));
      }
    }
    Arena ar = fresh();
    // U = Z_k * W, then the rotate-and-sum over the F feature positions
    HE_TRY(mul_relin_batch(c, Zc, Wb, l0, m, U, true, ar));
    for (uint32_t t = 0; t < P.logF; ++t) {
      ar = fresh();
      HE_TRY(rotate_batch(c, U, l0 - 1, m, gal_in[t], Tmp, ar));
      HE_TRY(addsub_batch(c, U, Tmp, U, 0, l0 - 1, m));
    }
    // T = M^2; A = c3 M; C = T A
    ar = fresh();
    HE_TRY(mul_relin_batch(c, U, U, l0 - 1, m, T, true, ar));
    HE_TRY(mul_int_batch(c, U, Tmp, P.kA, l0 - 1, m));
    ar = fresh();
    HE_TRY(rescale_batch(c, Tmp, l0 - 1, m, A, ar));
    ar = fresh();
    HE_TRY(mul_relin_batch(c, T, A, l0 - 2, m, Cc, true, ar));
    // B = c1 M (dropped to l0-3) ; Q = c2 M^2
    HE_TRY(mul_int_batch(c, U, Tmp, P.kB, l0 - 1, m));
    ar = fresh();
    HE_TRY(rescale_batch(c, Tmp, l0 - 1, m, B, ar));
    HE_TRY(addsub_batch(c, Cc, B, Cc, 0, l0 - 3, m));
    if (P.has_c2) {
      HE_TRY(mul_int_batch(c, T, Tmp, P.kQ, l0 - 2, m));
      ar = fresh();
      HE_TRY(rescale_batch(c, Tmp, l0 - 2, m, Q, ar));
      HE_TRY(addsub_batch(c, Cc, Q, Cc, 0, l0 - 3, m));
    }
    HE_TRY(add_int_batch(c, Cc, Cc, P.k0, l0 - 3, m));
    // G_k = S * Z_k, accumulated into G
    ar = fresh();
    HE_TRY(mul_relin_batch(c, Cc, Zc, l0 - 3, m, Gk, true, ar));
    HE_TRY(accumulate_batch(c, Gk, m, G, l0 - 4));
  }
  // per-feature sum over the g samples, mask, replicate
  for (uint32_t t = 0; t < P.logg; ++t) {
    Arena ar = fresh();
    HE_TRY(rotate_batch(c, G, l0 - 4, 1, gal_up[t], H1, ar));
    HE_TRY(addsub_batch(c, G, H1, G, 0, l0 - 4, 1));
  }
  {
    Arena ar = fresh();
    HE_TRY(mul_plain_dev(c, G, mask, H1, l0 - 4, 1, ar));
    ar = fresh();
    HE_TRY(rescale_batch(c, H1, l0 - 4, 1, R, ar));
  }
  for (uint32_t t = 0; t < P.logg; ++t) {
    Arena ar = fresh();
    HE_TRY(rotate_batch(c, R, l0 - 5, 1, gal_down[t], H1, ar));
    HE_TRY(addsub_batch(c, R, H1, R, 0, l0 - 5, 1));
  }
  const CtBatch Wo{W_out->data, 0, W_out->cap, 0};
  HE_TRY(addsub_batch(c, Wb, R, Wo, 0, l0 - 5, 1));
  W_out->level = l0 - 5;
  W_out->scale = W->scale;
  return HE_OK;
}
